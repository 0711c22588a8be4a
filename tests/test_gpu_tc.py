"""Tensor-core (tcgen05 + TMA, BF16 operands) path against the FP64 oracle (needs a GB300)."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import RTOL, grad_agreement, grad_groups, oracle_setup, rel_err, repack

pytestmark = pytest.mark.gpu

# BF16 operands (8-bit significand) with FP32 accumulation: the bound at fixed alpha, beta moves by
# a few units of 2^-9 relative to the scale of the terms it sums.  Tolerances are per network, about
# 3x the largest error measured on a GB300 (max |lb - oracle| / median |oracle|):
BF16_TOL = {
    "mlp_small": 4.5e-2,      # measured 1.0e-2 and 1.4e-2 (16-32-32-4: bounds near 0, few terms per sum)
    "mlp_784": 1.5e-3,        # measured 4.4e-4 (200 subdomains) and 4.9e-4 (the full 1024)
    "mlp_784_mixed": 1.5e-3,  # measured 4.1e-4 (3 properties), 5.1e-4 (64 properties)
    "tiny": 3.5e-2,           # measured 1.0e-2
    "tiny_odd": 2e-2,         # measured 6.2e-3
    "tiny_s3": 2e-2,          # measured 5.8e-3
    "tiny_tma": 6e-3,         # measured 1.7e-3
    "c3": 3e-3,               # conv_small: measured 7.9e-4 (24 subdomains), 1.0e-3 at full size
    "conv_small": 3e-3,
    "conv_big": 6e-5,         # measured 1.9e-5 at full size
    "wide_mlp": 4.5e-2,       # measured 1.4e-2
    "conv_limits": 1e-3,      # measured 3.0e-4
}
# BF16 gradients entry by entry, per hidden layer: the share of entries within GRAD_TOL of the
# oracle's (relative to |g| plus 1 % of the layer's largest |g|), and the cosine between the layer's
# gradient vectors.  BF16 rounding of x*, h and the stash moves zhat by a few 2^-9 of sum |W||h|,
# which is large against |zhat| where zhat is near 0, and can flip a relaxation choice where A or
# A^(0) is near 0: hence a share, not every entry.  Measured on a GB300 over every case below:
# share >= 0.9365 (the first layer's dbeta of conv_small; 0.98 or more elsewhere) and cosine
# >= 0.99891.  A zeroed or sign-flipped layer, or wrong entries on a few percent of the rows,
# fails both.
GRAD_TOL, GRAD_SHARE, GRAD_COS = 0.25, 0.9, 0.997


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x, np.float32)).cuda()


def _gpu(pb, props, batch):
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    return net, dom, bc.DeviceBatch.from_host(batch)


def _scale(ref):
    return max(float(np.median(np.abs(ref))), 1.0)


@pytest.mark.parametrize("which", ["small", "784"])
def test_bf16_bound_close_to_oracle(which):
    if which == "small":
        pb = wl.problem_mlp_small()
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 64, 0, 4, 1)
    else:
        pb = wl.problem_mlp_784()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [200], 12, 3)
    a, b = wl.random_alpha_beta(batch, 4, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    assert bc.status(net) == 0
    ref = O.bound(onet, props, batch, a, b)
    err = np.abs(lb - ref) / _scale(ref)
    print("bf16 bound %s: max err / median|lb| = %.3e" % (which, err.max()))
    assert np.all(np.isfinite(lb))
    assert err.max() <= BF16_TOL["mlp_small" if which == "small" else "mlp_784"]


def test_bf16_ragged_rows_and_multi_property():
    """R not a multiple of the 64-row tile; rows of one tile from different properties."""
    pb = wl.problem_mlp_784(n_props=3)
    onet = O.OracleNet(pb.layers, pb.C)
    l, u = O.root_bounds(onet, pb.x_lo, pb.x_hi)
    l, u = l.astype(np.float32), u.astype(np.float32)
    unst = [np.nonzero(O.unstable_mask(l[p], u[p]))[0] for p in range(pb.P)]
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
    batch = wl.random_batch(pb, unst, 37, 0, 6, 8, props=np.arange(37) % 3)
    a, b = wl.random_alpha_beta(batch, 5, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    ref = O.bound(onet, props, batch, a, b)
    assert bc.status(net) == 0
    err = (np.abs(lb - ref) / _scale(ref)).max()
    print("bf16 bound ragged/multi-property: max err / median|lb| = %.3e" % err)
    assert err <= BF16_TOL["mlp_784_mixed"]


def _check_grad(pb, onet, props, batch, da, dbeta, da_ref, db_ref, tag):
    """Entry-by-entry agreement of a BF16 gradient with the oracle's, per hidden layer."""
    la, lb_ = grad_groups(onet, batch, props)
    for kind, g, gr, lay in (("dalpha", da, da_ref, la), ("dbeta", dbeta, db_ref, lb_)):
        for i, (share, cos, n) in grad_agreement(g, gr, lay, GRAD_TOL).items():
            print("bf16 gradient %s %s layer %d: %d entries, share within tol %.4f, cosine %.6f"
                  % (tag, kind, i, n, share, cos))
            if n >= 20:
                assert share >= GRAD_SHARE and cos >= GRAD_COS, (tag, kind, i, share, cos)


@pytest.mark.parametrize("which", ["small", "784", "mixed"])
def test_bf16_gradient_close_to_oracle(which):
    """Adjoint pass of the fused kernel: layers narrower than an M chunk (small), full chunks
    (784), and tiles whose rows come from several properties with a ragged last tile (mixed)."""
    if which == "small":
        pb = wl.problem_mlp_small()
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 64, 0, 4, 1)
    elif which == "784":
        pb = wl.problem_mlp_784()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [64], 12, 9)
    else:
        pb = wl.problem_mlp_784(n_props=3)
        onet = O.OracleNet(pb.layers, pb.C)
        l, u = O.root_bounds(onet, pb.x_lo, pb.x_hi)
        l, u = l.astype(np.float32), u.astype(np.float32)
        unst = [np.nonzero(O.unstable_mask(l[p], u[p]))[0] for p in range(pb.P)]
        props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
        batch = wl.random_batch(pb, unst, 37, 0, 6, 8, props=np.arange(37) % 3)
    a, b = wl.random_alpha_beta(batch, 2, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.BF16)
    assert bc.status(net) == 0
    ref, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    key = {"small": "mlp_small", "784": "mlp_784", "mixed": "mlp_784_mixed"}[which]
    assert (np.abs(lb.cpu().numpy() - ref) / _scale(ref)).max() <= BF16_TOL[key]
    _check_grad(pb, onet, props, batch, da.cpu().numpy(), dbeta.cpu().numpy(), da_ref, db_ref, which)
    lb_fp32, da32, db32 = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.FP32)
    assert np.max(rel_err(lb_fp32.cpu().numpy(), ref)) <= RTOL


@pytest.mark.parametrize("which", ["small", "784"])
def test_bf16_optimize_is_certified_and_tight(which):
    if which == "small":
        pb = wl.problem_mlp_small()
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 64, 0, 4, 1)
    else:
        pb = wl.problem_mlp_784()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [128], 12, 5)
    a0, b0 = wl.initial_alpha_beta(batch)
    net, dom, db = _gpu(pb, props, batch)
    res = {}
    for prec in (bc.BF16, bc.FP32):
        at, bt = _t(a0), _t(b0)
        lb = bc.optimize(net, dom, db, at, bt, bc.OptCfg(precision=prec, certify=True)).cpu().numpy()
        assert bc.status(net) == 0
        a_best, b_best = at.cpu().numpy(), bt.cpu().numpy()
        ref = O.bound(onet, props, batch, a_best, b_best)
        # certified: never above the exact-arithmetic bound at the returned alpha, beta
        assert np.all(lb <= ref + 1e-12 * np.abs(ref))
        assert np.all((a_best >= 0) & (a_best <= 1)) and np.all(b_best >= 0)
        res[prec] = lb
    init = O.bound(onet, props, batch, a0, b0)
    gain32 = np.mean(res[bc.FP32] - init)
    gain16 = np.mean(res[bc.BF16] - init)
    print("mean improvement over the initial bound: FP32 %.4f, BF16 %.4f" % (gain32, gain16))
    assert gain16 >= 0.8 * gain32


def test_batching_64_properties_sampled():
    """The batching workload: 64 properties on the 784-256x6-10 net with log-uniform 16-4096
    subdomains each (about 47k subdomains, 420k rows, tree depths up to 20) in one launch per
    call.  Sampled rows against the oracle, BF16 and FP32; then a short BF16 optimisation whose
    certified bounds stay below the exact bounds at the returned alpha, beta."""
    pb = wl.problem_mlp_784(n_props=64)
    onet, props, unst = oracle_setup(pb)
    counts = wl.loguniform_counts(64, 16, 4096, 0)
    batch = wl.tree_batch(pb, unst, list(counts), 20, 4)
    a, b = wl.random_alpha_beta(batch, 6, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    U = np.array([len(x) for x in unst])
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(batch.B, 24, replace=False))
    sub, sa, sb = repack(pb, batch, U, idx, a, b)
    ref = O.bound(onet, props, sub, sa, sb).reshape(len(idx), pb.K)
    rows = (idx[:, None] * pb.K + np.arange(pb.K)[None, :])
    lb16 = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    assert bc.status(net) == 0
    assert np.all(np.isfinite(lb16))
    err = (np.abs(lb16[rows] - ref) / _scale(ref)).max()
    print("bf16 batching workload: max err / median|lb| = %.3e" % err)
    assert err <= BF16_TOL["mlp_784_mixed"]
    lb32 = bc.bound(net, dom, db, _t(a), _t(b), bc.FP32).cpu().numpy()
    assert np.max(rel_err(lb32[rows], ref)) <= RTOL
    a0, b0 = wl.initial_alpha_beta(batch)
    at, bt = _t(a0), _t(b0)
    lbc = bc.optimize(net, dom, db, at, bt, bc.OptCfg(iters=3, precision=bc.BF16, certify=True)).cpu().numpy()
    assert bc.status(net) == 0
    _, ra, rb = repack(pb, batch, U, idx, at.cpu().numpy(), bt.cpu().numpy())
    ref_opt = O.bound(onet, props, sub, ra, rb).reshape(len(idx), pb.K)
    assert np.all(lbc[rows] <= ref_opt + 1e-12 * np.abs(ref_opt))


_TINY_CONVS = {
    "tiny": ((2, 6, 6), [(3, 3, 2, 1), (4, 3, 1, 1)]),
    "tiny_odd": ((2, 7, 5), [(3, 3, 2, 1), (4, 4, 2, 1)]),   # odd maps: phases of unequal size
    "tiny_s3": ((2, 9, 8), [(3, 5, 3, 2), (4, 3, 1, 1)]),    # stride 3: nine phases
    # 8 (padded) channels on 16 x 16 and 8 x 8 maps: on the fused-epilogue path every pass reads its
    # operand by unswizzled TMA boxes of one tap each (strided in the stride-2 forward pass)
    "tiny_tma": ((3, 16, 16), [(8, 3, 1, 1), (8, 3, 2, 1)]),
}


def _tiny_conv(which="tiny"):
    shape, convs = _TINY_CONVS[which]
    layers = wl.conv_layers(shape, convs, [8, 4], 3)
    return wl.make_problem("tinyconv", layers, 2, 0.1, 3, 3)


@pytest.mark.parametrize("which", ["tiny", "tiny_odd", "tiny_s3", "tiny_tma", "c3"])
def test_bf16_conv_bound_and_gradient_close_to_oracle(which):
    """Conv layers as BF16 tensor-core GEMMs over an im2col operand, the transposed convolutions
    split into stride phases: tiny nets (channel counts and K far below one tile, strides 1-3,
    odd map sizes, two properties) and the c3 net (4x4 kernels, stride 2)."""
    if which != "c3":
        pb = _tiny_conv(which)
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 24, 0, 4, 1, props=np.arange(24) % 2)
    else:
        pb = wl.problem_conv_small()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [24], 16, 7)
    a, b = wl.random_alpha_beta(batch, 3, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    assert bc.status(net) == 0
    ref = O.bound(onet, props, batch, a, b)
    err = np.abs(lb - ref) / _scale(ref)
    print("bf16 conv bound %s: max err / median|lb| = %.3e" % (which, err.max()))
    assert err.max() <= BF16_TOL[which]
    lbg, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.BF16)
    assert bc.status(net) == 0
    ref_g, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    _check_grad(pb, onet, props, batch, da.cpu().numpy(), dbeta.cpu().numpy(), da_ref, db_ref, "conv " + which)


def test_bf16_conv_optimize_is_certified():
    pb = wl.problem_conv_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.tree_batch(pb, unst, [16], 16, 5)
    a0, b0 = wl.initial_alpha_beta(batch)
    net, dom, db = _gpu(pb, props, batch)
    at, bt = _t(a0), _t(b0)
    lb = bc.optimize(net, dom, db, at, bt, bc.OptCfg(precision=bc.BF16, certify=True)).cpu().numpy()
    assert bc.status(net) == 0
    ref = O.bound(onet, props, batch, at.cpu().numpy(), bt.cpu().numpy())
    assert np.all(lb <= ref + 1e-12 * np.abs(ref))
    init = O.bound(onet, props, batch, a0, b0)
    assert np.mean(lb - init) > 0


def test_bf16_wide_mlp_runs_every_contraction_as_a_tensor_core_gemm():
    """Hidden widths above the fused kernel's 256 (and an odd input width): BF16 takes the
    layer-by-layer path with each fully connected contraction a tcgen05 GEMM (N split into
    tiles of 256, unaligned rows written element by element)."""
    layers = wl.mlp_layers([37, 300, 260, 5], 11)
    pb = wl.make_problem("wide_mlp", layers, 2, 0.05, 4, 11)
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 40, 0, 5, 2, props=np.arange(40) % 2)
    a, b = wl.random_alpha_beta(batch, 5, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    assert bc.status(net) == 0
    ref = O.bound(onet, props, batch, a, b)
    err = np.abs(lb - ref) / _scale(ref)
    print("bf16 wide mlp bound: max err / median|lb| = %.3e" % err.max())
    assert err.max() <= BF16_TOL["wide_mlp"]
    _, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.BF16)
    assert bc.status(net) == 0
    _, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    _check_grad(pb, onet, props, batch, da.cpu().numpy(), dbeta.cpu().numpy(), da_ref, db_ref, "wide mlp")
    a0, b0 = wl.initial_alpha_beta(batch)
    at, bt = _t(a0), _t(b0)
    lbc = bc.optimize(net, dom, db, at, bt, bc.OptCfg(precision=bc.BF16, certify=True)).cpu().numpy()
    assert bc.status(net) == 0
    ref_opt = O.bound(onet, props, batch, at.cpu().numpy(), bt.cpu().numpy())
    assert np.all(lbc <= ref_opt + 1e-12 * np.abs(ref_opt))


LAYER_PATHS = {"layer_epi": bc.N.PATH_LAYER_EPI, "layer_gather": bc.N.PATH_LAYER_GATHER,
               "layer_im2col": bc.N.PATH_LAYER_IM2COL}


@pytest.mark.parametrize("path", list(LAYER_PATHS))
def test_every_layer_path_matches_oracle_on_the_tiny_conv_nets(path):
    """Each BF16 layer path chosen explicitly (GEMM epilogues; gather GEMMs with FP32 kernels between
    them; the im2col buffer in HBM read by TMA): bound and gradient against the oracle."""
    for which in ["tiny", "tiny_odd", "tiny_s3", "tiny_tma"]:
        pb = _tiny_conv(which)
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 24, 0, 4, 1, props=np.arange(24) % 2)
        a, b = wl.random_alpha_beta(batch, 3, 1.0)
        net, dom, db = _gpu(pb, props, batch)
        assert bc.path_supported(net, LAYER_PATHS[path])
        bc.set_launch(net, LAYER_PATHS[path])
        assert bc.get_launch(net, batch.B * pb.K)[0] == LAYER_PATHS[path]
        lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
        assert bc.status(net) == 0
        ref = O.bound(onet, props, batch, a, b)
        err = np.abs(lb - ref) / _scale(ref)
        print("bf16 %s %s: max err / median|lb| = %.3e" % (path, which, err.max()))
        assert err.max() <= BF16_TOL[which], which
        _, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.BF16)
        assert bc.status(net) == 0
        _, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
        _check_grad(pb, onet, props, batch, da.cpu().numpy(), dbeta.cpu().numpy(), da_ref, db_ref,
                    "%s %s" % (path, which))


def test_autotune_times_every_candidate_and_its_choice_is_taken():
    """The tuner's candidates are the supported paths (the GEMM paths at 1 and 2 CTAs per SM); the
    choice is the fastest, later calls with rows in the same power-of-two bucket take it, and a
    bound under it equals the bound with that configuration set by hand, bit for bit."""
    pb = wl.problem_conv_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 48, 1, 8, 2)
    a, b = wl.random_alpha_beta(batch, 5, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    best, cands = bc.autotune(net, dom, db, _t(a), _t(b), reps=2)
    assert bc.status(net) == 0
    paths = {c[0][0] for c in cands}
    assert paths == {bc.N.PATH_LAYER_EPI, bc.N.PATH_LAYER_GATHER, bc.N.PATH_LAYER_IM2COL}
    assert len(cands) == 5 and all(ms > 0 for _, ms in cands)
    assert best == min(cands, key=lambda c: c[1])[0]
    print("autotune conv_small (48 subdomains): " + ", ".join("%s/%d %.3f ms" % (bc.N.PATH_NAMES[c[0]], c[1], ms)
                                                             for c, ms in cands))
    R = batch.B * pb.K
    assert bc.get_launch(net, R) == best
    assert bc.get_launch(net, R + 1)[0] in paths            # another bucket: the built-in order
    lb_tuned = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    net2, dom2, db2 = _gpu(pb, props, batch)
    bc.set_launch(net2, *best)
    lb_set = bc.bound(net2, dom2, db2, _t(a), _t(b), bc.BF16).cpu().numpy()
    assert np.array_equal(lb_tuned, lb_set)
    ref = O.bound(onet, props, batch, a, b)
    assert (np.abs(lb_tuned - ref) / _scale(ref)).max() <= BF16_TOL["conv_small"]


@pytest.mark.parametrize("path", ["layer_gather", "layer_epi"])
def test_bf16_conv_at_the_size_limits_matches_oracle(path):
    """A conv layer at the limits of the tensor-core path: 256 output channels (N = 256, the
    whole 512-column TMEM for two accumulators) and K = 128 x 4 x 4 = 2048 (the largest gather
    table); the stride-2 backward pass split into 4 phases of K = 256 x 2 x 2.  On the
    fused-epilogue path the stride-2 forward pass reads its operand by strided TMA boxes."""
    layers = wl.conv_layers((128, 8, 8), [(256, 4, 2, 1)], [16, 4], 5)
    pb = wl.make_problem("conv_limits", layers, 1, 0.02, 3, 5)
    onet = O.OracleNet(pb.layers, pb.C)
    l, u = O.interval_bounds(onet, pb.x_lo, pb.x_hi)
    l, u = l.astype(np.float32), u.astype(np.float32)
    unst = [np.nonzero(O.unstable_mask(l[0], u[0]))[0]]
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
    batch = wl.random_batch(pb, unst, 6, 0, 4, 2)
    a, b = wl.random_alpha_beta(batch, 4, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    bc.set_launch(net, LAYER_PATHS[path])
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy()
    assert bc.status(net) == 0
    ref = O.bound(onet, props, batch, a, b)
    err = np.abs(lb - ref) / _scale(ref)
    print("bf16 conv at the limits (%s): max err / median|lb| = %.3e" % (path, err.max()))
    assert err.max() <= BF16_TOL["conv_limits"]
    _, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.BF16)
    _, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    _check_grad(pb, onet, props, batch, da.cpu().numpy(), dbeta.cpu().numpy(), da_ref, db_ref, "conv limits")


def test_bf16_conv_beyond_the_channel_limit_is_refused():
    """272 output channels exceed the tensor-core path: BF16 is refused (BCROWN_ERR_UNIMPLEMENTED)
    while FP32 bounds the same net."""
    layers = wl.conv_layers((2, 4, 4), [(272, 3, 1, 1)], [4], 6)
    pb = wl.make_problem("conv_wide", layers, 1, 0.05, 3, 6)
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 4, 0, 2, 3)
    a, b = wl.random_alpha_beta(batch, 5, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    with pytest.raises(bc.BcrownError) as ei:
        bc.bound(net, dom, db, _t(a), _t(b), bc.BF16)
    assert ei.value.code == -6
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.FP32).cpu().numpy()
    assert np.max(rel_err(lb, O.bound(onet, props, batch, a, b))) <= RTOL


@pytest.mark.parametrize("path", ["layer_gather", "layer_epi"])
@pytest.mark.parametrize("which", ["conv_small", "conv_big"])
def test_bf16_conv_full_size_sampled(which, path):
    """The conv workloads at their full sizes in BF16 (the bench's configuration: 2048 and 4096
    BaB-tree subdomains x 9 specs in one bound pass), on the gather GEMMs the autotuner picks for
    the bench and on the fused-epilogue GEMMs; sampled subdomains recomputed by the oracle one by
    one."""
    if which == "conv_small":
        pb = wl.problem_conv_small()
        onet, props, unst = oracle_setup(pb)
        n, depth, n_check = 2048, 16, 12
    else:
        pb = wl.problem_conv_big()
        onet = O.OracleNet(pb.layers, pb.C)
        l, u = O.interval_bounds(onet, pb.x_lo, pb.x_hi)
        l, u = l.astype(np.float32), u.astype(np.float32)
        unst = [np.nonzero(O.unstable_mask(l[0], u[0]))[0]]
        props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
        n, depth, n_check = 4096, 24, 3
    batch = wl.tree_batch(pb, unst, [n], depth, 1)
    a, b = wl.random_alpha_beta(batch, 6, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    bc.set_launch(net, LAYER_PATHS[path])
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.BF16).cpu().numpy().reshape(batch.B, pb.K)
    assert bc.status(net) == 0 and batch.B == n
    idx = np.sort(np.random.default_rng(0).choice(batch.B, size=n_check, replace=False))
    sb, sa, sbeta = repack(pb, batch, [len(x) for x in unst], idx, a, b)
    ref = O.bound(onet, props, sb, sa, sbeta).reshape(len(idx), pb.K)
    err = np.abs(lb[idx] - ref) / _scale(ref)
    print("%s %s full size, %d sampled subdomains: max err / median|lb| = %.3e" % (which, path, n_check, err.max()))
    assert err.max() <= BF16_TOL[which]

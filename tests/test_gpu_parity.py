"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300)."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import RTOL, oracle_setup, rel_err, repack

pytestmark = pytest.mark.gpu


def _gpu(pb, props, batch):
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    db = bc.DeviceBatch.from_host(batch)
    return net, dom, db


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x, np.float32)).cuda()


def _U(props, net_o):
    _, U = O.unstable_ranks(net_o, props["l"], props["u"])
    return U


# ------------------------------------------------------------------ bound at fixed alpha, beta

def test_mlp_small_bound_parity_and_certify():
    pb = wl.problem_mlp_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 64, 0, 4, 1)
    a, b = wl.random_alpha_beta(batch, 2, 1.0)
    ref = O.bound(onet, props, batch, a, b)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.FP32).cpu().numpy()
    assert np.max(rel_err(lb, ref)) <= RTOL
    lbc = bc.bound(net, dom, db, _t(a), _t(b), bc.CERTIFY).cpu().numpy()
    assert np.all(lbc <= ref + 1e-12 * np.abs(ref))
    assert np.max(rel_err(lbc, ref)) <= 1e-4
    assert bc.status(net) == 0


def test_mlp_784_bound_parity_sampled():
    pb = wl.problem_mlp_784()
    onet, props, unst = oracle_setup(pb)
    batch = wl.tree_batch(pb, unst, [1024], 12, 3)
    a, b = wl.random_alpha_beta(batch, 4, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.FP32).cpu().numpy().reshape(batch.B, pb.K)
    U = _U(props, onet)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(batch.B - 1, 95, replace=False), [batch.B - 1]])
    sb, sa, sbeta = repack(pb, batch, U, idx, a, b)
    ref = O.bound(onet, props, sb, sa, sbeta).reshape(len(idx), pb.K)
    assert np.max(rel_err(lb[idx], ref)) <= RTOL
    lbc = bc.bound(net, dom, db, _t(a), _t(b), bc.CERTIFY).cpu().numpy().reshape(batch.B, pb.K)
    assert np.all(lbc[idx] <= ref + 1e-12 * np.abs(ref))
    assert bc.status(net) == 0


def _tiny_conv():
    layers = wl.conv_layers((2, 6, 6), [(3, 3, 2, 1), (4, 3, 1, 1)], [8, 4], 3)
    return wl.make_problem("tinyconv", layers, 2, 0.1, 3, 3)


def test_conv_bound_and_grad_parity():
    pb = _tiny_conv()
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 33, 0, 4, 5)
    a, b = wl.random_alpha_beta(batch, 6, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    ref, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    lb, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.FP32)
    assert np.max(rel_err(lb.cpu().numpy(), ref)) <= RTOL
    scale = max(np.abs(da_ref).max(initial=0), 1e-6)
    assert np.max(np.abs(da.cpu().numpy() - da_ref), initial=0) <= 1e-4 * scale
    scale = max(np.abs(db_ref).max(initial=0), 1e-6)
    assert np.max(np.abs(dbeta.cpu().numpy() - db_ref), initial=0) <= 1e-4 * scale


def test_conv_c3_bound_parity_sampled():
    pb = wl.problem_conv_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.tree_batch(pb, unst, [48], 16, 7)
    a, b = wl.random_alpha_beta(batch, 8, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.FP32).cpu().numpy()
    ref = O.bound(onet, props, batch, a, b)
    assert np.max(rel_err(lb, ref)) <= RTOL


# ------------------------------------------------------------------ gradient

@pytest.mark.parametrize("which", ["small", "784"])
def test_gradient_parity(which):
    if which == "small":
        pb = wl.problem_mlp_small()
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 64, 0, 4, 1)
    else:
        pb = wl.problem_mlp_784()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [48], 12, 9)
    a, b = wl.random_alpha_beta(batch, 2, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb, da, dbeta = bc.bound_grad(net, dom, db, _t(a), _t(b), bc.FP32)
    ref, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    assert np.max(rel_err(lb.cpu().numpy(), ref)) <= RTOL
    for g, gr in ((da.cpu().numpy(), da_ref), (dbeta.cpu().numpy(), db_ref)):
        tol = 1e-3 * (np.abs(gr) + 1e-3 * max(np.abs(gr).max(initial=0), 1e-6))
        assert np.all(np.abs(g - gr) <= tol)
    # finite differences of the FP64 oracle on a few coordinates (kink-free ones)
    rng = np.random.default_rng(1)
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    h = 1e-6
    for idx in rng.choice(len(a64), 6, replace=False):
        p, m = a64.copy(), a64.copy()
        p[idx] += h
        m[idx] -= h
        fd = (O.bound(onet, props, batch, p, b64).sum() - O.bound(onet, props, batch, m, b64).sum()) / (2 * h)
        assert abs(fd - da.cpu().numpy()[idx]) <= 1e-3 * (1 + abs(fd))


def test_autograd_function_matches_adjoint():
    pb = wl.problem_mlp_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 16, 0, 3, 2)
    a, b = wl.random_alpha_beta(batch, 3, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    U = _U(props, onet)
    ra, rb = bc.param_rows(db, pb.K, U)
    at = _t(a).requires_grad_(True)
    bt = _t(b).requires_grad_(True)
    w = torch.arange(batch.B * pb.K, device="cuda", dtype=torch.float32) / 7.0
    lb = bc.BoundFunction.apply(at, bt, net, dom, db, ra, rb, bc.FP32)
    (lb * w).sum().backward()
    _, da_ref, db_ref = O.grad(onet, props, batch, a.astype(np.float64), b.astype(np.float64))
    wr = w.cpu().numpy().astype(np.float64)
    assert np.allclose(at.grad.cpu().numpy(), da_ref * wr[ra.cpu().numpy()], rtol=1e-3, atol=1e-5)
    assert np.allclose(bt.grad.cpu().numpy(), db_ref * wr[rb.cpu().numpy()], rtol=1e-3, atol=1e-5)


# ------------------------------------------------------------------ root bounds

@pytest.mark.parametrize("maker", [wl.problem_mlp_small, wl.problem_mlp_784, _tiny_conv])
def test_root_bounds_parity(maker):
    pb = maker()
    onet = O.OracleNet(pb.layers, pb.C)
    l_ref, u_ref = O.root_bounds(onet, pb.x_lo, pb.x_hi)
    net = bc.load_net(pb.layers, pb.C)
    l, u, cnt = bc.root_bounds(net, _t(pb.x_lo), _t(pb.x_hi), bc.ALPHA_ADAPTIVE, 0.5, bc.FP32)
    l, u = l.cpu().numpy(), u.cpu().numpy()
    # FP32 back-substitution against FP64, every layer at the 1e-5 bar (measured on a GB300: at
    # most 1.2e-6 relative to max(|bound|, 1), on the deepest layer of the 784-256x6 net)
    scale = np.maximum(np.abs(l_ref), 1.0)
    assert np.max(np.abs(l - l_ref) / scale) <= RTOL
    assert np.max(np.abs(u - u_ref) / np.maximum(np.abs(u_ref), 1.0)) <= RTOL
    assert np.array_equal(cnt.cpu().numpy(), ((l < 0) & (u > 0)).sum(axis=1))
    lc, uc, _ = bc.root_bounds(net, _t(pb.x_lo), _t(pb.x_hi), bc.ALPHA_ADAPTIVE, 0.5, bc.CERTIFY)
    lc, uc = lc.cpu().numpy(), uc.cpu().numpy()
    # sound against sampled pre-activations of the exact network
    rng = np.random.default_rng(0)
    xs = rng.uniform(pb.x_lo[0].astype(np.float64), pb.x_hi[0].astype(np.float64), size=(4000, pb.x_lo.shape[1]))
    z = np.concatenate([zi for zi in onet.preacts(xs)[1:]], axis=1)
    assert np.all(z >= lc[0] - 1e-9) and np.all(z <= uc[0] + 1e-9)
    assert np.all(lc <= uc)
    # stated gap of the outward-rounded bounds to the FP64 oracle (a priori GEMM error terms
    # grow with |W| M; about 1 % on the deepest layer of the 784-256x6 net)
    assert np.max(np.abs(lc - l_ref) / scale) <= 2e-2


# ------------------------------------------------------------------ bookkeeping (bit-exact)

def test_neuron_codes_bit_exact():
    pb = wl.problem_mlp_784()
    onet, props, unst = oracle_setup(pb)
    batch = wl.tree_batch(pb, unst, [300], 12, 11)
    net, dom, db = _gpu(pb, props, batch)
    codes = bc.neuron_codes(net, dom, db).cpu().numpy()
    rows = O.expand_rows(onet, batch, props["l"], props["u"])
    ref = np.concatenate(O.neuron_codes(onet, rows, props["l"], props["u"])[1:], axis=1)
    assert np.array_equal(codes, ref)


def test_batch_split_bit_exact():
    pb = wl.problem_mlp_784()
    onet, props, unst = oracle_setup(pb)
    batch = wl.tree_batch(pb, unst, [100], 8, 13)
    U = _U(props, onet)
    a, b = wl.random_alpha_beta(batch, 1, 1.0)
    rng = np.random.default_rng(3)
    gsel = np.array([rng.choice(unst[0]) for _ in range(batch.B)])
    layer, idx = wl.neuron_layer_index(pb.hidden_widths, gsel)
    net, dom, db = _gpu(pb, props, batch)
    child, ca, cb = bc.batch_split(net, dom, db, torch.as_tensor(layer.astype(np.uint8)).cuda(),
                                   torch.as_tensor(idx.astype(np.int32)).cuda(), _t(a), _t(b), U)
    ref = O.batch_split(batch, pb.K, U, layer, idx, a, b)
    got = [child.prop_of, child.split_off, child.split_cnt, child.split_layer, child.split_idx, child.split_sign,
           child.alpha_off, ca, cb]
    for g, r in zip(got, ref):
        assert np.array_equal(g.cpu().numpy().astype(np.float64), np.asarray(r).astype(np.float64))
    assert bc.status(net) == 0


# ------------------------------------------------------------------ optimiser

@pytest.mark.parametrize("which", ["small", "784"])
def test_optimize_parity(which):
    if which == "small":
        pb = wl.problem_mlp_small()
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 64, 0, 4, 1)
    else:
        pb = wl.problem_mlp_784()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [64], 12, 5)
    a0, b0 = wl.initial_alpha_beta(batch)
    net, dom, db = _gpu(pb, props, batch)
    at, bt = _t(a0), _t(b0)
    lb = bc.optimize(net, dom, db, at, bt, bc.OptCfg(precision=bc.FP32, certify=True)).cpu().numpy()
    a_best, b_best = at.cpu().numpy(), bt.cpu().numpy()
    ref_at_best = O.bound(onet, props, batch, a_best, b_best)
    assert np.all(lb <= ref_at_best + 1e-12 * np.abs(ref_at_best))
    # stated certification gap: the a priori FP32 contraction terms gamma_n |Lambda| |W| M
    # (Higham, Accuracy and Stability of Numerical Algorithms, 3.1) are worst-case sums of
    # magnitudes, several times |lb| on these nets; measured on a GB300: 1.02e-4 (784-256x6,
    # 64 subdomains) and 7.7e-5 (16-32-32-4) of max(|lb|, 1)
    gap = np.max(rel_err(lb, ref_at_best))
    print("certified gap at the optimised alpha, beta (%s): %.3e" % (which, gap))
    assert gap <= 2e-4
    init = O.bound(onet, props, batch, a0, b0)
    assert np.all(ref_at_best >= init - 1e-5 * np.maximum(np.abs(init), 1))
    ref_opt, _, _, _ = O.optimize(onet, props, batch, a0, b0)
    assert np.median(np.abs(ref_at_best - ref_opt) / np.maximum(np.abs(ref_opt), 1)) <= 1e-3
    assert bc.status(net) == 0


# ------------------------------------------------------------------ edge cases and invariances

def test_edge_cases():
    pb = wl.problem_mlp_small()
    onet, props, unst = oracle_setup(pb)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    # empty batch
    empty = wl.pack_batch(pb.hidden_widths, pb.K, [len(unst[0])], [])
    deb = bc.DeviceBatch.from_host(empty)
    out = bc.bound(net, dom, deb, _t(np.zeros(1)), _t(np.zeros(1)))
    assert out.numel() == 0
    # one subdomain with no split, ragged row count
    one = wl.random_batch(pb, unst, 1, 0, 0, 0)
    a, b = wl.initial_alpha_beta(one)
    lb = bc.bound(net, dom, bc.DeviceBatch.from_host(one), _t(a), _t(b)).cpu().numpy()
    assert np.max(rel_err(lb, O.bound(onet, props, one, a, b))) <= RTOL
    # out-of-range split index: skipped, reported through the status word, no fault
    bad = wl.random_batch(pb, unst, 4, 1, 2, 3)
    bad.split_idx = bad.split_idx.copy()
    bad.split_idx[0] = 100000
    a, b = wl.initial_alpha_beta(bad)
    assert bc.status(net) == 0
    bc.bound(net, dom, bc.DeviceBatch.from_host(bad), _t(a), _t(b))
    assert bc.status(net) == -1      # BCROWN_ERR_ARG, then cleared
    assert bc.status(net) == 0


def test_power_of_two_scaling_is_bit_exact():
    pb = wl.problem_mlp_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 32, 0, 4, 4)
    a, b = wl.random_alpha_beta(batch, 4, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    lb = bc.bound(net, dom, db, _t(a), _t(b)).cpu().numpy()
    net4 = bc.load_net(pb.layers, pb.C * 4.0)
    lb4 = bc.bound(net4, dom, db, _t(a), _t(b * 4.0)).cpu().numpy()
    assert np.array_equal(lb4, lb * 4.0)


def test_conv_c5_bound_parity_and_certify_sampled():
    """The precision workload's net (3x32x32 -> four 3x3 conv layers -> fc 8192-512-10,
    123,392 hidden neurons).  Intermediate bounds by the oracle's interval propagation (CROWN
    root bounds over 65,536-wide layers are out of reach for the oracle; any valid l <= z <= u
    serves the bound).  FP32 within 1e-5 of the FP64 oracle; the certified pass never above it,
    with its gap printed."""
    pb = wl.problem_conv_big()
    onet = O.OracleNet(pb.layers, pb.C)
    l, u = O.interval_bounds(onet, pb.x_lo, pb.x_hi)
    l, u = l.astype(np.float32), u.astype(np.float32)
    unst = [np.nonzero(O.unstable_mask(l[0], u[0]))[0]]
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
    batch = wl.tree_batch(pb, unst, [6], 24, 3)
    a, b = wl.random_alpha_beta(batch, 4, 1.0)
    net, dom, db = _gpu(pb, props, batch)
    ref = O.bound(onet, props, batch, a, b)
    lb = bc.bound(net, dom, db, _t(a), _t(b), bc.FP32).cpu().numpy()
    assert bc.status(net) == 0
    assert np.max(rel_err(lb, ref)) <= RTOL
    lbc = bc.bound(net, dom, db, _t(a), _t(b), bc.CERTIFY).cpu().numpy()
    assert bc.status(net) == 0
    assert np.all(lbc <= ref)
    gap = np.max((ref - lbc) / np.maximum(np.abs(ref), 1.0))
    print("conv c5 certified gap (relative): %.3e" % gap)
    assert gap <= 2e-2

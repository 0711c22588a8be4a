"""Joint optimisation of intermediate-layer bounds (Section 3.3) on the GPU against the FP64 oracle
(needs a GB300): the layout, the recomputed bounds and the final bound at fixed variables, the
gradient entry by entry, the optimiser, and the ablation switches (Table A4)."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from oracle import joint as J
from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import RTOL, oracle_setup, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "tiny": dict(widths=[5, 8, 8, 8, 3], seed=3, eps=0.2, n_sub=12, depth=4),
    "mlp_small": dict(widths=[16, 32, 32, 4], seed=0, eps=0.05, n_sub=16, depth=4),
    "mlp_deep": dict(widths=[12, 24, 24, 24, 24, 6], seed=2, eps=0.08, n_sub=8, depth=6),
}


def _setup(which):
    c = CASES[which]
    pb = wl.make_problem(which, wl.mlp_layers(c["widths"], c["seed"]), 2, c["eps"], 3, c["seed"])
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, c["n_sub"], 0, c["depth"], 7, props=np.arange(c["n_sub"]) % 2)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    return pb, onet, props, batch, net, dom, bc.DeviceBatch.from_host(batch)


def _vars(onet, props, batch, seed, beta_max=0.5):
    rng = np.random.default_rng(seed)
    lay = J.joint_layout(onet, batch, props["l"], props["u"])
    f = lambda n, hi: rng.uniform(0, hi, n).astype(np.float32)
    return f(batch.n_alpha, 1.0), f(batch.n_beta, beta_max), f(lay.n_alpha_p, 1.0), f(lay.n_beta_p, beta_max)


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x, np.float32)).cuda()


@pytest.mark.parametrize("which", list(CASES))
def test_layout_and_initial_alpha_prime_match_the_oracle(which):
    pb, onet, props, batch, net, dom, db = _setup(which)
    lay = J.joint_layout(onet, batch, props["l"], props["u"])
    assert bc.joint_sizes(net, dom, db) == (lay.n_alpha_p, lay.n_beta_p)
    ap, bp = bc.joint_init_alpha(net, dom, db)
    assert bc.status(net) == 0
    assert np.array_equal(ap.cpu().numpy(), J.init_alpha_p(onet, batch, props["l"], props["u"]).astype(np.float32))
    assert bp.numel() == lay.n_beta_p and float(bp.abs().sum()) == 0.0


@pytest.mark.parametrize("which", list(CASES))
def test_bound_and_recomputed_bounds_match_the_oracle(which):
    """At fixed alpha, beta, alpha', beta' (with splits): every row's bound and every subdomain's
    recomputed l, u within the FP32 bar of the oracle."""
    pb, onet, props, batch, net, dom, db = _setup(which)
    a, b, ap, bp = _vars(onet, props, batch, 1)
    lb, l, u = bc.bound_joint(net, dom, db, _t(a), _t(b), _t(ap), _t(bp))
    assert bc.status(net) == 0
    rl, rlo, rhi = J.joint_bound(onet, props, batch, a, b, ap, bp)
    e = [rel_err(lb.cpu().numpy(), rl).max(), rel_err(l.cpu().numpy(), rlo).max(), rel_err(u.cpu().numpy(), rhi).max()]
    print("joint %s: max rel err lb %.2e, l %.2e, u %.2e" % (which, *e))
    assert max(e) <= RTOL
    # the recomputed bounds are tighter than the root's somewhere (the splits reach them)
    assert (rlo > props["l"][batch.prop_of] + 1e-6).any()


def test_no_split_at_the_root_rule_gives_the_plain_bound():
    pb, onet, props, batch, net, dom, db = _setup("mlp_deep")
    nb = wl.pack_batch(pb.hidden_widths, pb.K, [int(x) for x in O.unstable_ranks(onet, props["l"], props["u"])[1]],
                       [(p, np.zeros(0, np.int64), np.zeros(0, np.int8)) for p in (0, 1, 1, 0)])
    ndb = bc.DeviceBatch.from_host(nb)
    a, b = wl.random_alpha_beta(nb, 4, 1.0)
    ap, bp = bc.joint_init_alpha(net, dom, ndb)
    lb, l, u = bc.bound_joint(net, dom, ndb, _t(a), _t(b), ap, bp)
    plain = bc.bound(net, dom, ndb, _t(a), _t(b), bc.FP32)
    assert bc.status(net) == 0
    assert rel_err(lb.cpu().numpy(), plain.cpu().numpy()).max() <= RTOL
    assert rel_err(l.cpu().numpy(), props["l"][nb.prop_of]).max() <= RTOL
    assert rel_err(u.cpu().numpy(), props["u"][nb.prop_of]).max() <= RTOL


@pytest.mark.parametrize("which", list(CASES))
def test_gradient_matches_the_oracle_entry_by_entry(which):
    """d(sum of bounds)/d(alpha, beta, alpha', beta') against the oracle's automatic
    differentiation: every entry within 1e-3 of |g| + 1e-3 max|g| of its group (FP32 through up
    to L - 1 nested passes), the same entries zero, and a nonzero alpha' and beta' gradient."""
    pb, onet, props, batch, net, dom, db = _setup(which)
    a, b, ap, bp = _vars(onet, props, batch, 2)
    lb, *g = bc.bound_joint_grad(net, dom, db, _t(a), _t(b), _t(ap), _t(bp))
    assert bc.status(net) == 0
    ref = J.joint_grad(onet, props, batch, a, b, ap, bp)
    assert rel_err(lb.cpu().numpy(), ref[0]).max() <= RTOL
    for name, gg, gr in zip(("alpha", "beta", "alpha'", "beta'"), g, ref[1:]):
        gg = gg.cpu().numpy().astype(np.float64)
        if gr.size == 0:
            continue
        tol = 1e-3 * (np.abs(gr) + 1e-3 * np.abs(gr).max())
        bad = np.abs(gg - gr) > tol
        print("joint %s d%s: %d entries, max |err| %.2e, outside tol %d" % (which, name, gr.size,
                                                                          np.abs(gg - gr).max(), bad.sum()))
        assert bad.sum() <= max(1, gr.size // 1000), (name, np.nonzero(bad)[0][:10])
    if which != "mlp_small":
        assert np.abs(g[2].cpu().numpy()).max() > 0 and np.abs(g[3].cpu().numpy()).max() > 0


def test_optimizer_follows_the_oracle_and_the_switches_hold_their_groups():
    pb, onet, props, batch, net, dom, db = _setup("tiny")
    a0, b0 = wl.initial_alpha_beta(batch)
    ap0 = J.init_alpha_p(onet, batch, props["l"], props["u"]).astype(np.float32)
    bp0 = np.zeros(J.joint_layout(onet, batch, props["l"], props["u"]).n_beta_p, np.float32)
    for fa, fb in ((False, False), (True, False), (False, True)):
        th = [_t(x) for x in (a0, b0, ap0, bp0)]
        cfg = bc.OptCfg(iters=10, certify=False, freeze_alpha=fa, freeze_beta=fb)
        lb, l, u = bc.optimize_joint(net, dom, db, *th, cfg=cfg)
        assert bc.status(net) == 0
        ocfg = J.JointCfg(iters=10, lr_alpha=cfg.lr_alpha, lr_beta=cfg.lr_beta, decay=cfg.decay,
                          freeze_alpha=fa, freeze_beta=fb)
        rlb, *_ = J.joint_optimize(onet, props, batch, a0, b0, ap0, bp0, ocfg)
        gap = np.abs(lb.cpu().numpy() - rlb) / np.maximum(np.abs(rlb), 1.0)
        print("joint optimise (freeze alpha %s, beta %s): median / max rel gap to the oracle %.2e / %.2e"
              % (fa, fb, np.median(gap), gap.max()))
        assert np.median(gap) <= 1e-3
        if fa:
            assert np.array_equal(th[0].cpu().numpy(), a0) and np.array_equal(th[2].cpu().numpy(), ap0)
        if fb:
            assert np.array_equal(th[1].cpu().numpy(), b0) and np.array_equal(th[3].cpu().numpy(), bp0)
        # the kept iterate's bound is at least the starting one, per subdomain
        start = J.joint_bound(onet, props, batch, a0, b0, ap0, bp0)[0].reshape(batch.B, pb.K).sum(axis=1)
        assert np.all(lb.cpu().numpy().reshape(batch.B, pb.K).sum(axis=1) >= start - 1e-4 * np.abs(start))


def test_freeze_switches_of_the_plain_optimizer():
    """bcrown_optimize with alpha or beta frozen (the beta-only and alpha-only ablations): the frozen
    group comes back bit for bit, the other moves."""
    pb, onet, props, batch, net, dom, db = _setup("mlp_small")
    a0, b0 = wl.random_alpha_beta(batch, 3, 0.5)
    for fa, fb in ((True, False), (False, True)):
        for prec in (bc.FP32, bc.BF16):
            a, b = _t(a0), _t(b0)
            bc.optimize(net, dom, db, a, b, bc.OptCfg(precision=prec, certify=True, freeze_alpha=fa, freeze_beta=fb))
            assert bc.status(net) == 0
            if fa:
                assert np.array_equal(a.cpu().numpy(), a0) and not np.array_equal(b.cpu().numpy(), b0)
            if fb:
                assert np.array_equal(b.cpu().numpy(), b0) and not np.array_equal(a.cpu().numpy(), a0)

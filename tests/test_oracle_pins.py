"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import bcrown_oracle as O
from oracle import lp_pins as LP
from paper_2103_06624_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _setup(pb):
    net = O.OracleNet(pb.layers, pb.C)
    l, u = O.root_bounds(net, pb.x_lo, pb.x_hi)
    unst = [np.nonzero(O.unstable_mask(l[p], u[p]))[0] for p in range(pb.P)]
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
    return net, props, unst


def tiny_problem(seed=5, widths=(3, 6, 6, 3), eps=0.3, K=2):
    layers = wl.mlp_layers(list(widths), seed)
    return wl.make_problem("tiny", layers, 1, eps, K, seed)


def tiny_conv_problem(seed=3):
    layers = wl.conv_layers((2, 6, 6), [(3, 3, 2, 1), (4, 3, 1, 1)], [8, 4], seed)
    return wl.make_problem("tinyconv", layers, 2, 0.1, 3, seed)


# ------------------------------------------------------------------ golden worked example

def test_golden_intro_example():
    g = json.load(open(os.path.join(GOLD, "intro_2d_example.json")))
    nw = g["network"]
    layers = [wl.Layer("fc", np.array(nw["W1"], np.float32), np.array(nw["b1"], np.float32), (2,), (2,)),
              wl.Layer("fc", np.array(nw["W2"], np.float32), np.array(nw["b2"], np.float32), (2,), (1,))]
    C = np.ones((1, 1), np.float32)
    net = O.OracleNet(layers, C)
    x_lo = np.array([g["box"]["x_lo"]])
    x_hi = np.array([g["box"]["x_hi"]])
    l, u = O.root_bounds(net, x_lo, x_hi)
    assert np.allclose(l[0], g["root_bounds_printed_in_paper"]["l"])
    assert np.allclose(u[0], g["root_bounds_printed_in_paper"]["u"])
    props = dict(x_lo=x_lo, x_hi=x_hi, l=l, u=u)
    for case in g["cases"]:
        s = case["split"]
        subs = [(0, np.array([1] if s else [], np.int64), np.array([s] if s else [], np.int8))]
        batch = wl.pack_batch([2], 1, [2], subs)
        alpha = np.array([case["alpha1"], 0.5])          # neuron 2's alpha is unused
        beta = np.array([case["beta2"]] if s else [])
        lb = O.bound(net, props, batch, alpha, beta)
        assert lb[0] == pytest.approx(case["lb"], abs=1e-12), case
        ex = LP.exact_min(net, x_lo[0], x_hi[0], l[0], u[0], [(1, 1, s)] if s else [], 0)
        assert ex == pytest.approx(g["exact_min"][str(s)], abs=1e-9)
        assert lb[0] <= ex + 1e-12


# ------------------------------------------------------------------ three formulas agree

@pytest.mark.parametrize("maker", [tiny_problem, tiny_conv_problem, wl.problem_mlp_small])
def test_recursion_explicit_dual_agree(maker):
    pb = maker()
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 6, 0, 4, 11)
    a, b = wl.random_alpha_beta(batch, 2, 3.0)
    lb = O.bound(net, props, batch, a, b)
    lbe = O.bound_explicit(net, props, batch, a, b)
    lbd = O.bound_dual(net, props, batch, a, b)
    scale = 1.0 + np.abs(lb)
    assert np.max(np.abs(lb - lbe) / scale) < 1e-12
    assert np.max(np.abs(lb - lbd) / scale) < 1e-12


def test_beta_zero_no_split_is_crown():
    """beta = 0 with splits present equals CROWN on the split-free net with the same D (Section 3.1):
    with no split at all, the dual form reduces to Wong & Kolter's / CROWN's."""
    pb = wl.problem_mlp_small()
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 4, 0, 0, 1)
    a, b = wl.random_alpha_beta(batch, 3)
    assert batch.n_beta == 0
    lb = O.bound(net, props, batch, a, b)
    lbd = O.bound_dual(net, props, batch, a, b)
    assert np.allclose(lb, lbd, rtol=0, atol=1e-12)


def test_eps_zero_closed_form():
    """At eps = 0 every neuron is stable and the bound is c_k^T f(x0) exactly."""
    pb = wl.problem_mlp_small(seed=4)
    pb.x_lo = pb.x0.copy()
    pb.x_hi = pb.x0.copy()
    net, props, unst = _setup(pb)
    assert all(len(u) == 0 for u in unst)
    batch = wl.random_batch(pb, unst, 2, 0, 0, 0)
    lb = O.bound(net, props, batch, np.zeros(0), np.zeros(0))
    f = net.forward(pb.x0[0].astype(np.float64))[0]
    assert np.allclose(lb.reshape(2, -1), f[None, :], rtol=0, atol=1e-12)


def test_linear_net_vertex_bruteforce():
    """With no unstable neuron the bound is the exact minimum over the box's vertices."""
    layers = wl.mlp_layers([5, 7, 7, 3], 9)
    for ly in layers[:-1]:
        ly.b = ly.b + np.float32(8.0)       # every neuron active on the box
    pb = wl.make_problem("lin", layers, 1, 0.2, 2, 9)
    net, props, unst = _setup(pb)
    assert all(len(u) == 0 for u in unst)
    batch = wl.random_batch(pb, unst, 1, 0, 0, 0)
    lb = O.bound(net, props, batch, np.zeros(0), np.zeros(0))
    verts = np.array(list(itertools.product([0, 1], repeat=5)), np.float64)
    xs = pb.x_lo[0].astype(np.float64) + verts * (pb.x_hi[0].astype(np.float64) - pb.x_lo[0])
    f = net.forward(xs)
    assert np.allclose(lb, f.min(axis=0), rtol=0, atol=1e-12)


# ------------------------------------------------------------------ soundness, LP, completeness

def test_soundness_against_samples():
    pb = wl.problem_mlp_small(seed=1)
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 12, 0, 4, 5)
    rng = np.random.default_rng(0)
    for trial in range(3):
        a, b = wl.random_alpha_beta(batch, 10 + trial, 10.0)
        lb = O.bound(net, props, batch, a, b)
        for bi in range(batch.B):
            o, c = batch.split_off[bi], batch.split_cnt[bi]
            splits = list(zip(batch.split_layer[o:o + c], batch.split_idx[o:o + c], batch.split_sign[o:o + c]))
            for k in range(pb.K):
                m, n = LP.sampled_min(net, pb.x_lo[0].astype(float), pb.x_hi[0].astype(float), splits, k,
                                      20000, rng)
                assert lb[bi * pb.K + k] <= m + 1e-9


def test_lp_corollary():
    """g(alpha, beta) <= p*_LP for any feasible alpha, beta; optimised g reaches p*_LP (Corollary 3.1)."""
    pb = tiny_problem()
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 6, 0, 3, 0)
    a, b = wl.random_alpha_beta(batch, 1, 2.0)
    lb = O.bound(net, props, batch, a, b)
    cfg = O.AdamCfg(iters=600, lr_alpha=0.05, lr_beta=0.05, decay=0.995)
    a0, b0 = wl.initial_alpha_beta(batch)
    lbo, _, _, _ = O.optimize(net, props, batch, a0, b0, cfg)
    for bi in range(batch.B):
        o, c = batch.split_off[bi], batch.split_cnt[bi]
        splits = list(zip(batch.split_layer[o:o + c], batch.split_idx[o:o + c], batch.split_sign[o:o + c]))
        for k in range(pb.K):
            r = bi * pb.K + k
            p = LP.lp_value(net, pb.x_lo[0].astype(float), pb.x_hi[0].astype(float),
                            props["l"][0], props["u"][0], splits, k)
            assert lb[r] <= p + 1e-8
            assert lbo[r] <= p + 1e-8
            assert p - lbo[r] <= 2e-3 * abs(p) + 1e-5


def test_completeness_full_split():
    """All unstable neurons split: optimised beta reaches the exact per-pattern minimum (Theorem 3.3)."""
    pb = tiny_problem(seed=5)
    net, props, unst = _setup(pb)
    U = len(unst[0])
    rng = np.random.default_rng(2)
    subs = []
    H = int(sum(pb.hidden_widths))
    for _ in range(4):
        # signs read off the activation pattern at a random box point, so the subdomain is feasible
        x = rng.uniform(pb.x_lo[0].astype(np.float64), pb.x_hi[0].astype(np.float64))
        z = np.concatenate([zi[0] for zi in net.preacts(x)[1:]])
        assert z.shape[0] == H
        signs = np.where(z[unst[0]] >= 0, -1, 1).astype(np.int8)
        subs.append((0, unst[0].astype(np.int64), signs))
    batch = wl.pack_batch(pb.hidden_widths, pb.K, [U], subs)
    a0, b0 = wl.initial_alpha_beta(batch)
    cfg = O.AdamCfg(iters=3000, lr_alpha=0.0, lr_beta=0.05, decay=0.999)
    lbo, _, _, _ = O.optimize(net, props, batch, a0, b0, cfg)
    n_checked = 0
    for bi in range(batch.B):
        o, c = batch.split_off[bi], batch.split_cnt[bi]
        splits = list(zip(batch.split_layer[o:o + c], batch.split_idx[o:o + c], batch.split_sign[o:o + c]))
        for k in range(pb.K):
            ex = LP.exact_min(net, pb.x_lo[0].astype(float), pb.x_hi[0].astype(float),
                              props["l"][0], props["u"][0], splits, k)
            r = bi * pb.K + k
            if np.isfinite(ex):
                assert lbo[r] <= ex + 1e-9
                assert ex - lbo[r] <= 1e-4 * (1 + abs(ex))
                n_checked += 1
    assert n_checked > 0


# ------------------------------------------------------------------ gradient

@pytest.mark.parametrize("maker", [wl.problem_mlp_small, tiny_conv_problem])
def test_gradient_finite_differences(maker):
    pb = maker()
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 4, 1, 4, 3)
    a, b = wl.random_alpha_beta(batch, 4, 2.0)
    a, b = a.astype(np.float64), b.astype(np.float64)
    _, da, db = O.grad(net, props, batch, a, b)
    h = 1e-6
    rng = np.random.default_rng(0)
    for vec, g in ((a, da), (b, db)):
        for idx in rng.choice(len(vec), min(12, len(vec)), replace=False):
            p, m = vec.copy(), vec.copy()
            p[idx] += h
            m[idx] -= h
            args_p = (p, b) if vec is a else (a, p)
            args_m = (m, b) if vec is a else (a, m)
            fp = O.bound(net, props, batch, *args_p).sum()
            fm = O.bound(net, props, batch, *args_m).sum()
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * (1 + abs(fd)), (idx, fd, g[idx])


# ------------------------------------------------------------------ root bounds

def test_root_bounds_layer1_exact_and_sound():
    pb = tiny_problem(widths=(4, 6, 5, 2), eps=0.4)
    net, props, _ = _setup(pb)
    l, u = props["l"][0], props["u"][0]
    verts = np.array(list(itertools.product([0, 1], repeat=4)), np.float64)
    xs = pb.x_lo[0].astype(np.float64) + verts * (pb.x_hi[0].astype(np.float64) - pb.x_lo[0])
    z1 = net.preacts(xs)[1]
    assert np.allclose(l[:6], z1.min(axis=0), atol=1e-12)
    assert np.allclose(u[:6], z1.max(axis=0), atol=1e-12)
    rng = np.random.default_rng(1)
    xs = rng.uniform(pb.x_lo[0], pb.x_hi[0], size=(50000, 4))
    zs = net.preacts(xs)
    for i in range(1, net.L):
        lo, hi = net.hoff[i - 1], net.hoff[i]
        assert np.all(zs[i] >= l[lo:hi] - 1e-12)
        assert np.all(zs[i] <= u[lo:hi] + 1e-12)


def test_interval_bounds_exact_layer1_sound_and_degenerate():
    """Interval bounds: layer 1 is the exact interval (= CROWN's), every layer contains the
    pre-activations of box samples, and a zero-width box collapses them onto z(x0)."""
    for pb in (tiny_problem(widths=(4, 6, 5, 2), eps=0.4), tiny_conv_problem()):
        net, props, _ = _setup(pb)
        l, u = O.interval_bounds(net, pb.x_lo, pb.x_hi)
        h1 = net.hoff[1]
        assert np.allclose(l[0, :h1], props["l"][0][:h1], atol=1e-6)
        assert np.allclose(u[0, :h1], props["u"][0][:h1], atol=1e-6)
        rng = np.random.default_rng(2)
        xs = rng.uniform(pb.x_lo[0], pb.x_hi[0], size=(20000, pb.x_lo.shape[1]))
        zs = net.preacts(xs)
        for i in range(1, net.L):
            lo, hi = net.hoff[i - 1], net.hoff[i]
            assert np.all(zs[i] >= l[0, lo:hi] - 1e-12)
            assert np.all(zs[i] <= u[0, lo:hi] + 1e-12)
        x0 = 0.5 * (pb.x_lo[0].astype(np.float64) + pb.x_hi[0])
        l0, u0 = O.interval_bounds(net, x0[None, :], x0[None, :])
        z0 = np.concatenate([z[0] for z in net.preacts(x0[None, :])[1:]])
        assert np.allclose(l0[0], z0, atol=1e-12) and np.allclose(u0[0], z0, atol=1e-12)


# ------------------------------------------------------------------ library-routine pins

def test_conv_matrix_matches_torch_conv2d():
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F
    pb = tiny_conv_problem()
    rng = np.random.default_rng(0)
    for ly in pb.layers:
        if ly.kind != "conv":
            continue
        M = O.conv_matrix(ly)
        x = rng.normal(size=ly.in_shape)
        ref = F.conv2d(torch.tensor(x)[None], torch.tensor(ly.W.astype(np.float64)), None,
                       stride=ly.stride, padding=ly.pad)[0].numpy().ravel()
        assert np.allclose(M @ x.ravel(), ref, atol=1e-12)


def test_adam_step_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    theta = rng.uniform(0, 1, 50)
    cfg = O.AdamCfg()
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=cfg.lr_alpha, betas=(cfg.beta1, cfg.beta2), eps=cfg.eps, maximize=True)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, cfg.decay)
    th, m, v = theta.copy(), np.zeros(50), np.zeros(50)
    for t in range(5):
        g = rng.normal(size=50)
        p.grad = torch.tensor(g)
        opt.step()
        sched.step()
        th, m, v = O.adam_ascent_step(th, m, v, g, t, cfg.lr_alpha * cfg.decay ** t, cfg, -np.inf, np.inf)
        assert np.allclose(th, p.detach().numpy(), atol=1e-12)


def test_batch_split_definition():
    pb = wl.problem_mlp_small()
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 3, 1, 2, 0)
    _, U = O.unstable_ranks(net, props["l"], props["u"])
    a, b = wl.random_alpha_beta(batch, 0)
    pick_layer = np.array([1, 2, 1])
    pick_idx = np.array([3, 5, 7])
    out = O.batch_split(batch, pb.K, U, pick_layer, pick_idx, a, b)
    prop, off, cnt, lay, idx, sgn, aoff, a2, b2 = out
    assert len(prop) == 6
    for c in range(6):
        par = c // 2
        po, pc = batch.split_off[par], batch.split_cnt[par]
        assert cnt[c] == pc + 1
        assert list(lay[off[c]:off[c] + pc]) == list(batch.split_layer[po:po + pc])
        assert lay[off[c] + pc] == pick_layer[par] and idx[off[c] + pc] == pick_idx[par]
        assert sgn[off[c] + pc] == (-1 if c % 2 == 0 else 1)
        n = U[0] * pb.K
        assert np.array_equal(a2[aoff[c]:aoff[c] + n], a[batch.alpha_off[par]:batch.alpha_off[par] + n])
        for k in range(pb.K):
            blk = b2[off[c] * pb.K + k * cnt[c]: off[c] * pb.K + (k + 1) * cnt[c]]
            assert np.array_equal(blk[:-1], b[po * pb.K + k * pc: po * pb.K + (k + 1) * pc])
            assert blk[-1] == 0.0


# ------------------------------------------------------------------ planted mistakes are caught

def test_planted_mistakes_fail_a_pin(monkeypatch):
    """Each plausible slip in the recursion breaks agreement with the dual form or FD."""
    pb = wl.problem_mlp_small()
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 6, 1, 4, 2)
    a, b = wl.random_alpha_beta(batch, 5, 2.0)
    ref = O.bound_dual(net, props, batch, a, b)
    good_relax = O.relax

    def drop_intercept(A, li, ui, al, sign):
        D, lam = good_relax(A, li, ui, al, sign)
        return D, lam * 0.0

    def wrong_branch(A, li, ui, al, sign):
        return good_relax(-A, li, ui, al, sign)

    for bad in (drop_intercept, wrong_branch):
        monkeypatch.setattr(O, "relax", bad)
        lb = O.bound(net, props, batch, a, b)
        monkeypatch.setattr(O, "relax", good_relax)
        assert np.max(np.abs(lb - ref)) > 1e-6, bad.__name__
    # a flipped split sign is caught by the sampled-minimum soundness pin or the dual form
    sb = wl.Batch(**{**batch.__dict__, "split_sign": (-batch.split_sign).astype(np.int8)})
    lb_flip = O.bound(net, props, sb, a, b)
    assert np.max(np.abs(lb_flip - ref)) > 1e-6


def test_infeasible_split_has_an_unbounded_dual():
    """A split that contradicts stability (z_j <= 0 on a layer-1 neuron whose exact interval has
    l_j > 0) leaves an empty subdomain: the LP of Eq. lp_verify_split is infeasible and the
    bound grows without limit in beta.  Once beta dominates, the growth per unit of beta is the
    minimum of z_j over the box (the exact layer-1 interval)."""
    from tests.helpers import oracle_setup
    pb = wl.problem_mlp_small()
    onet, props, unst = oracle_setup(pb)
    l = props["l"][0].astype(np.float64)
    d1 = pb.hidden_widths[0]
    j = int(np.argmax(l[:d1]))
    assert l[j] > 0.5
    lps = [LP.lp_value(onet, pb.x_lo[0], pb.x_hi[0], props["l"][0], props["u"][0], [(1, j, 1)], k)
           for k in range(pb.K)]
    assert all(np.isinf(v) for v in lps)
    batch = wl.pack_batch(pb.hidden_widths, pb.K, [len(x) for x in unst], [(0, np.array([j]), np.array([1], np.int8))])
    a = np.full(batch.n_alpha, 0.5)
    lb = {t: O.bound(onet, props, batch, a, np.full(batch.n_beta, float(t))) for t in (0, 10, 100, 1000)}
    assert np.all(lb[10] > lb[0]) and np.all(lb[100] > lb[10]) and np.all(lb[1000] > lb[100])
    # min over the box of z_j = W_j x + b_j, written out in FP64
    W = pb.layers[0].W.astype(np.float64)[j]
    zmin = np.sum(np.minimum(W * pb.x_lo[0], W * pb.x_hi[0])) + float(pb.layers[0].b[j])
    np.testing.assert_allclose((lb[1000] - lb[100]) / 900.0, zmin, rtol=1e-9)


def test_split_children_cover_the_parent():
    """Branching is sound: a subdomain's exact minimum is the smaller of its two children's
    (z_j >= 0 and z_j <= 0 cover every point), on the root and on a depth-1 parent."""
    from tests.helpers import oracle_setup
    pb = wl.make_problem("cover", wl.mlp_layers([5, 10, 10, 4], 1), 1, 0.15, 3, 1)
    onet, props, unst = oracle_setup(pb)
    offs = np.concatenate([[0], np.cumsum(pb.hidden_widths)])

    def lj(g):
        i = int(np.searchsorted(offs, g, side="right"))
        return i, int(g - offs[i - 1])

    un = [lj(g) for g in unst[0][:2]]
    args = (onet, pb.x_lo[0], pb.x_hi[0], props["l"][0], props["u"][0])
    for parent in ([], [(un[0][0], un[0][1], 1)]):
        i, j = un[1]
        for k in range(pb.K):
            p = LP.exact_min(*args, parent, k)
            c = [LP.exact_min(*args, parent + [(i, j, s)], k) for s in (-1, 1)]
            np.testing.assert_allclose(p, min(c), rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------ root bounds beyond layer 1

def _truncated(pb, i, props):
    """The network cut after layer i with C = [I; -I] (2 d_i specs: +z_j and -z_j), and the
    properties restricted to the hidden layers below i."""
    d = pb.layers[i - 1].d_out
    C = np.concatenate([np.eye(d), -np.eye(d)]).astype(np.float32)
    tnet = O.OracleNet(pb.layers[:i], C)
    h = int(sum(pb.hidden_widths[:i - 1]))
    tprops = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=props["l"][:, :h], u=props["u"][:, :h])
    return tnet, tprops, d


def _relaxation_gap_area(alpha, l, u, n=4001):
    """Area between ReLU and the lower line alpha * z over [l, u] (trapezoid rule)."""
    z = np.linspace(l, u, n)
    return np.trapezoid(np.maximum(z, 0.0) - alpha * z, z)


@pytest.mark.parametrize("maker", [lambda: tiny_problem(widths=(3, 6, 6, 5, 3), eps=0.3), tiny_conv_problem])
def test_root_bounds_equal_the_dual_form_on_the_truncated_net(maker):
    """Layer i >= 2 root bounds are CROWN's: on the net cut after layer i with the specs +-e_j,
    the dual objective of Theorem 3.2 at beta = 0 and the same lower slopes alpha' gives l_j and
    -u_j (the dual form is a second formula, not the back-substitution loop of root_bounds).
    FIXED rules use alpha' = v everywhere; the ADAPTIVE rule's alpha' is recomputed here as the
    lower line (z or 0) whose gap to ReLU over [l, u] has the smaller area."""
    pb = maker()
    net = O.OracleNet(pb.layers, pb.C)
    for rule, value in ((O.ALPHA_FIXED, 0.0), (O.ALPHA_FIXED, 0.3), (O.ALPHA_FIXED, 1.0), (O.ALPHA_ADAPTIVE, 0.5)):
        l, u = O.root_bounds(net, pb.x_lo, pb.x_hi, rule, value)
        props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
        for i in range(2, net.L):
            tnet, tprops, d = _truncated(pb, i, props)
            _, U = O.unstable_ranks(tnet, tprops["l"], tprops["u"])
            unst = [np.nonzero(O.unstable_mask(tprops["l"][p], tprops["u"][p]))[0] for p in range(pb.P)]
            subs = [(p, np.zeros(0, np.int64), np.zeros(0, np.int8)) for p in range(pb.P)]
            batch = wl.pack_batch(pb.hidden_widths[:i - 1], 2 * d, U, subs)
            alpha = np.zeros(batch.n_alpha)
            for p in range(pb.P):
                if rule == O.ALPHA_FIXED:
                    ap = np.full(len(unst[p]), value)
                else:
                    ap = np.array([1.0 if _relaxation_gap_area(1.0, tprops["l"][p, j], tprops["u"][p, j])
                                   <= _relaxation_gap_area(0.0, tprops["l"][p, j], tprops["u"][p, j]) else 0.0
                                   for j in unst[p]])
                off = int(batch.alpha_off[p])
                alpha[off:off + 2 * d * len(ap)] = np.tile(ap, 2 * d)
            g = O.bound_dual(tnet, tprops, batch, alpha, np.zeros(0)).reshape(pb.P, 2 * d)
            lo, hi = net.hoff[i - 1], net.hoff[i]
            np.testing.assert_allclose(g[:, :d], l[:, lo:hi], rtol=1e-10, atol=1e-10)
            np.testing.assert_allclose(-g[:, d:], u[:, lo:hi], rtol=1e-10, atol=1e-10)


def test_root_bounds_contain_the_exact_range_and_lie_below_the_lp():
    """Every root bound is sound and no tighter than the LP relaxation allows: on a tiny net,
    l_j <= p*_LP(z_j) <= min z_j (exact, by activation patterns) and u_j >= the matching maxima,
    for every neuron of layers 2 and 3 (Corollary 3.1 applied to the truncated net)."""
    pb = tiny_problem(widths=(3, 5, 5, 4, 2), eps=0.3)
    net, props, _ = _setup(pb)
    l, u = props["l"], props["u"]
    for i in range(2, net.L):
        tnet, tprops, d = _truncated(pb, i, props)
        lo = net.hoff[i - 1]
        args = (tnet, pb.x_lo[0].astype(np.float64), pb.x_hi[0].astype(np.float64), tprops["l"][0], tprops["u"][0], [])
        for j in range(d):
            zmin = LP.exact_min(*args, j)
            zmax = -LP.exact_min(*args, d + j)
            pmin = LP.lp_value(*args, j)
            pmax = -LP.lp_value(*args, d + j)
            assert l[0, lo + j] <= pmin + 1e-9 and pmin <= zmin + 1e-9
            assert u[0, lo + j] >= pmax - 1e-9 and pmax >= zmax - 1e-9
            assert zmin <= zmax + 1e-12


# ------------------------------------------------------------------ neuron codes

def test_neuron_codes_hand_derived_cases():
    """Codes for hand-picked l, u (boundaries l = 0, u = 0, l = u = 0) and split lists, including
    splits on stable neurons, written out by hand in tests/golden/neuron_codes_cases.json."""
    g = json.load(open(os.path.join(GOLD, "neuron_codes_cases.json")))
    H = len(g["l"])
    layers = wl.mlp_layers([3, H, 2], 0)
    net = O.OracleNet(layers, np.eye(2, dtype=np.float32)[:1])
    l = np.array([g["l"]], np.float64)
    u = np.array([g["u"]], np.float64)
    _, U = O.unstable_ranks(net, l, u)
    subs = [(0, np.array([s[0] for s in r["splits"]], np.int64), np.array([s[1] for s in r["splits"]], np.int8))
            for r in g["rows"]]
    batch = wl.pack_batch([H], 1, U, subs)
    rows = O.expand_rows(net, batch, l, u)
    codes = O.neuron_codes(net, rows, l, u)[1]
    assert np.array_equal(codes, np.array([r["codes"] for r in g["rows"]], np.int8))


def test_neuron_codes_agree_with_the_relaxation():
    """The code of each (row, neuron) matches the slope the relaxation applies: D = 1 and no
    intercept for codes 1 and 3, D = 0 and no intercept for 0 and 4, and alpha (A >= 0) or the
    upper chord (A < 0) for code 2."""
    pb = wl.problem_mlp_small(seed=2)
    net, props, unst = _setup(pb)
    batch = wl.random_batch(pb, unst, 20, 0, 4, 9)
    a, _ = wl.random_alpha_beta(batch, 1)
    rows = O.expand_rows(net, batch, props["l"], props["u"])
    codes = O.neuron_codes(net, rows, props["l"], props["u"])
    rng = np.random.default_rng(0)
    for i in range(1, net.L):
        lo, hi = net.hoff[i - 1], net.hoff[i]
        li, ui = props["l"][rows.prop][:, lo:hi], props["u"][rows.prop][:, lo:hi]
        al = np.where(rows.alpha_idx[i] >= 0, a[np.maximum(rows.alpha_idx[i], 0)], 0.0)
        A = rng.normal(size=li.shape)
        D, lam = O.relax(A, li, ui, al, rows.sign[i])
        c = codes[i]
        one = (c == 1) | (c == 3)
        zero = (c == 0) | (c == 4)
        assert np.all(D[one] == 1.0) and np.all(lam[one] == 0.0)
        assert np.all(D[zero] == 0.0) and np.all(lam[zero] == 0.0)
        two = c == 2
        assert np.all(np.where(two & (A >= 0), D == al, True))
        chord = ui / np.where(two, ui - li, 1.0)
        assert np.all(np.where(two & (A < 0), np.isclose(D, chord, rtol=1e-15), True))
        assert np.all(np.where(two & (A < 0), lam > 0, True))
        assert np.all((c == 2).sum(axis=1) <= len(unst[0]))

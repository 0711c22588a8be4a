"""Pins of the joint intermediate-bound oracle (Section 3.3) against the paper and the mathematics:
the root bounds and the plain bound it must reduce to, the dual form of every target pass
(Theorem 3.2), the exact minima over each subdomain, finite differences, and the claim that
recomputed bounds take the final bound past the LP with fixed intermediate bounds."""
import numpy as np
import pytest

from oracle import bcrown_oracle as O
from oracle import joint as J
from oracle import lp_pins as LP
from paper_2103_06624_gb300 import workloads as wl


def _problem(widths=(5, 8, 8, 8, 3), seed=3, eps=0.2, K=3):
    pb = wl.make_problem("joint", wl.mlp_layers(list(widths), seed), 1, eps, K, seed)
    net = O.OracleNet(pb.layers, pb.C)
    l, u = O.root_bounds(net, pb.x_lo, pb.x_hi)
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
    unst = np.nonzero(O.unstable_mask(l[0], u[0]))[0]
    return pb, net, props, unst


def _batch(pb, unst, n_sub, depth, seed):
    rng = np.random.default_rng(seed)
    subs = [(0, np.zeros(0, np.int64), np.zeros(0, np.int8))]
    for _ in range(n_sub - 1):
        ns, ss = wl.random_split_sets(rng, unst, 1, depth)
        subs.append((0, ns, ss))
    return wl.pack_batch(pb.hidden_widths, pb.K, [len(unst)], subs)


def _random_vars(net, props, batch, seed, beta_max=0.5):
    rng = np.random.default_rng(seed)
    lay = J.joint_layout(net, batch, props["l"], props["u"])
    a = rng.uniform(0, 1, batch.n_alpha)
    b = rng.uniform(0, beta_max, batch.n_beta)
    ap = rng.uniform(0, 1, lay.n_alpha_p)
    bp = rng.uniform(0, beta_max, lay.n_beta_p)
    return a, b, ap, bp


def test_layout_sizes():
    pb, net, props, unst = _problem()
    batch = _batch(pb, unst, 4, 3, 0)
    lay = J.joint_layout(net, batch, props["l"], props["u"])
    offs = net.hoff
    m = O.unstable_mask(props["l"][0], props["u"][0])
    per = 2 * sum(int(m[:offs[i - 1]].sum()) for i in range(2, net.L))
    assert lay.n_alpha_p == 4 * per and list(lay.ap_off) == [0, per, 2 * per, 3 * per, 4 * per]
    assert lay.n_beta_p == 2 * (net.L - 2) * int(batch.split_cnt.sum())


def test_no_split_at_the_adaptive_rule_reproduces_root_bounds_and_bound():
    """alpha' at CROWN's adaptive rule and beta' = 0 on an unsplit subdomain: every target pass is
    the root computation of Section 3.3, so l, u are the root bounds and the final bound is
    Theorem 3.1's with those bounds."""
    pb, net, props, unst = _problem()
    batch = wl.pack_batch(pb.hidden_widths, pb.K, [len(unst)], [(0, np.zeros(0, np.int64), np.zeros(0, np.int8))] * 2)
    ap = J.init_alpha_p(net, batch, props["l"], props["u"])
    bp = np.zeros(J.joint_layout(net, batch, props["l"], props["u"]).n_beta_p)
    a, b, _, _ = _random_vars(net, props, batch, 1)
    import torch
    lb, l, u, raw = J.joint_forward(net, props, batch, *[torch.tensor(v) for v in (a, b, ap, bp)], raw=True)
    for bb in range(2):
        np.testing.assert_allclose(l[bb].numpy(), props["l"][0], rtol=0, atol=1e-12)
        np.testing.assert_allclose(u[bb].numpy(), props["u"][0], rtol=0, atol=1e-12)
        for i in range(2, net.L):
            sl = slice(net.hoff[i - 1], net.hoff[i])
            np.testing.assert_allclose(raw[(bb, i, 0)].detach().numpy(), props["l"][0, sl], rtol=0, atol=1e-12)
            np.testing.assert_allclose(raw[(bb, i, 1)].detach().numpy(), props["u"][0, sl], rtol=0, atol=1e-12)
    np.testing.assert_allclose(lb.numpy(), O.bound(net, props, batch, a, b), rtol=0, atol=1e-12)


def _truncated(pb, i, sign):
    """The network cut after layer i with C = sign * I: its specs are +-z^(i)."""
    d = pb.layers[i - 1].d_out
    return O.OracleNet(pb.layers[:i], sign * np.eye(d)), d


def test_every_target_pass_equals_the_dual_form_of_the_truncated_network():
    """Theorem 3.2 on the network truncated at target layer i with C = +I (lower bounds of z^(i))
    and C = -I (the negated upper bounds), with the subdomain's current bounds of layers < i,
    alpha' broadcast to every row and beta' on the splits in layers < i."""
    pb, net, props, unst = _problem()
    batch = _batch(pb, unst, 5, 4, 2)
    a, b, ap, bp = _random_vars(net, props, batch, 3)
    import torch
    _, l, u, raw = J.joint_forward(net, props, batch, *[torch.tensor(v) for v in (a, b, ap, bp)], raw=True)
    lay = J.joint_layout(net, batch, props["l"], props["u"])
    checked = 0
    for bb in range(batch.B):
        off, cnt = int(batch.split_off[bb]), int(batch.split_cnt[bb])
        for i in range(2, net.L):
            H_ = int(net.hoff[i - 1])
            lt, ut = l[bb].numpy()[None, :H_], u[bb].numpy()[None, :H_]
            keep = [t for t in range(cnt) if int(batch.split_layer[off + t]) < i]
            gidx = np.array([net.hoff[int(batch.split_layer[off + t]) - 1] + int(batch.split_idx[off + t])
                             for t in keep], np.int64)
            sg = np.array([int(batch.split_sign[off + t]) for t in keep], np.int8)
            sub_unst = np.nonzero(O.unstable_mask(lt[0], ut[0]))[0]
            for direction, sign in ((0, 1.0), (1, -1.0)):
                tnet, d = _truncated(pb, i, sign)
                tb = wl.pack_batch(pb.hidden_widths[:i - 1], d, [len(sub_unst)], [(0, gidx, sg)])
                s, n = J._alpha_p_block(lay, net, batch, bb, i, direction)
                al_row = ap[s:s + n][lay.rank[0][sub_unst]]
                sb, _ = J._beta_p_block(net, batch, bb, i, direction)
                be_row = bp[sb:sb + cnt][keep]
                tprops = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=lt, u=ut)
                g = O.bound_dual(tnet, tprops, tb, np.tile(al_row, d), np.tile(be_row, d))
                got = raw[(bb, i, direction)].detach().numpy()
                np.testing.assert_allclose(sign * got, g, rtol=1e-10, atol=1e-10)
                checked += 1
    assert checked == batch.B * (net.L - 2) * 2


def test_bounds_lie_below_the_exact_minima_over_each_subdomain():
    """l^(i)_j <= min z^(i)_j and u^(i)_j >= max z^(i)_j over the box with the subdomain's splits in
    layers < i (activation patterns enumerated); the final bound below the exact minimum of each
    spec over the subdomain."""
    pb, net, props, unst = _problem(widths=(4, 6, 5, 4, 3), seed=5, eps=0.2)
    batch = _batch(pb, unst, 4, 3, 4)
    a, b, ap, bp = _random_vars(net, props, batch, 5)
    lb, l, u = J.joint_bound(net, props, batch, a, b, ap, bp)
    off_l = net.hoff
    for bb in range(batch.B):
        o, c = int(batch.split_off[bb]), int(batch.split_cnt[bb])
        splits = [(int(batch.split_layer[o + t]), int(batch.split_idx[o + t]), int(batch.split_sign[o + t]))
                  for t in range(c)]
        for i in range(2, net.L):
            sp_i = [s for s in splits if s[0] < i]
            for sign in (1.0, -1.0):
                tnet, d = _truncated(pb, i, sign)
                H_ = int(off_l[i - 1])
                for j in range(d):
                    ex = LP.exact_min(tnet, pb.x_lo[0], pb.x_hi[0], props["l"][0][:H_], props["u"][0][:H_], sp_i, j)
                    if not np.isfinite(ex):
                        continue
                    if sign > 0:
                        assert l[bb, off_l[i - 1] + j] <= ex + 1e-9
                    else:
                        assert u[bb, off_l[i - 1] + j] >= -ex - 1e-9
        for k in range(pb.K):
            ex = LP.exact_min(net, pb.x_lo[0], pb.x_hi[0], props["l"][0], props["u"][0], splits, k)
            assert lb[bb * pb.K + k] <= ex + 1e-9


def test_gradient_matches_central_finite_differences():
    pb, net, props, unst = _problem()
    batch = _batch(pb, unst, 3, 3, 6)
    theta = list(_random_vars(net, props, batch, 7))
    lb, *g = J.joint_grad(net, props, batch, *theta)
    rng = np.random.default_rng(8)
    h = 1e-6
    agreed = [0, 0, 0, 0]

    def f(th):
        return J.joint_bound(net, props, batch, *th)[0].sum()

    for q in range(4):
        n = len(theta[q])
        for idx in rng.choice(n, size=min(n, 12), replace=False):
            fd = []
            for hh in (h, h / 2):
                tp = [v.copy() for v in theta]
                tm = [v.copy() for v in theta]
                tp[q][idx] += hh
                tm[q][idx] -= hh
                fd.append((f(tp) - f(tm)) / (2 * hh))
            if abs(fd[0] - fd[1]) > 1e-6 * max(1.0, abs(fd[0])):
                continue      # a kink of the piecewise-linear bound within +-h
            assert abs(g[q][idx] - fd[0]) <= 1e-6 * max(1.0, abs(fd[0])), (q, idx, g[q][idx], fd[0])
            agreed[q] += 1
    assert all(a_ >= 4 for a_ in agreed), agreed
    # alpha' and beta' reach the final bound: some of their derivatives are nonzero
    assert np.abs(g[2]).max() > 1e-6 and np.abs(g[3]).max() > 1e-6


def test_switches_hold_their_groups_and_best_tracking_never_loses():
    pb, net, props, unst = _problem()
    batch = _batch(pb, unst, 3, 3, 9)
    a0, b0 = np.full(batch.n_alpha, 0.5), np.zeros(batch.n_beta)
    ap0 = J.init_alpha_p(net, batch, props["l"], props["u"])
    bp0 = np.zeros(J.joint_layout(net, batch, props["l"], props["u"]).n_beta_p)
    lb0 = J.joint_bound(net, props, batch, a0, b0, ap0, bp0)[0]
    cfg = J.JointCfg(iters=5)
    for fa, fb in ((True, False), (False, True), (False, False)):
        lb, a, b, ap, bp, _, _, hist = J.joint_optimize(net, props, batch, a0, b0, ap0, bp0,
                                                         J.replace(cfg, freeze_alpha=fa, freeze_beta=fb))
        if fa:
            assert np.array_equal(a, a0) and np.array_equal(ap, ap0)
        if fb:
            assert np.array_equal(b, b0) and np.array_equal(bp, bp0)
        s = lb.reshape(batch.B, pb.K).sum(axis=1)
        assert np.all(s >= lb0.reshape(batch.B, pb.K).sum(axis=1) - 1e-12)
        assert np.allclose(s, np.max([h_.reshape(batch.B, pb.K).sum(axis=1) for h_ in hist], axis=0))


def test_recomputed_bounds_take_the_bound_past_the_fixed_bound_lp():
    """Section 3.3: with intermediate bounds optimised jointly, beta-CROWN can exceed the LP of
    Eq. lp_verify_split built on the fixed root bounds (which bounds every fixed-bound alpha, beta
    by Corollary 3.1)."""
    pb, net, props, unst = _problem(widths=(4, 8, 8, 6, 3), seed=11, eps=0.35)
    batch = _batch(pb, unst, 3, 2, 12)
    a0, b0 = np.full(batch.n_alpha, 0.5), np.zeros(batch.n_beta)
    ap0 = J.init_alpha_p(net, batch, props["l"], props["u"])
    bp0 = np.zeros(J.joint_layout(net, batch, props["l"], props["u"]).n_beta_p)
    lb, *_ = J.joint_optimize(net, props, batch, a0, b0, ap0, bp0, J.JointCfg(iters=40, lr_alpha=0.1, lr_beta=0.1))
    gain = []
    for bb in range(batch.B):
        o, c = int(batch.split_off[bb]), int(batch.split_cnt[bb])
        splits = [(int(batch.split_layer[o + t]), int(batch.split_idx[o + t]), int(batch.split_sign[o + t]))
                  for t in range(c)]
        for k in range(pb.K):
            lp = LP.lp_value(net, pb.x_lo[0], pb.x_hi[0], props["l"][0], props["u"][0], splits, k)
            if np.isfinite(lp):
                gain.append(lb[bb * pb.K + k] - lp)
    assert max(gain) > 1e-3, gain

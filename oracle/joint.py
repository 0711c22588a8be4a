"""FP64 reference for the joint optimisation of intermediate-layer bounds (test infrastructure only).

Section 3.3 ("Joint Optimization of Free Variables in beta-CROWN"): the bounds l^(i), u^(i)
of every hidden layer i >= 2 are themselves beta-CROWN bounds (Theorem 3.1 with the
objective f := z^(i)_j for l, f := -z^(i)_j for u), each with its own free variables
alpha', beta'.  The final bound g then depends on alpha' and beta' through the relaxations
built from l, u, and all of (alpha, beta, alpha', beta') are optimised together
(Eq. opt_non_convex).  Following the section's O(L^2 d) variant, alpha' and beta' are shared
by all target neurons of one layer: one vector per (subdomain, target layer i, direction).

Plain and slow: the recursion of Theorem 3.1 written with torch float64 tensors, one
subdomain at a time, so that torch's automatic differentiation (the library primitive the
paper itself uses for the gradient, Section 3.1) supplies d g / d(alpha, beta, alpha', beta').

Readings (where Section 3.3 leaves details open):

* Variable space.  alpha' of (subdomain b, target layer i, direction) has one entry per
  root-unstable neuron of b's property in layers 1..i-1 (the property's unstable neurons in
  layer-major rank order, so a prefix of the rank order).  beta' of (b, i, direction) has one
  entry per entry of b's split list; entries of splits in layers >= i are unused (zero
  gradient).  Direction 0 bounds z^(i) from below (l), direction 1 bounds -z^(i) (u = -bound).
* Layout.  Per subdomain, alpha' blocks are ordered by target layer i = 2..L-1, then
  direction, then rank; beta' blocks the same with the split position inside.  Subdomain b's
  alpha' block starts at the sum of the earlier subdomains' sizes; its beta' block at
  2 (L-2) split_off[b].
* Layer 1 keeps the root's bounds (an interval of an affine map, already exact).  For
  i >= 2 the new bounds are intersected with the root's: l = max(l_root, l_new),
  u = min(u_root, u_new) -- both are valid on the subdomain, so the intersection is.
* Neurons that the tighter bounds make stable (l >= 0 or u <= 0) take D = 1 or 0; their
  alpha entries stay in the layout with zero gradient.  Split neurons ignore l, u as before.
* The objective for the shared alpha', beta' of a subdomain is the sum of its K spec bounds.
* Best tracking is per subdomain on that sum (l, u belong to the subdomain, not to a row):
  the variables of the best iteration are kept and the final bound is recomputed there.
* Ablation switches (Table A4): freezing alpha holds alpha and alpha' at their inputs,
  freezing beta holds beta and beta'.

Parity pins (``tests/test_oracle_joint.py``): with alpha' at the root's adaptive rule, beta' = 0
and no split, the bounds equal ``root_bounds`` and the final bound equals ``bound``; every
target pass equals the dual nu-form ``bound_dual`` (Theorem 3.2) of the network truncated at
the target layer with C = +-I; bounds of every neuron lie below / above its exact minimum /
maximum over the subdomain (activation patterns enumerated); the autograd gradient matches
float64 central finite differences.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np
import scipy.sparse as sp
import torch

from . import bcrown_oracle as O

F64 = torch.float64


# --------------------------------------------------------------------------------------
# Layout of alpha' and beta'
# --------------------------------------------------------------------------------------

@dataclass
class JointLayout:
    rank: np.ndarray       # [P, H] root rank among the property's unstable neurons, -1 if stable
    U: np.ndarray          # [P] root-unstable neurons per property
    first: np.ndarray      # [P, L] first[p, i] = unstable neurons of p in layers 1..i-1
    ap_off: np.ndarray     # [B + 1] alpha' block offsets
    n_alpha_p: int
    n_beta_p: int


def joint_layout(net, batch, l_root, u_root) -> JointLayout:
    rank, U = O.unstable_ranks(net, l_root, u_root)
    m = O.unstable_mask(np.asarray(l_root), np.asarray(u_root))
    P = m.shape[0]
    first = np.zeros((P, net.L), np.int64)
    for i in range(1, net.L):
        first[:, i] = m[:, :net.hoff[i - 1]].sum(axis=1)
    sizes = np.array([2 * int(first[int(p), 2:net.L].sum()) for p in batch.prop_of], np.int64)
    ap_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    nb = 2 * max(net.L - 2, 0) * int(np.sum(batch.split_cnt))
    return JointLayout(rank, U, first, ap_off, int(ap_off[-1]), nb)


def _alpha_p_block(lay, net, batch, b, i, direction):
    """Start and length of alpha' of (subdomain b, target layer i, direction)."""
    p = int(batch.prop_of[b])
    start = int(lay.ap_off[b])
    for t in range(2, i):
        start += 2 * int(lay.first[p, t])
    n = int(lay.first[p, i])
    return start + direction * n, n


def _beta_p_block(net, batch, b, i, direction):
    cnt = int(batch.split_cnt[b])
    start = 2 * (net.L - 2) * int(batch.split_off[b]) + (2 * (i - 2) + direction) * cnt
    return start, cnt


def init_alpha_p(net, batch, l_root, u_root):
    """alpha' at the root's adaptive rule (1 where u >= -l, else 0), per source neuron."""
    lay = joint_layout(net, batch, l_root, u_root)
    ap = np.zeros(lay.n_alpha_p)
    for b in range(batch.B):
        p = int(batch.prop_of[b])
        unst = np.nonzero(lay.rank[p] >= 0)[0]
        rule = np.where(np.asarray(u_root)[p, unst] >= -np.asarray(l_root)[p, unst], 1.0, 0.0)
        for i in range(2, net.L):
            for direction in (0, 1):
                s, n = _alpha_p_block(lay, net, batch, b, i, direction)
                ap[s:s + n] = rule[:n]
    return ap


# --------------------------------------------------------------------------------------
# The bound with recomputed intermediate bounds (torch float64, differentiable)
# --------------------------------------------------------------------------------------

def _tw(W):
    if sp.issparse(W):
        W = W.tocoo()
        idx = torch.tensor(np.vstack([W.row, W.col]), dtype=torch.long)
        return torch.sparse_coo_tensor(idx, torch.tensor(W.data, dtype=F64), W.shape).coalesce()
    return torch.tensor(np.asarray(W, np.float64))


def _mm(A, W):
    """A [R, d_i] times W [d_i, d_{i-1}]."""
    if W.is_sparse:
        return torch.sparse.mm(W.t(), A.t()).t()
    return A @ W


def _relax(A, li, ui, al, sign):
    """D, lambda of Lemma 2.1 / Eq. definition_D with l, u, alpha, split signs broadcast over rows."""
    act = li >= 0
    inact = (~act) & (ui <= 0)
    unst = (~act) & (~inact)
    den = torch.where(unst, ui - li, torch.ones_like(ui))
    slope = ui / den
    icpt = -ui * li / den
    one, zero = torch.ones_like(A), torch.zeros_like(A)
    D = torch.where(A >= 0, al.expand_as(A), slope.expand_as(A))
    D = torch.where(unst.expand_as(A), D, torch.where(act.expand_as(A), one, zero))
    lam = torch.where(unst.expand_as(A) & (A < 0), icpt.expand_as(A), zero)
    split = (sign != 0).expand_as(A)
    D = torch.where(split, torch.where((sign == -1).expand_as(A), one, zero), D)
    lam = torch.where(split, zero, lam)
    return D, lam


class _Sub:
    """One subdomain's split list as per-layer sign and beta-slot vectors."""

    def __init__(self, net, batch, b):
        self.sign = [None] + [torch.zeros(net.d[i], dtype=torch.int64) for i in range(1, net.L)]
        self.slot = [None] + [torch.full((net.d[i],), -1, dtype=torch.int64) for i in range(1, net.L)]
        off, cnt = int(batch.split_off[b]), int(batch.split_cnt[b])
        self.cnt = cnt
        for t in range(cnt):
            i = int(batch.split_layer[off + t])
            j = int(batch.split_idx[off + t])
            self.sign[i][j] = int(batch.split_sign[off + t])
            self.slot[i][j] = t


def _take(vec, idx):
    """vec[idx] with 0 where idx < 0 (differentiable in vec)."""
    safe = torch.clamp(idx, min=0)
    out = vec[safe] if vec.numel() else torch.zeros(idx.shape, dtype=F64)
    return torch.where(idx >= 0, out, torch.zeros_like(out))


def _backsub(tn, net, sub, top, A, c, l, u, al_of, be_of, xlo, xhi):
    """Theorem 3.1's recursion from layer `top` - 1 down to the input, for rows A (objective
    A h^(top-1) + c), with the subdomain's bounds l, u and alpha / beta given per layer by
    al_of(m) -> [d_m] and be_of(m) -> [d_m].  Returns the lower bound of every row."""
    for m in range(top - 1, 0, -1):
        lo, hi = int(net.hoff[m - 1]), int(net.hoff[m])
        sg = sub.sign[m].unsqueeze(0)
        D, lam = _relax(A, l[lo:hi].unsqueeze(0), u[lo:hi].unsqueeze(0), al_of(m).unsqueeze(0), sg)
        Lam = A * D + be_of(m).unsqueeze(0) * sg.to(A.dtype)
        c = c + Lam @ tn["b"][m] + (A * lam).sum(dim=1)
        A = _mm(Lam, tn["W"][m])
    return c + torch.minimum(A * xlo, A * xhi).sum(dim=1)


def _tensors(net):
    return {"W": [None] + [_tw(net.W[i]) for i in range(1, net.L)],
            "Wd": [None] + [torch.tensor(net.W[i].toarray() if sp.issparse(net.W[i]) else net.W[i])
                            for i in range(1, net.L)],
            "b": [None] + [torch.tensor(net.b[i]) for i in range(1, net.L)],
            "Wbar": torch.tensor(net.Wbar), "bbar": torch.tensor(net.bbar)}


def joint_forward(net, props, batch, alpha, beta, alpha_p, beta_p, raw=False):
    """lb [B K] of every row and the subdomains' recomputed bounds l, u [B, H] (torch tensors;
    alpha .. beta_p may require grad).  props holds the root's x_lo, x_hi, l, u per property.
    With raw, also the unintersected target-pass bounds {(b, i, direction): tensor [d_i]}."""
    tn = _tensors(net)
    lay = joint_layout(net, batch, props["l"], props["u"])
    K = net.K
    lbs, ls, us = [], [], []
    raws = {}
    for b in range(batch.B):
        p = int(batch.prop_of[b])
        sub = _Sub(net, batch, b)
        xlo = torch.tensor(np.asarray(props["x_lo"], np.float64)[p])
        xhi = torch.tensor(np.asarray(props["x_hi"], np.float64)[p])
        l = torch.tensor(np.asarray(props["l"], np.float64)[p])
        u = torch.tensor(np.asarray(props["u"], np.float64)[p])
        rank = torch.tensor(lay.rank[p])
        for i in range(2, net.L):
            lo, hi = int(net.hoff[i - 1]), int(net.hoff[i])
            new = []
            for direction in (0, 1):
                s, n = _alpha_p_block(lay, net, batch, b, i, direction)
                ap = alpha_p[s:s + n]
                sb, nb = _beta_p_block(net, batch, b, i, direction)
                bp = beta_p[sb:sb + nb]

                def al_of(m, ap=ap, n=n):
                    rk = rank[int(net.hoff[m - 1]):int(net.hoff[m])]
                    return _take(ap, torch.where(rk < n, rk, torch.full_like(rk, -1)))

                def be_of(m, bp=bp):
                    return _take(bp, sub.slot[m])

                sgn = 1.0 if direction == 0 else -1.0
                A = sgn * tn["Wd"][i]
                c = sgn * tn["b"][i]
                new.append(_backsub(tn, net, sub, i, A, c, l, u, al_of, be_of, xlo, xhi))
            if raw:
                raws[(b, i, 0)], raws[(b, i, 1)] = new[0], -new[1]
            l = torch.cat([l[:lo], torch.maximum(l[lo:hi], new[0]), l[hi:]])
            u = torch.cat([u[:lo], torch.minimum(u[lo:hi], -new[1]), u[hi:]])
        ls.append(l)
        us.append(u)
        Up = int(lay.U[p])
        for k in range(K):
            a0 = int(batch.alpha_off[b]) + k * Up
            al_row = alpha[a0:a0 + Up]
            b0 = int(batch.split_off[b]) * K + k * sub.cnt
            be_row = beta[b0:b0 + sub.cnt]

            def al_of(m, al_row=al_row):
                return _take(al_row, rank[int(net.hoff[m - 1]):int(net.hoff[m])])

            def be_of(m, be_row=be_row):
                return _take(be_row, sub.slot[m])

            lbs.append(_backsub(tn, net, sub, net.L, tn["Wbar"][k:k + 1], tn["bbar"][k:k + 1], l, u,
                                al_of, be_of, xlo, xhi))
    lb = torch.cat(lbs) if lbs else torch.zeros(0, dtype=F64)
    L_ = torch.stack(ls) if ls else torch.zeros((0, int(sum(net.hidden))), dtype=F64)
    U_ = torch.stack(us) if us else torch.zeros((0, int(sum(net.hidden))), dtype=F64)
    if raw:
        return lb, L_, U_, raws
    return lb, L_, U_


def _leaf(x):
    return torch.tensor(np.asarray(x, np.float64), requires_grad=True)


def joint_bound(net, props, batch, alpha, beta, alpha_p, beta_p):
    """(lb [B K], l [B, H], u [B, H]) as float64 arrays."""
    with torch.no_grad():
        lb, l, u = joint_forward(net, props, batch, *[torch.tensor(np.asarray(v, np.float64))
                                                       for v in (alpha, beta, alpha_p, beta_p)])
    return lb.numpy(), l.numpy(), u.numpy()


def joint_grad(net, props, batch, alpha, beta, alpha_p, beta_p):
    """lb and d(sum of lb)/d(alpha, beta, alpha', beta') by automatic differentiation."""
    leaves = [_leaf(v) for v in (alpha, beta, alpha_p, beta_p)]
    lb, _, _ = joint_forward(net, props, batch, *leaves)
    if lb.numel():
        lb.sum().backward()
    grads = [v.grad.numpy() if v.grad is not None else np.zeros(v.shape) for v in leaves]
    return (lb.detach().numpy(), *grads)


# --------------------------------------------------------------------------------------
# Projected Adam on (alpha, beta, alpha', beta') with the ablation switches
# --------------------------------------------------------------------------------------

@dataclass
class JointCfg(O.AdamCfg):
    freeze_alpha: bool = False
    freeze_beta: bool = False


def subdomain_of_params(net, batch, lay, U):
    """Subdomain owning each alpha, beta, alpha' and beta' entry."""
    ra, rb = O.row_of_params(net, batch, U)
    K = net.K
    sp_ = np.zeros(lay.n_alpha_p, np.int64)
    sb = np.zeros(lay.n_beta_p, np.int64)
    for b in range(batch.B):
        sp_[lay.ap_off[b]:lay.ap_off[b + 1]] = b
        s = 2 * (net.L - 2) * int(batch.split_off[b])
        sb[s:s + 2 * (net.L - 2) * int(batch.split_cnt[b])] = b
    return ra // K, rb // K, sp_, sb


def joint_optimize(net, props, batch, alpha0, beta0, alpha_p0, beta_p0, cfg=JointCfg()):
    """Returns (lb at the best iterate, alpha, beta, alpha', beta', l, u, history of lb).

    Iteration t evaluates g and its gradient at theta_t, keeps per subdomain the iterate with
    the largest sum of its spec bounds, then takes one projected Adam step per group with
    learning rates lr0 * decay^t (alpha, alpha' in [0, 1] at lr_alpha; beta, beta' >= 0 at
    lr_beta).  Frozen groups are not stepped."""
    lay = joint_layout(net, batch, props["l"], props["u"])
    sa, sbeta, sap, sbp = subdomain_of_params(net, batch, lay, lay.U)
    theta = [np.asarray(v, np.float64).copy() for v in (alpha0, beta0, alpha_p0, beta_p0)]
    ms = [np.zeros_like(v) for v in theta]
    vs = [np.zeros_like(v) for v in theta]
    owner = [sa, sbeta, sap, sbp]
    lr = [cfg.lr_alpha, cfg.lr_beta, cfg.lr_alpha, cfg.lr_beta]
    box = [(0.0, 1.0), (0.0, np.inf), (0.0, 1.0), (0.0, np.inf)]
    frozen = [cfg.freeze_alpha, cfg.freeze_beta, cfg.freeze_alpha, cfg.freeze_beta]
    B, K = batch.B, net.K
    best = np.full(B, -np.inf)
    kept = [v.copy() for v in theta]
    hist = []
    for t in range(cfg.iters):
        lb, *g = joint_grad(net, props, batch, *theta)
        hist.append(lb.copy())
        score = lb.reshape(B, K).sum(axis=1) if B else np.zeros(0)
        improved = score > best
        best = np.where(improved, score, best)
        for q in range(4):
            kept[q] = np.where(improved[owner[q]], theta[q], kept[q])
        fac = cfg.decay ** t
        for q in range(4):
            if not frozen[q]:
                theta[q], ms[q], vs[q] = O.adam_ascent_step(theta[q], ms[q], vs[q], g[q], t, lr[q] * fac,
                                                            cfg, *box[q])
    lb, l, u = joint_bound(net, props, batch, *kept)
    return lb, kept[0], kept[1], kept[2], kept[3], l, u, hist


def plain_cfg(cfg: JointCfg) -> O.AdamCfg:
    """The optimiser settings without the switches (for the joint-off ablation)."""
    return O.AdamCfg(**{f: getattr(cfg, f) for f in O.AdamCfg.__dataclass_fields__})


__all__ = ["JointLayout", "joint_layout", "init_alpha_p", "joint_forward", "joint_bound", "joint_grad",
           "JointCfg", "joint_optimize", "plain_cfg", "replace"]

"""FP64 reference for batched beta-CROWN bound propagation (test infrastructure only).

Plain, slow and meant to be read beside the paper (Wang et al., "Beta-CROWN:
Efficient Bound Propagation with Per-neuron Split Constraints for Complete and
Incomplete Neural Network Verification", arXiv 2103.06624).  Every layer,
fully connected or convolutional, is an explicit (dense or sparse) matrix
built from its definition; the bound is computed row by row in float64 with
NumPy/SciPy matrix products as the only library steps.  Rows (subdomain,
spec) are independent, so the functions take all rows of a batch at once.

Functions and what pins them (tests under ``tests/test_oracle_*.py``):

* ``bound``          -- Theorem 3.1 in the recursive form of Eq. definition_A /
                        Lemma A.2 (Eq. eq_a, with the two constant terms the
                        proof's induction carries).  Pinned by: the explicit
                        Theorem 3.1 terms ``bound_explicit``; the dual nu-form
                        ``bound_dual`` (Theorem 3.2, Eq. nu_eq); the closed
                        form at eps = 0; brute force over box vertices for
                        networks with no unstable neuron; sampled minima over
                        the subdomain; the scipy LP of Eq. lp_verify_split
                        (Corollary 3.1); exhaustive activation patterns.
* ``bound_explicit`` -- Theorem 3.1 with a, P, q, c written out via Omega
                        (Appendix A, Definition A.1).  Pinned against ``bound``
                        and ``bound_dual``.
* ``bound_dual``     -- Theorem 3.2 dual objective g(alpha, beta).  Pinned as above.
* ``grad``           -- adjoint of the bound w.r.t. alpha and beta.  Pinned by
                        float64 central finite differences of ``bound``.
* ``root_bounds``    -- CROWN intermediate bounds (Section 3.3, Lemma 2.2) with
                        fixed alpha'.  Pinned by: exact interval for layer 1
                        (vertex brute force), soundness against sampled z.
* ``optimize``       -- projected Adam ascent on alpha in [0,1], beta >= 0
                        (Eq. opt_alpha_beta; Appendix C.1 hyper-parameters).
                        One step pinned against torch.optim.Adam (maximize).
* ``batch_split``    -- children of a split (Algorithm 1, batch_split).  Pinned
                        by its definition on hand-written cases.

Readings of points the paper leaves open:
split overrides stability; l >= 0 is active, u <= 0 inactive, l < 0 < u
unstable; a tie A_j = 0 takes the alpha branch; each (subdomain, spec) row has
its own alpha and beta; x* takes x_lo where A^(0)_m = 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

# neuron codes (per row, per hidden neuron) derived from l, u and the split list
CODE_INACTIVE, CODE_ACTIVE, CODE_UNSTABLE, CODE_SPLIT_POS, CODE_SPLIT_NEG = 0, 1, 2, 3, 4


# --------------------------------------------------------------------------------------
# Network as explicit matrices (Section 2.1, Eq. 1)
# --------------------------------------------------------------------------------------

def conv_matrix(ly) -> sp.csr_matrix:
    """Sparse matrix of a convolution, built from its definition.

    z[co, oy, ox] = sum_{ci, ky, kx} W[co, ci, ky, kx] * x[ci, oy*s - p + ky, ox*s - p + kx]
    with x = 0 outside the image; indices are flattened channel-major (C, H, W).
    """
    cout, cin, k, _ = ly.W.shape
    _, H, Wd = ly.in_shape
    _, Ho, Wo = ly.out_shape
    s, p = ly.stride, ly.pad
    co, ci, oy, ox = np.meshgrid(np.arange(cout), np.arange(cin), np.arange(Ho), np.arange(Wo),
                                 indexing="ij")
    rows_all, cols_all, vals_all = [], [], []
    for ky in range(k):
        for kx in range(k):
            iy = oy * s - p + ky
            ix = ox * s - p + kx
            ok = (iy >= 0) & (iy < H) & (ix >= 0) & (ix < Wd)
            rows_all.append((co * Ho * Wo + oy * Wo + ox)[ok])
            cols_all.append((ci * H * Wd + iy * Wd + ix)[ok])
            vals_all.append(ly.W[co[ok], ci[ok], ky, kx].astype(np.float64))
    rows = np.concatenate(rows_all)
    cols = np.concatenate(cols_all)
    vals = np.concatenate(vals_all)
    return sp.csr_matrix((vals, (rows, cols)), shape=(cout * Ho * Wo, cin * H * Wd))


def _mm(A, W):
    """A [R, d_i] times W [d_i, d_{i-1}] (W dense or sparse) -> dense [R, d_{i-1}]."""
    if sp.issparse(W):
        return np.asarray((W.T @ A.T).T)
    return A @ W


def _mv(W, h):
    """W [d_i, d_{i-1}] times rows of h [R, d_{i-1}] -> [R, d_i]."""
    if sp.issparse(W):
        return np.asarray((W @ h.T).T)
    return h @ W.T


class OracleNet:
    """W[i], b[i] for paper layers i = 1..L (index 0 unused); the spec merged into layer L.

    The specification matrix C is folded into the last layer (Section 2.1):
    Wbar = C W^(L), bbar = C b^(L), one row per spec.
    """

    def __init__(self, layers, C):
        self.L = len(layers)
        self.W = [None]
        self.b = [None]
        for ly in layers:
            if ly.kind == "fc":
                self.W.append(ly.W.astype(np.float64))
                self.b.append(ly.b.astype(np.float64))
            else:
                self.W.append(conv_matrix(ly))
                hw = ly.out_shape[1] * ly.out_shape[2]
                self.b.append(np.repeat(ly.b.astype(np.float64), hw))
        C64 = np.asarray(C, np.float64)
        WL = self.W[self.L]
        WL = WL.toarray() if sp.issparse(WL) else WL
        self.Wbar = C64 @ WL
        self.bbar = C64 @ self.b[self.L]
        self.K = C64.shape[0]
        self.d = [self.W[1].shape[1]] + [self.W[i].shape[0] for i in range(1, self.L + 1)]
        self.hidden = self.d[1:self.L]
        self.hoff = np.concatenate([[0], np.cumsum(self.hidden)]).astype(np.int64)

    def forward(self, x):
        """f_k(x) = (C z^(L)(x))_k for rows of x (Eq. 1 with the spec merged)."""
        h = np.atleast_2d(np.asarray(x, np.float64))
        for i in range(1, self.L):
            h = np.maximum(_mv(self.W[i], h) + self.b[i], 0.0)
        return h @ self.Wbar.T + self.bbar

    def preacts(self, x):
        """Pre-activations z^(i)(x) for i = 1..L-1 (list, index 0 unused)."""
        h = np.atleast_2d(np.asarray(x, np.float64))
        zs = [None]
        for i in range(1, self.L):
            z = _mv(self.W[i], h) + self.b[i]
            zs.append(z)
            h = np.maximum(z, 0.0)
        return zs


# --------------------------------------------------------------------------------------
# Per-row expansion of a batch (Eq. 3 split encoding, alpha/beta layout)
# --------------------------------------------------------------------------------------

def unstable_mask(l, u):
    """l < 0 < u (reading: l >= 0 is active, u <= 0 inactive)."""
    return (l < 0) & (u > 0)


def unstable_ranks(net, l, u):
    """Per property: rank of each hidden neuron among the unstable ones (layer-major), -1 if stable.

    l, u: [P, H] float arrays.  Returns (rank [P, H] int64, U [P])."""
    m = unstable_mask(np.asarray(l), np.asarray(u))
    rank = np.where(m, np.cumsum(m, axis=1) - 1, -1).astype(np.int64)
    return rank, m.sum(axis=1).astype(np.int64)


@dataclass
class Rows:
    """Dense per-row view of a batch: for each hidden layer i, per (row, neuron)."""
    R: int
    prop: np.ndarray        # [R]
    spec: np.ndarray        # [R]
    sign: list              # [i] -> [R, d_i] int8, S^(i)_jj (Eq. 3)
    beta_idx: list          # [i] -> [R, d_i] int64 (-1 where not split)
    alpha_idx: list         # [i] -> [R, d_i] int64 (-1 where not unstable)


def expand_rows(net, batch, l, u):
    K = net.K
    B = batch.B
    R = B * K
    prop = np.repeat(np.asarray(batch.prop_of, np.int64), K)
    spec = np.tile(np.arange(K), B)
    rank, U = unstable_ranks(net, l, u)
    sign, bidx, aidx = [None], [None], [None]
    for i in range(1, net.L):
        sign.append(np.zeros((R, net.d[i]), np.int8))
        bidx.append(np.full((R, net.d[i]), -1, np.int64))
        lo, hi = net.hoff[i - 1], net.hoff[i]
        rk = rank[prop][:, lo:hi]
        base = (np.repeat(np.asarray(batch.alpha_off, np.int64), K)
                + spec * U[prop])[:, None]
        aidx.append(np.where(rk >= 0, base + rk, -1))
    for b in range(B):
        off, cnt = int(batch.split_off[b]), int(batch.split_cnt[b])
        for t in range(cnt):
            i = int(batch.split_layer[off + t])
            j = int(batch.split_idx[off + t])
            s = int(batch.split_sign[off + t])
            for k in range(K):
                r = b * K + k
                sign[i][r, j] = s
                bidx[i][r, j] = off * K + k * cnt + t
    return Rows(R, prop, spec, sign, bidx, aidx)


def _gather(vec, idx):
    """vec[idx] with 0 where idx < 0."""
    out = np.zeros(idx.shape, np.float64)
    m = idx >= 0
    out[m] = np.asarray(vec, np.float64)[idx[m]]
    return out


def neuron_codes(net, rows, l, u):
    """Per-row neuron code from l, u and the split list: split overrides stability."""
    codes = [None]
    for i in range(1, net.L):
        lo, hi = net.hoff[i - 1], net.hoff[i]
        li, ui = np.asarray(l)[rows.prop][:, lo:hi], np.asarray(u)[rows.prop][:, lo:hi]
        c = np.full(li.shape, CODE_UNSTABLE, np.int8)
        c[ui <= 0] = CODE_INACTIVE
        c[li >= 0] = CODE_ACTIVE
        c[rows.sign[i] == -1] = CODE_SPLIT_POS
        c[rows.sign[i] == 1] = CODE_SPLIT_NEG
        codes.append(c)
    return codes


# --------------------------------------------------------------------------------------
# Relaxation (Lemma 2.1 full form, Eq. relax_single_d/_b; Theorem 3.1 Eq. definition_D,
# definition_lowerb) and the backward recursion (Eq. definition_A)
# --------------------------------------------------------------------------------------

def relax(A, li, ui, alpha, sign):
    """Diagonal D and intercepts lambda of one ReLU layer for every row.

    D = 1 for l >= 0 or a "z >= 0" split; 0 for u <= 0 or a "z < 0" split;
    for unstable unsplit neurons D = alpha when A_j >= 0, else the upper chord
    slope u/(u-l) with intercept -u*l/(u-l).  The lower bound of A^T ReLU(z) is
    A^T (D z + lambda)  (Lemma 2.1, b' = A^T lambda).
    """
    D = np.zeros_like(A)
    lam = np.zeros_like(A)
    active = li >= 0
    inactive = (~active) & (ui <= 0)
    unst = (~active) & (~inactive) & (sign == 0)
    D[active] = 1.0
    D[inactive] = 0.0
    pos = unst & (A >= 0)
    neg = unst & (A < 0)
    D[pos] = alpha[pos]
    slope = np.where(unst, ui / np.where(unst, ui - li, 1.0), 0.0)
    D[neg] = slope[neg]
    lam[neg] = (-ui * li / np.where(unst, ui - li, 1.0))[neg]
    D[sign == -1] = 1.0
    D[sign == 1] = 0.0
    lam[sign != 0] = 0.0
    return D, lam


@dataclass
class Trace:
    A: list        # A^(i) for i = 0..L-1 (rows), before relaxation
    D: list
    lam: list
    Lam: list      # A^(i) D^(i) + beta^(i) S^(i)
    c: np.ndarray  # constant after all layers


def _layer_inputs(net, rows, props, i, alpha, beta):
    lo, hi = net.hoff[i - 1], net.hoff[i]
    li = np.asarray(props["l"], np.float64)[rows.prop][:, lo:hi]
    ui = np.asarray(props["u"], np.float64)[rows.prop][:, lo:hi]
    al = _gather(alpha, rows.alpha_idx[i])
    be = _gather(beta, rows.beta_idx[i])
    return li, ui, al, be


def bound(net, props, batch, alpha, beta, rows=None, trace=False):
    """Lower bound of c_k^T f(x) on every row (Theorem 3.1, recursive form).

    A^(L-1) = Wbar_k, c = bbar_k; for i = L-1 .. 1:
        Lambda^(i) = A^(i) D^(i) + beta^(i)^T S^(i)
        c         += Lambda^(i) b^(i) + A^(i) lambda^(i)
        A^(i-1)    = Lambda^(i) W^(i)
    lb = c + sum_m min(A^(0)_m x_lo_m, A^(0)_m x_hi_m)   (Eq. beta_crown_lp, Hoelder for a box)

    props: dict with x_lo, x_hi [P, d0] and l, u [P, H] (float arrays).
    """
    rows = rows or expand_rows(net, batch, props["l"], props["u"])
    A = net.Wbar[rows.spec].copy()
    c = net.bbar[rows.spec].copy()
    As, Ds, lams, Lams = [None] * net.L, [None] * net.L, [None] * net.L, [None] * net.L
    for i in range(net.L - 1, 0, -1):
        li, ui, al, be = _layer_inputs(net, rows, props, i, alpha, beta)
        D, lam = relax(A, li, ui, al, rows.sign[i])
        Lam = A * D + be * rows.sign[i]
        c = c + (Lam * net.b[i][None, :]).sum(axis=1) + (A * lam).sum(axis=1)
        As[i], Ds[i], lams[i], Lams[i] = A, D, lam, Lam
        A = _mm(Lam, net.W[i])
    As[0] = A
    xlo = np.asarray(props["x_lo"], np.float64)[rows.prop]
    xhi = np.asarray(props["x_hi"], np.float64)[rows.prop]
    lb = c + np.minimum(A * xlo, A * xhi).sum(axis=1)
    if trace:
        return lb, Trace(As, Ds, lams, Lams, c)
    return lb


def bound_explicit(net, props, batch, alpha, beta):
    """Theorem 3.1 with each term written out (Appendix A, Definition A.1 and Eq. beta_crown_linear_app).

    Omega(i,i) = I, Omega(k+1,i) = W^(k+1) D^(k) Omega(k,i);
      a   = [Omega(L,1) W^(1)]^T
      P_i = S^(i) Omega(i,1) W^(1)
      q_i = sum_{k=1..i} S^(i) Omega(i,k) b^(k) + sum_{k=2..i} S^(i) Omega(i,k) W^(k) lambda^(k-1)
      c   = sum_{i=1..L} Omega(L,i) b^(i) + sum_{i=2..L} Omega(L,i) W^(i) lambda^(i-1)
    bound = min_x (a + P beta)^T x + q^T beta + c.  D and lambda are those the
    recursion selects (they depend on A, Eq. definition_D).  Dense, one row at a
    time: for tiny networks only.
    """
    rows = expand_rows(net, batch, props["l"], props["u"])
    _, tr = bound(net, props, batch, alpha, beta, rows=rows, trace=True)
    L = net.L
    dense = [None] + [(net.W[i].toarray() if sp.issparse(net.W[i]) else net.W[i]) for i in range(1, L)]
    out = np.zeros(rows.R)
    xlo_all = np.asarray(props["x_lo"], np.float64)
    xhi_all = np.asarray(props["x_hi"], np.float64)
    for r in range(rows.R):
        Wl = [None] + dense[1:] + [net.Wbar[rows.spec[r]][None, :]]
        bl = [None] + [net.b[i] for i in range(1, L)] + [np.array([net.bbar[rows.spec[r]]])]
        Dm = [None] + [np.diag(tr.D[i][r]) for i in range(1, L)]
        lam = [None] + [tr.lam[i][r] for i in range(1, L)]
        S = [None] + [np.diag(rows.sign[i][r].astype(np.float64)) for i in range(1, L)]
        be = [None] + [_gather(beta, rows.beta_idx[i][r]) for i in range(1, L)]

        def omega(k, i):
            # Omega(i,i) = I (size d_i); Omega(k,i) = W^(k) D^(k-1) ... W^(i+1) D^(i)
            M = np.eye(net.d[i]) if i < L else np.eye(1)
            for m in range(i, k):
                M = Wl[m + 1] @ Dm[m] @ M
            return M

        a = (omega(L, 1) @ Wl[1]).ravel()
        Pb = np.zeros(net.d[0])
        qb = 0.0
        for i in range(1, L):
            Pi = S[i] @ omega(i, 1) @ Wl[1]
            Pb += Pi.T @ be[i]
            qi = sum(S[i] @ omega(i, k) @ bl[k] for k in range(1, i + 1))
            qi = qi + sum((S[i] @ omega(i, k) @ Wl[k] @ lam[k - 1] for k in range(2, i + 1)),
                          np.zeros(net.d[i]))
            qb += qi @ be[i]
        c = sum((omega(L, i) @ bl[i]).item() for i in range(1, L + 1))
        c += sum((omega(L, i) @ Wl[i] @ lam[i - 1]).item() for i in range(2, L + 1))
        coef = a + Pb
        xlo, xhi = xlo_all[rows.prop[r]], xhi_all[rows.prop[r]]
        out[r] = np.minimum(coef * xlo, coef * xhi).sum() + qb + c
    return out


def bound_dual(net, props, batch, alpha, beta):
    """Dual objective g(alpha, beta) of Theorem 3.2 (Eq. final_beta_dual, nu_eq), box form.

    nu^(L) = -1 (spec row), nu_hat^(i-1) = W^(i)^T nu^(i);  for hidden layers:
      u <= 0 (unsplit): nu = 0;   l >= 0 (unsplit): nu = nu_hat;
      unstable unsplit: [nu]^+ = u/(u-l) [nu_hat]^+,  [nu]^- = alpha [nu_hat]^-;
      j in Z^- : nu = -beta;      j in Z^+ : nu = beta + nu_hat.
    g = -sum_i nu^(i)T b^(i) - nu_hat^(0)T x0 - sum_m |nu_hat^(0)_m| eps_m
        + sum_{unstable unsplit} l_j [nu_j]^+,
    with x0 the box centre and eps_m its half-width per coordinate.
    """
    rows = expand_rows(net, batch, props["l"], props["u"])
    R = rows.R
    g = -(-1.0) * net.bbar[rows.spec]          # -nu^(L) b^(L)
    nu_hat = -net.Wbar[rows.spec]              # W^(L)^T nu^(L), nu^(L) = -1
    for i in range(net.L - 1, 0, -1):
        li, ui, al, be = _layer_inputs(net, rows, props, i, alpha, beta)
        sg = rows.sign[i]
        nu = np.zeros_like(nu_hat)
        act = (li >= 0) & (sg == 0)
        nu[act] = nu_hat[act]
        unst = (li < 0) & (ui > 0) & (sg == 0)
        pos_part = np.maximum(nu_hat, 0.0)
        neg_part = np.maximum(-nu_hat, 0.0)
        den = np.where(unst, ui - li, 1.0)
        nu_u = (ui / den) * pos_part - al * neg_part
        nu[unst] = nu_u[unst]
        nu[sg == 1] = -be[sg == 1]
        nu[sg == -1] = be[sg == -1] + nu_hat[sg == -1]
        g = g - (nu * net.b[i][None, :]).sum(axis=1)
        g = g + np.where(unst, li * np.maximum(nu, 0.0), 0.0).sum(axis=1)
        nu_hat = _mm(nu, net.W[i])
    xlo = np.asarray(props["x_lo"], np.float64)[rows.prop]
    xhi = np.asarray(props["x_hi"], np.float64)[rows.prop]
    x0 = 0.5 * (xlo + xhi)
    eps = 0.5 * (xhi - xlo)
    g = g - (nu_hat * x0).sum(axis=1) - (np.abs(nu_hat) * eps).sum(axis=1)
    return g


# --------------------------------------------------------------------------------------
# Gradient of the bound w.r.t. alpha and beta (adjoint of the recursion)
# --------------------------------------------------------------------------------------

def grad(net, props, batch, alpha, beta, rows=None):
    """(lb, dlb/dalpha, dlb/dbeta) per row, in the alpha/beta layouts.

    With D, lambda and the signs of A fixed by the bound pass, lb equals
    bbar_k + Wbar_k h^(L-1) + sum_i sum_j beta_j S_jj zhat^(i)_j along the
    primal path h^(0) = x* (x_lo where A^(0)_m >= 0, else x_hi),
    zhat^(i) = W^(i) h^(i-1) + b^(i), h^(i) = D^(i) zhat^(i) + lambda^(i).
    Hence dlb/dalpha_j = A^(i)_j zhat^(i)_j where alpha_j is the slope in use
    (unstable, unsplit, A_j >= 0; zero otherwise) and dlb/dbeta_j = S_jj zhat^(i)_j.
    The paper obtains the same gradient by automatic differentiation (Section 3.1).
    """
    rows = rows or expand_rows(net, batch, props["l"], props["u"])
    lb, tr = bound(net, props, batch, alpha, beta, rows=rows, trace=True)
    xlo = np.asarray(props["x_lo"], np.float64)[rows.prop]
    xhi = np.asarray(props["x_hi"], np.float64)[rows.prop]
    h = np.where(tr.A[0] >= 0, xlo, xhi)
    da = np.zeros(len(alpha), np.float64)
    db = np.zeros(len(beta), np.float64)
    for i in range(1, net.L):
        zhat = _mv(net.W[i], h) + net.b[i]
        li, ui, _, _ = _layer_inputs(net, rows, props, i, alpha, beta)
        A = tr.A[i]
        sg = rows.sign[i]
        use_alpha = (li < 0) & (ui > 0) & (sg == 0) & (A >= 0)
        m = use_alpha & (rows.alpha_idx[i] >= 0)
        np.add.at(da, rows.alpha_idx[i][m], (A * zhat)[m])
        ms = sg != 0
        np.add.at(db, rows.beta_idx[i][ms], (sg * zhat)[ms])
        h = tr.D[i] * zhat + tr.lam[i]
    return lb, da, db


# --------------------------------------------------------------------------------------
# Root intermediate bounds (Section 3.3 with fixed alpha'; Lemma 2.2 CROWN)
# --------------------------------------------------------------------------------------

ALPHA_ADAPTIVE, ALPHA_FIXED = 0, 1


def _root_alpha(li, ui, rule, value):
    if rule == ALPHA_ADAPTIVE:
        return np.where(ui >= -li, 1.0, 0.0)
    return np.full_like(li, value)


def root_bounds(net, x_lo, x_hi, rule=ALPHA_ADAPTIVE, value=0.5):
    """l, u [P, H] for all hidden neurons by CROWN with no splits and beta = 0.

    Layer 1: interval of W^(1) x + b^(1) over the box (exact for a linear map).
    Layer i >= 2: the lower bound of z^(i)_j (objective f := z^(i)_j) and of
    -z^(i)_j, back-substituted through layers i-1..1 using the bounds already
    found, with the lower-slope alpha' given by the rule (adaptive: 1 if
    u >= -l else 0; fixed: value).
    """
    x_lo = np.atleast_2d(np.asarray(x_lo, np.float64))
    x_hi = np.atleast_2d(np.asarray(x_hi, np.float64))
    P = x_lo.shape[0]
    H = int(sum(net.hidden))
    l = np.zeros((P, H))
    u = np.zeros((P, H))
    for p in range(P):
        mid = 0.5 * (x_lo[p] + x_hi[p])
        rad = 0.5 * (x_hi[p] - x_lo[p])
        W1 = net.W[1]
        c1 = _mv(W1, mid[None, :])[0] + net.b[1]
        absW = abs(W1)
        r1 = _mv(absW, rad[None, :])[0]
        l[p, :net.hoff[1]] = c1 - r1
        u[p, :net.hoff[1]] = c1 + r1
        for i in range(2, net.L):
            Wi = net.W[i].toarray() if sp.issparse(net.W[i]) else net.W[i]
            di = net.d[i]
            A = np.concatenate([Wi, -Wi], axis=0)
            c = np.concatenate([net.b[i], -net.b[i]])
            for m in range(i - 1, 0, -1):
                lo, hi = net.hoff[m - 1], net.hoff[m]
                li = np.broadcast_to(l[p, lo:hi], A.shape)
                ui = np.broadcast_to(u[p, lo:hi], A.shape)
                al = _root_alpha(li, ui, rule, value)
                D, lam = relax(A, li, ui, al, np.zeros(A.shape, np.int8))
                Lam = A * D
                c = c + (Lam * net.b[m][None, :]).sum(axis=1) + (A * lam).sum(axis=1)
                A = _mm(Lam, net.W[m])
            lb = c + np.minimum(A * x_lo[p], A * x_hi[p]).sum(axis=1)
            l[p, net.hoff[i - 1]:net.hoff[i]] = lb[:di]
            u[p, net.hoff[i - 1]:net.hoff[i]] = -lb[di:]
    return l, u


def interval_bounds(net, x_lo, x_hi):
    """l, u [P, H] by interval propagation: z^(i) in W^(i) [h_lo, h_hi] + b^(i) with
    h = ReLU(z), layer by layer from the box (centre/radius form, |W| for the radius).

    Valid (sound, looser than CROWN) intermediate bounds for any network size; the bound of
    Theorem 3.1 only needs some l <= z <= u (Section 2.1), so they serve where CROWN root
    bounds over very wide layers are out of reach for this oracle.
    """
    x_lo = np.atleast_2d(np.asarray(x_lo, np.float64))
    x_hi = np.atleast_2d(np.asarray(x_hi, np.float64))
    P = x_lo.shape[0]
    H = int(sum(net.hidden))
    l = np.zeros((P, H))
    u = np.zeros((P, H))
    for p in range(P):
        lo, hi = x_lo[p], x_hi[p]
        for i in range(1, net.L):
            mid, rad = 0.5 * (lo + hi), 0.5 * (hi - lo)
            c = _mv(net.W[i], mid[None, :])[0] + net.b[i]
            r = _mv(abs(net.W[i]), rad[None, :])[0]
            l[p, net.hoff[i - 1]:net.hoff[i]] = c - r
            u[p, net.hoff[i - 1]:net.hoff[i]] = c + r
            lo, hi = np.maximum(c - r, 0.0), np.maximum(c + r, 0.0)
    return l, u


# --------------------------------------------------------------------------------------
# Projected Adam ascent on alpha in [0,1], beta >= 0 (Eq. opt_alpha_beta; Appendix C.1)
# --------------------------------------------------------------------------------------

@dataclass
class AdamCfg:
    iters: int = 20
    lr_alpha: float = 0.1
    lr_beta: float = 0.05
    decay: float = 0.98
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


def row_of_params(net, batch, U):
    """Row index owning each alpha and each beta entry."""
    K = net.K
    ra = np.zeros(batch.n_alpha, np.int64)
    rb = np.zeros(batch.n_beta, np.int64)
    for b in range(batch.B):
        Up = int(U[batch.prop_of[b]])
        cnt = int(batch.split_cnt[b])
        for k in range(K):
            s = int(batch.alpha_off[b]) + k * Up
            ra[s:s + Up] = b * K + k
            s = int(batch.split_off[b]) * K + k * cnt
            rb[s:s + cnt] = b * K + k
    return ra, rb


def adam_ascent_step(theta, m, v, g, t, lr, cfg, lo, hi):
    """One Adam step (Kingma & Ba) taken uphill, then projection onto [lo, hi]; t counts from 0."""
    m = cfg.beta1 * m + (1.0 - cfg.beta1) * g
    v = cfg.beta2 * v + (1.0 - cfg.beta2) * g * g
    mhat = m / (1.0 - cfg.beta1 ** (t + 1))
    vhat = v / (1.0 - cfg.beta2 ** (t + 1))
    theta = theta + lr * mhat / (np.sqrt(vhat) + cfg.eps)
    return np.clip(theta, lo, hi), m, v


def optimize(net, props, batch, alpha0, beta0, cfg=AdamCfg()):
    """Projected Adam on the sum of row bounds; returns (lb at best theta, alpha_best, beta_best, history).

    Iteration t (0..iters-1) evaluates lb and its gradient at theta_t, keeps
    per row the best lb seen and its theta, then steps with learning rates
    lr0 * decay^t.  Any alpha in [0,1] and beta >= 0 gives a valid bound, so
    the best one is returned (and re-evaluated as the final bound).
    """
    rows = expand_rows(net, batch, props["l"], props["u"])
    _, U = unstable_ranks(net, props["l"], props["u"])
    ra, rb = row_of_params(net, batch, U)
    a = np.asarray(alpha0, np.float64).copy()
    b = np.asarray(beta0, np.float64).copy()
    ma, va = np.zeros_like(a), np.zeros_like(a)
    mb, vb = np.zeros_like(b), np.zeros_like(b)
    best = np.full(rows.R, -np.inf)
    a_best, b_best = a.copy(), b.copy()
    hist = []
    for t in range(cfg.iters):
        lb, da, db = grad(net, props, batch, a, b, rows=rows)
        hist.append(lb.copy())
        improved = lb > best
        best = np.where(improved, lb, best)
        a_best = np.where(improved[ra], a, a_best)
        b_best = np.where(improved[rb], b, b_best)
        fac = cfg.decay ** t
        a, ma, va = adam_ascent_step(a, ma, va, da, t, cfg.lr_alpha * fac, cfg, 0.0, 1.0)
        b, mb, vb = adam_ascent_step(b, mb, vb, db, t, cfg.lr_beta * fac, cfg, 0.0, np.inf)
    lb_final = bound(net, props, batch, a_best, b_best, rows=rows)
    return lb_final, a_best, b_best, hist


# --------------------------------------------------------------------------------------
# batch_split (Algorithm 1): children of picked subdomains
# --------------------------------------------------------------------------------------

def batch_split(batch, K, U, pick_layer, pick_idx, alpha, beta):
    """Each parent b splits neuron (pick_layer[b], pick_idx[b]) into two children.

    Child 2b is C^l (split z >= 0, S = -1), child 2b+1 is C^u (z < 0, S = +1).
    Both inherit the parent's split list (the new split appended last), the
    parent's alpha block, and the parent's beta with 0 for the new split.
    Returns (prop_of, split_off, split_cnt, split_layer, split_idx, split_sign,
    alpha_off, alpha, beta) of the 2B children, in the C-ABI layouts.
    """
    B = batch.B
    prop, cnt, off = [], [], []
    lay, idx, sgn = [], [], []
    a_off, a_out, b_out = [], [], []
    pos_a = 0
    pos_s = 0
    for b in range(B):
        o, c = int(batch.split_off[b]), int(batch.split_cnt[b])
        a0 = int(batch.alpha_off[b])
        a1 = a0 + int(U[batch.prop_of[b]]) * K
        for s in (-1, 1):
            prop.append(int(batch.prop_of[b]))
            off.append(pos_s)
            cnt.append(c + 1)
            lay.extend(list(batch.split_layer[o:o + c]) + [int(pick_layer[b])])
            idx.extend(list(batch.split_idx[o:o + c]) + [int(pick_idx[b])])
            sgn.extend(list(batch.split_sign[o:o + c]) + [s])
            a_off.append(pos_a)
            a_out.append(np.asarray(alpha[a0:a1]))
            for k in range(K):
                blk = np.asarray(beta[o * K + k * c:o * K + (k + 1) * c])
                b_out.append(np.concatenate([blk, [0.0]]))
            pos_a += a1 - a0
            pos_s += c + 1
    return (np.array(prop, np.int32), np.array(off, np.int32), np.array(cnt, np.int32),
            np.array(lay, np.uint8), np.array(idx, np.uint32), np.array(sgn, np.int8),
            np.array(a_off, np.int64),
            np.concatenate(a_out) if a_out else np.zeros(0),
            np.concatenate(b_out) if b_out else np.zeros(0))

"""Independent pins for the oracle's bounds on tiny networks (test infrastructure only).

* ``lp_value``      -- the LP with neuron split constraints, Eq. lp_verify_split
                       (Section 3.2), solved by scipy's HiGHS.  By Corollary 3.1
                       every alpha in [0,1], beta >= 0 gives g <= p*_LP, and the
                       optimum of g equals p*_LP.
* ``exact_min``     -- min of c_k^T f(x) over the box and the split constraints,
                       by enumerating the activation patterns of the unstable
                       unsplit neurons and solving one LP per pattern (the network
                       is linear on each pattern's region; Appendix B, proof of
                       Theorem 3.3).
* ``sampled_min``   -- min of c_k^T f over uniform samples and box vertices that
                       satisfy the split constraints (soundness check).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


def _dense(W):
    return W.toarray() if sp.issparse(W) else np.asarray(W)


def _split_maps(net, splits):
    """splits: list of (layer i, index j, sign S) -> per-layer dict j -> S."""
    per = [dict() for _ in range(net.L)]
    for i, j, s in splits:
        per[int(i)][int(j)] = int(s)
    return per


def lp_value(net, x_lo, x_hi, l, u, splits, k):
    """p*_LP of Eq. lp_verify_split for spec row k (inf if the LP is infeasible).

    Variables: x (= h^(0)), then for each hidden layer z^(i) and h^(i).
    Constraints: z^(i) = W^(i) h^(i-1) + b^(i); x in the box; stable neurons
    h = z (l >= 0) or h = 0 (u <= 0); unstable unsplit neurons h >= 0, h >= z,
    h <= u/(u-l) (z - l); a "z >= 0" split h = z, z >= 0; a "z < 0" split h = 0,
    z <= 0 (closure of the strict inequality).  Objective Wbar_k h^(L-1) + bbar_k.
    """
    L = net.L
    d = net.d
    per = _split_maps(net, splits)
    # variable offsets
    offs = {}
    n = d[0]
    offs[("h", 0)] = 0
    for i in range(1, L):
        offs[("z", i)] = n
        n += d[i]
        offs[("h", i)] = n
        n += d[i]
    Aeq, beq, Aub, bub = [], [], [], []

    def row():
        return np.zeros(n)

    for i in range(1, L):
        Wi = _dense(net.W[i])
        for j in range(d[i]):
            r = row()
            r[offs[("z", i)] + j] = 1.0
            r[offs[("h", i - 1)]:offs[("h", i - 1)] + d[i - 1]] = -Wi[j]
            Aeq.append(r)
            beq.append(net.b[i][j])
        lo, hi = net.hoff[i - 1], net.hoff[i]
        li, ui = l[lo:hi], u[lo:hi]
        for j in range(d[i]):
            zj, hj = offs[("z", i)] + j, offs[("h", i)] + j
            s = per[i].get(j, 0)
            if s == -1:
                r = row(); r[hj] = 1; r[zj] = -1; Aeq.append(r); beq.append(0.0)
                r = row(); r[zj] = -1; Aub.append(r); bub.append(0.0)
            elif s == 1:
                r = row(); r[hj] = 1; Aeq.append(r); beq.append(0.0)
                r = row(); r[zj] = 1; Aub.append(r); bub.append(0.0)
            elif li[j] >= 0:
                r = row(); r[hj] = 1; r[zj] = -1; Aeq.append(r); beq.append(0.0)
            elif ui[j] <= 0:
                r = row(); r[hj] = 1; Aeq.append(r); beq.append(0.0)
            else:
                r = row(); r[hj] = -1; Aub.append(r); bub.append(0.0)
                r = row(); r[zj] = 1; r[hj] = -1; Aub.append(r); bub.append(0.0)
                sl = ui[j] / (ui[j] - li[j])
                # h <= sl*z - sl*l
                r = row(); r[hj] = 1; r[zj] = -sl; Aub.append(r); bub.append(-sl * li[j])
    cobj = row()
    cobj[offs[("h", L - 1)]:offs[("h", L - 1)] + d[L - 1]] = net.Wbar[k]
    bounds = [(float(x_lo[m]), float(x_hi[m])) for m in range(d[0])] + [(None, None)] * (n - d[0])
    res = linprog(cobj, A_ub=np.array(Aub) if Aub else None, b_ub=np.array(bub) if bub else None,
                  A_eq=np.array(Aeq), b_eq=np.array(beq), bounds=bounds, method="highs")
    if res.status == 2:
        return np.inf
    assert res.status == 0, res.message
    return res.fun + net.bbar[k]


def exact_min(net, x_lo, x_hi, l, u, splits, k, max_unstable=14):
    """Exact min over {x in box, z in split set} by enumerating activation patterns."""
    L = net.L
    d = net.d
    per = _split_maps(net, splits)
    fixed = []   # per layer: array of pattern values (1 active, 0 inactive, -1 free)
    free = []
    for i in range(1, L):
        lo, hi = net.hoff[i - 1], net.hoff[i]
        li, ui = l[lo:hi], u[lo:hi]
        pat = np.full(d[i], -1, np.int64)
        for j in range(d[i]):
            s = per[i].get(j, 0)
            if s == -1:
                pat[j] = 1
            elif s == 1:
                pat[j] = 0
            elif li[j] >= 0:
                pat[j] = 1
            elif ui[j] <= 0:
                pat[j] = 0
            else:
                free.append((i, j))
        fixed.append(pat)
    assert len(free) <= max_unstable, len(free)
    best = np.inf
    Wd = [None] + [_dense(net.W[i]) for i in range(1, L)]
    for bits in itertools.product([0, 1], repeat=len(free)):
        pats = [p.copy() for p in fixed]
        for (i, j), v in zip(free, bits):
            pats[i - 1][j] = v
        # z^(i) = M_i x + v_i along this pattern; constraints on the sign of z
        M = np.eye(d[0])
        v = np.zeros(d[0])
        Aub, bub = [], []
        for i in range(1, L):
            Mz = Wd[i] @ M
            vz = Wd[i] @ v + net.b[i]
            pat = pats[i - 1]
            for j in range(d[i]):
                sj = per[i].get(j, 0)
                if pat[j] == 1:     # z >= 0  ->  -Mz x <= vz
                    Aub.append(-Mz[j]); bub.append(vz[j])
                else:               # z <= 0
                    Aub.append(Mz[j]); bub.append(-vz[j])
                _ = sj
            M = Mz * pat[:, None]
            v = vz * pat
        cvec = net.Wbar[k] @ M
        c0 = net.Wbar[k] @ v + net.bbar[k]
        res = linprog(cvec, A_ub=np.array(Aub), b_ub=np.array(bub),
                      bounds=[(float(x_lo[m]), float(x_hi[m])) for m in range(d[0])], method="highs")
        if res.status == 0:
            best = min(best, res.fun + c0)
    return best


def satisfies_splits(net, x, splits):
    zs = net.preacts(x)
    ok = np.ones(np.atleast_2d(x).shape[0], bool)
    for i, j, s in splits:
        z = zs[int(i)][:, int(j)]
        ok &= (z >= 0) if int(s) == -1 else (z <= 0)
    return ok


def sampled_min(net, x_lo, x_hi, splits, k, n, rng):
    d0 = len(x_lo)
    xs = rng.uniform(x_lo, x_hi, size=(n, d0))
    if d0 <= 12:
        verts = np.array(list(itertools.product([0, 1], repeat=d0)), np.float64)
        xs = np.concatenate([xs, x_lo + verts * (x_hi - x_lo)])
    ok = satisfies_splits(net, xs, splits)
    if not ok.any():
        return np.inf, 0
    f = net.forward(xs[ok])[:, k]
    return f.min(), int(ok.sum())

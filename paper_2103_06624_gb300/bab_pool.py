"""Branch and bound (Algorithm 1) with the subdomain pool held in arrays, alpha and beta on the device.

The same algorithm as bab.bab_many -- lowest-bound-first batches, each parent split on the next
neuron of the static branching order into its two children (alpha inherited, the new split's beta
at 0), the optimised beta-CROWN bound of the children in one engine call, Domain_Filter, the upper
bound f(x*) at the minimiser of every bounded subdomain's linear bound (Appendix B.1), and the
beta-only ascent on fully split subdomains (Theorem 3.3) -- but no subdomain is a Python object
and no alpha or beta leaves the device while branching:

  host    per open subdomain: its depth, its property (owner), the signs of its splits [D] and
          the lowest of its K bounds.  Every subdomain grown from the root has split exactly
          the first `depth` neurons of its property's branching order, so its split list is
          implicit.  The batches in the C-ABI layout are built from these arrays with vectorised
          index arithmetic (no per-subdomain loop).
  device  per open subdomain: alpha [K * Umax] (the property's K * U_p values, then padding) and
          beta [K, D] (split t of spec k at [k, t]; unused slots 0).  Children are row gathers of
          their parents' rows; the engine's compact beta (split_off * K + k * cnt + t) is a masked
          view of the padded rows.

Per round the host does O(batch) array work plus a handful of device calls
(`python bench.py --workload mlp784 --bab` measures its cost per child against the engine's).  Subdomains whose
every root-unstable neuron is split leave the arrays for the host-side line search of bab.py.
The order in which subdomains are taken, split and filtered is the one bab.bab_many follows, so on
a deterministic engine both drivers produce the same rounds, counts and verdicts (tested).

The engine here takes batches with device tensors: engine.optimize_rows(batch, alpha, beta) -> lb
[B*K] (alpha [B, K*Umax] and compact beta updated in place), engine.xstar_rows(batch, alpha, beta)
-> (x* [B*K, d0], C f(x*) [B*K, K]) and engine.margins(x) -> C f(x) in FP64 on the host; for the
exhausted subdomains it also needs bab.py's list interface (optimize, xstar).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import bab
from . import workloads as wl


def pool_batch(hidden_widths, K, Umax, orders, props, depth, owner, signs):
    """C-ABI batch of subdomains given by (depth, owner, signs): subdomain b has split neurons
    orders[owner[b]][:depth[b]] with signs[b, :depth[b]]; its alpha block starts at b * K * Umax."""
    B = int(depth.shape[0])
    cnt = depth.astype(np.int32)
    off = np.zeros(B, np.int32)
    if B > 1:
        off[1:] = np.cumsum(cnt)[:-1]
    S = int(cnt.sum())
    rowid = np.repeat(np.arange(B), cnt)
    t = np.arange(S) - off[rowid]
    gidx = orders[owner[rowid], t]
    sgn = signs[rowid, t]
    if S:
        layer, idx = wl.neuron_layer_index(hidden_widths, gidx)
    else:
        layer = idx = np.zeros(0, np.int64)
    return wl.Batch(np.asarray(props, np.int32)[owner], off, cnt, layer.astype(np.uint8), idx.astype(np.uint32),
                    sgn.astype(np.int8), np.arange(B, dtype=np.int64) * K * Umax, B * K * Umax, S * K)


def beta_mask(cnt_t, K, D):
    """[B, K, D] mask of the used beta slots: the masked flatten is the compact layout."""
    used = torch.arange(D, device=cnt_t.device)[None, :] < cnt_t[:, None]
    return used[:, None, :].expand(-1, K, -1)


MAX_SPLITS = 64   # the library's limit of splits per subdomain (BCROWN_MAX_SPLITS)


class _Pool:
    """Open subdomains: host arrays (depth, owner, signs, lowest bound, the K bounds) and device
    rows of alpha [n, K * Umax] and beta [n, K, D], in the order the driver keeps them."""

    def __init__(self, K, Umax, D, device):
        self.K, self.Umax, self.D, self.dev = K, Umax, D, device
        self.depth = np.zeros(0, np.int32)
        self.owner = np.zeros(0, np.int32)
        self.signs = np.zeros((0, D), np.int8)
        self.lb = np.zeros((0, K), np.float32)
        self.alpha = torch.zeros((0, K * Umax), dtype=torch.float32, device=device)
        self.beta = torch.zeros((0, K, D), dtype=torch.float32, device=device)

    @property
    def n(self):
        return int(self.depth.shape[0])

    def take(self, idx):
        """Rows idx (host int array), in that order, as a new pool."""
        p = _Pool(self.K, self.Umax, self.D, self.dev)
        it = torch.as_tensor(idx, dtype=torch.int64, device=self.dev)
        p.depth, p.owner, p.signs, p.lb = self.depth[idx], self.owner[idx], self.signs[idx], self.lb[idx]
        p.alpha, p.beta = self.alpha.index_select(0, it), self.beta.index_select(0, it)
        return p

    def append(self, o):
        self.depth = np.concatenate([self.depth, o.depth])
        self.owner = np.concatenate([self.owner, o.owner])
        self.signs = np.concatenate([self.signs, o.signs])
        self.lb = np.concatenate([self.lb, o.lb])
        self.alpha = torch.cat([self.alpha, o.alpha])
        self.beta = torch.cat([self.beta, o.beta])


def _children(par):
    """The two children of every row of pool `par` (split on the next neuron of the order):
    rows 2i (z >= 0, sign -1) and 2i + 1 (z <= 0, sign +1); alpha and beta rows copied, the new
    split's beta slot is the parent's unused (zero) slot."""
    c = _Pool(par.K, par.Umax, par.D, par.dev)
    c.depth = np.repeat(par.depth + 1, 2).astype(np.int32)
    c.owner = np.repeat(par.owner, 2)
    c.signs = np.repeat(par.signs, 2, axis=0)
    c.signs[np.arange(c.n), c.depth - 1] = np.tile(np.array([-1, 1], np.int8), par.n)
    c.lb = np.repeat(par.lb, 2, axis=0)
    c.alpha = par.alpha.repeat_interleave(2, dim=0)
    c.beta = par.beta.repeat_interleave(2, dim=0)
    return c


class _Ctx:
    """The properties being decided: their branching orders (padded to one matrix), unstable counts
    and library property indices."""

    def __init__(self, engine, cases, D):
        self.K = engine.K
        self.hw = engine.pb.hidden_widths
        orders, self.U = [], []
        for prop, l, u, x_lo, x_hi in cases:
            s = bab.branching_scores(l, u)
            U = int(np.isfinite(s).sum())
            self.U.append(U)
            orders.append(np.argsort(-s, kind="stable")[:U])   # root-unstable, widest first
        self.Umax = max(self.U + [1])
        self.D = D
        self.orders = np.zeros((len(cases), max(self.Umax, 1)), np.int64)
        for c, o in enumerate(orders):
            self.orders[c, :len(o)] = o
        self.props = np.array([c[0] for c in cases], np.int32)
        self.Uarr = np.array(self.U, np.int32)

    def batch(self, p):
        return pool_batch(self.hw, self.K, self.Umax, self.orders, self.props, p.depth, p.owner, p.signs)


def _bound_rows(engine, ctx, p):
    """One engine call on every row of pool p: its K bounds, alpha and beta rows updated."""
    hb = ctx.batch(p)
    cnt_t = torch.as_tensor(p.depth, dtype=torch.int64, device=p.dev)
    m = beta_mask(cnt_t, ctx.K, ctx.D)
    bc = p.beta[m].contiguous()
    a = p.alpha.contiguous()
    lb = engine.optimize_rows(hb, a, bc)
    p.alpha = a
    p.beta = torch.zeros_like(p.beta)
    p.beta[m] = bc
    p.lb = lb.reshape(p.n, ctx.K).cpu().numpy().astype(np.float32)
    return hb, a, bc


def _upper_rows(engine, ctx, p, hb, a, bc, res):
    """f(x*) for every row of pool p (bounded just before): the lowest margin at the points that
    minimise the rows' linear bounds.  A negative one (re-checked in FP64) decides its property."""
    if p.n == 0:
        return
    xs, m = engine.xstar_rows(hb, a, bc)
    K = ctx.K
    worst_row = m.amin(dim=1)                               # [n*K]
    w = worst_row.reshape(p.n, K)
    wmin, jmin = w.min(dim=1)
    wmin, jmin = wmin.cpu().numpy(), jmin.cpu().numpy()
    up = np.array([r.upper for r in res])
    for i in np.nonzero((wmin < up[p.owner]) | (wmin < 0))[0]:   # the others cannot lower any upper bound
        r = res[p.owner[i]]
        if wmin[i] < r.upper or wmin[i] < 0:
            x = xs[i * K + int(jmin[i])].double().cpu().numpy()
            m64 = engine.margins(x[None])[0]
            r.upper = min(r.upper, float(m64.min()))
            if m64.min() < 0 and r.status != "violated":
                r.status, r.witness, r.witness_margins = "violated", x, m64


def _domain(ctx, p, i):
    """Row i of pool p as a bab.Domain (host arrays; for the line search of fully split ones)."""
    c, d = int(p.owner[i]), int(p.depth[i])
    K, U = ctx.K, ctx.U[c]
    return bab.Domain(ctx.orders[c, :d].copy(), p.signs[i, :d].copy(),
                      p.alpha[i, :K * U].cpu().numpy().copy(), p.beta[i, :, :d].reshape(-1).cpu().numpy().copy(),
                      p.lb[i].copy(), c)


def bab_pool(engine, cases, batch_size=512, max_rounds=50, max_bounded=1_000_000, n_samples=256, seed=0,
             time_limit=None, alpha_init=0.5, pgd_steps=20, starts=None, upper=True, line_search=True, device=None):
    """Decide properties cases = [(prop, l, u, x_lo, x_hi), ...], as bab.bab_many does, with the
    pool in arrays and alpha, beta on `device` (default: CUDA when available).  starts, if given,
    holds each case's start subdomains as (neuron indices, signs) pairs whose neurons are the first
    ones of the case's branching order (as bab.rank_starts gives them); "verified" then covers their
    union.  Returns one bab.BabResult per case."""
    t0 = time.perf_counter()
    dev = torch.device(device if device is not None else ("cuda" if torch.cuda.is_available() else "cpu"))
    K = engine.K
    n = len(cases)
    res = [bab.BabResult("unknown") for _ in range(n)]
    ctx0 = _Ctx(engine, cases, 1)
    D = max(1, min(ctx0.Umax, MAX_SPLITS))
    ctx = _Ctx(engine, cases, D)
    open_case = np.ones(n, bool)
    for c, (prop, l, u, x_lo, x_hi) in enumerate(cases):
        x, m = bab._falsify(engine, np.asarray(x_lo, np.float64), np.asarray(x_hi, np.float64), n_samples,
                            np.random.default_rng(seed + c), pgd_steps)
        if m.min() < 0:
            res[c].status, res[c].witness, res[c].witness_margins = "violated", x, m
            open_case[c] = False

    def close_decided():
        for c in range(n):
            if open_case[c] and res[c].status == "violated":
                open_case[c] = False

    def count(p):
        np.add.at(bounded_per, p.owner, 1)
        for c in np.unique(p.owner):
            res[c].max_depth = max(res[c].max_depth, int(p.depth[p.owner == c].max()))

    bounded_per = np.zeros(n, np.int64)
    pool = _Pool(K, ctx.Umax, D, dev)
    first = []   # (owner, depth, signs) of the start subdomains
    for c in np.nonzero(open_case)[0]:
        for sp, sg in ([(np.zeros(0, np.int64), np.zeros(0, np.int8))] if starts is None else starts[c]):
            sp = np.asarray(sp, np.int64)
            d = len(sp)
            if d > min(D, ctx.U[c]) or not np.array_equal(sp, ctx.orders[c, :d]):
                raise ValueError("a start subdomain must split the first neurons of its property's branching order")
            first.append((c, d, np.asarray(sg, np.int8)))
    if len(first):
        f = _Pool(K, ctx.Umax, D, dev)
        f.depth = np.array([d for _, d, _ in first], np.int32)
        f.owner = np.array([c for c, _, _ in first], np.int32)
        f.signs = np.zeros((len(first), D), np.int8)
        for i, (_, d, sg) in enumerate(first):
            f.signs[i, :d] = sg
        f.lb = np.full((len(first), K), -np.inf, np.float32)
        f.alpha = torch.full((len(first), K * ctx.Umax), alpha_init, dtype=torch.float32, device=dev)
        f.beta = torch.zeros((len(first), K, D), dtype=torch.float32, device=dev)
        hb, a, bcmp = _bound_rows(engine, ctx, f)
        if upper:
            _upper_rows(engine, ctx, f, hb, a, bcmp, res)
        count(f)
        pool = f.take(np.nonzero(f.lb.min(axis=1) <= 0)[0])
    close_decided()
    pool = pool.take(np.nonzero(open_case[pool.owner])[0])
    exhausted = []
    rounds = bounded = 0
    while pool.n or any(open_case[d.owner] and not getattr(d, "searched", False) for d in exhausted):
        if rounds >= max_rounds or bounded >= max_bounded or (
                time_limit is not None and time.perf_counter() - t0 > time_limit):
            break
        rounds += 1
        order = np.argsort(pool.lb.min(axis=1), kind="stable")   # lowest bound first (stable, as list.sort)
        take, rest = order[:batch_size], order[batch_size:]
        for c in np.unique(pool.owner[take]):
            res[c].rounds += 1
        full = pool.depth[take] >= ctx.Uarr[pool.owner[take]]       # every root-unstable neuron split
        if np.any(pool.depth[take][~full] >= D):
            raise RuntimeError("a subdomain would exceed %d splits, the library's limit" % MAX_SPLITS)
        for i in take[full]:
            exhausted.append(_domain(ctx, pool, i))
        par = pool.take(take[~full])
        pool = pool.take(rest)
        if par.n:
            kids = _children(par)
            hb, a, bcmp = _bound_rows(engine, ctx, kids)
            if upper:
                _upper_rows(engine, ctx, kids, hb, a, bcmp, res)
            bounded += kids.n
            count(kids)
            pool.append(kids.take(np.nonzero(kids.lb.min(axis=1) <= 0)[0]))   # Domain_Filter
        close_decided()
        pool = pool.take(np.nonzero(open_case[pool.owner])[0])
        # fully split subdomains: beta alone, to the exact subdomain minimum (Theorem 3.3)
        fresh = [d for d in exhausted if open_case[d.owner] and not getattr(d, "searched", False)]
        if fresh and not line_search:
            for d in fresh:
                d.searched = True
        elif fresh:
            cert, conv = bab._line_search(engine, fresh, cases, K)
            bab._upper(engine, fresh, cases, res)
            keep = []
            for d, ok in zip(fresh, conv):
                d.searched = True
                res[d.owner].line_searched += 1
                if d.lb.min() > 0:
                    res[d.owner].infeasible += int(not ok)
                else:
                    keep.append(d)
            exhausted = [d for d in exhausted if not getattr(d, "searched", False)] + keep
            close_decided()
        exhausted = [d for d in exhausted if open_case[d.owner]]
        lbm = pool.lb.min(axis=1).astype(np.float64)
        for c in np.nonzero(open_case)[0]:
            mine = pool.owner == c
            left = [float(d.lb.min()) for d in exhausted if d.owner == c]
            vals = ([float(lbm[mine].min())] if mine.any() else []) + left
            res[c].history.append((int(mine.sum()) + len(left), min(vals, default=float("inf"))))
    for c in range(n):
        res[c].bounded = int(bounded_per[c])
        if not open_case[c] or res[c].status == "violated":
            continue
        mine = pool.owner == c
        left = [float(d.lb.min()) for d in exhausted if d.owner == c]
        res[c].open_domains = int(mine.sum()) + len(left)
        res[c].min_lb = min(left + ([float(pool.lb[mine].min())] if mine.any() else []), default=float("inf"))
        res[c].status = "verified" if res[c].open_domains == 0 else "unknown"
    dt = time.perf_counter() - t0
    for r in res:
        r.seconds = dt
    return res

"""Branch and bound around the batched bound (Algorithm 1): the driver that decides a property.

A property is verified when every margin spec k has c_k^T f(x) > 0 on the whole input box.
The driver keeps a pool of subdomains (split assignments of root-unstable neurons, Eq. 3), takes
the ones with the lowest certified bound in batches, splits each on one neuron into its two
children (z >= 0 and z <= 0; the parent's alpha is inherited and the new split's beta starts at
0, as batch_split does), bounds the children with the optimised beta-CROWN bound (Theorem 3.1,
Eq. opt_alpha_beta; one engine call per batch) and drops those whose bound is positive for every
spec (Domain_Filter).  The property is

  verified  when the pool empties;
  violated  when an input of the box has a negative margin (re-checked in FP64): searched before
            branching among random points of the box and its centre, then by projected
            sign-gradient descent on the lowest margin from the best of them; and, as branching
            goes on, at the point x* that minimises each bounded subdomain's linear bound (the
            upper bound f(x*) that Algorithm 1 keeps beside the lower bound, Appendix B.1);
  unknown   when the budget (rounds, bounded subdomains, time) runs out.

A subdomain with every root-unstable neuron split is linear on its region, so its bound is
concave in beta alone (Theorem 3.3): the driver then maximises it by projected gradient ascent
with a backtracking line search until the step vanishes (the bound then equals the subdomain's
exact minimum, Corollary 3.1) or the bound turns positive, which also catches the subdomains
whose splits contradict each other (an empty region makes the dual unbounded, Appendix B.3).
A negative converged bound is turned into a witness by evaluating the network at x*; without
one the subdomain stays open and the verdict unknown.

Branching rule: the paper names BaBSR and FSB but does not define their scores, so a static
rule stands in: the unsplit root-unstable neuron with the widest triangle relaxation, measured
by the intercept of its upper chord, u (-l) / (u - l).

The engine does the bounding: engine.optimize(subdomains, alpha, beta) -> (lb, alpha, beta) on
one batch (subdomains as (property, neuron indices, signs)); engine.bound_grad(...) -> (lb,
dlb/dalpha, dlb/dbeta) and engine.certify(...) -> lb at fixed alpha, beta; engine.xstar(...) ->
(x*, C f(x*)) per row; engine.margins(x) -> C f(x) in FP64 for rows of inputs.  GpuEngine runs
the library (BF16 iterations and the certifying pass; FP32 for the line search and x*).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as wl


@dataclass
class Domain:
    splits: np.ndarray   # global hidden-neuron indices, in split order
    signs: np.ndarray    # int8: -1 for z >= 0 (active), +1 for z <= 0 (inactive)
    alpha: np.ndarray    # [K * U] float32, layout [k][unstable rank]
    beta: np.ndarray     # [K * len(splits)] float32, layout [k][split]
    lb: np.ndarray       # [K] certified lower bounds of the margins
    owner: int = 0       # which of the properties being decided (bab_many) it belongs to

    @property
    def depth(self) -> int:
        return len(self.splits)


@dataclass
class BabResult:
    status: str                          # "verified", "violated" or "unknown"
    rounds: int = 0
    bounded: int = 0                     # subdomains bounded (the root included)
    max_depth: int = 0
    open_domains: int = 0
    min_lb: float = float("inf")         # lowest bound among open subdomains at exit
    witness: np.ndarray | None = None    # an input with a negative margin (violated)
    witness_margins: np.ndarray | None = None
    seconds: float = 0.0
    history: list = field(default_factory=list)   # per round: (open domains, min lb)
    upper: float = float("inf")          # lowest margin found at an input of the box (f-bar)
    line_searched: int = 0               # fully split subdomains maximised over beta alone
    infeasible: int = 0                  # of those, the ones whose bound grew past zero


def branching_scores(l, u):
    """Upper-chord intercept u (-l) / (u - l) of root-unstable neurons, -inf for stable ones."""
    l = np.asarray(l, np.float64)
    u = np.asarray(u, np.float64)
    un = (l < 0) & (u > 0)
    s = np.full(l.shape, -np.inf)
    s[un] = u[un] * (-l[un]) / (u[un] - l[un])
    return s


def _children(parent, j, K):
    """The two subdomains of splitting neuron j: alpha inherited, beta of the new split 0.

    The children share their parent's alpha and beta arrays: nothing writes them in place (a
    bounding call replaces them with views of its own results)."""
    cnt = parent.depth
    beta = np.zeros((K, cnt + 1), np.float32)
    beta[:, :cnt] = parent.beta.reshape(K, cnt)
    beta = beta.reshape(-1)
    splits = np.append(parent.splits, j)
    return [Domain(splits, np.append(parent.signs, np.int8(sign)), parent.alpha, beta, parent.lb, parent.owner)
            for sign in (-1, 1)]


def _next_neuron(d, order):
    """The first neuron of the branching order that d has not split.  Where d's splits are exactly
    the first depth neurons of the order (every subdomain the driver grows from the root), that is
    order[depth]; otherwise (subdomains given as starting points) scan."""
    k = d.depth
    if k < len(order) and np.array_equal(d.splits, order[:k]):
        return int(order[k])
    used = set(d.splits.tolist())
    return next((int(v) for v in order if int(v) not in used), None)


def _margin_fn(problem):
    """Differentiable margins C f(x) of rows of inputs (float64 torch on the host)."""
    import torch
    import torch.nn.functional as F
    layers = [(ly.kind, torch.as_tensor(np.asarray(ly.W, np.float64)), torch.as_tensor(np.asarray(ly.b, np.float64)),
               tuple(ly.in_shape), ly.stride, ly.pad) for ly in problem.layers]
    C = torch.as_tensor(np.asarray(problem.C, np.float64))

    def f(x):
        h, n = x, x.shape[0]
        for i, (kind, W, b, shape, stride, pad) in enumerate(layers):
            if kind == "fc":
                z = h.reshape(n, -1) @ W.T + b
            else:
                z = F.conv2d(h.reshape((n,) + shape), W, b, stride=stride, padding=pad).reshape(n, -1)
            h = torch.relu(z) if i < len(layers) - 1 else z
        return h @ C.T
    return f


def _pgd(problem, starts, x_lo, x_hi, steps, step_frac=0.25):
    """Projected sign-gradient descent on min_k margin_k(x) over the box from each start; returns
    the visited point with the lowest margin."""
    import torch
    f = _margin_fn(problem)
    lo = torch.as_tensor(x_lo)
    hi = torch.as_tensor(x_hi)
    x = torch.as_tensor(np.asarray(starts, np.float64)).clone()
    best_x, best_m = None, np.inf
    for t in range(steps):
        x.requires_grad_(True)
        m = f(x).min(dim=1).values
        md = m.detach()
        i = int(torch.argmin(md))
        if float(md[i]) < best_m:
            best_m, best_x = float(md[i]), x[i].detach().clone().numpy()
        (g,) = torch.autograd.grad(m.sum(), x)
        step = step_frac * (1.0 - t / steps) * (hi - lo)
        x = torch.minimum(torch.maximum(x.detach() - step * torch.sign(g), lo), hi)
    return best_x


def _falsify(engine, x_lo, x_hi, n_samples, rng, pgd_steps=0, pgd_starts=8):
    """Random points of the box and its centre, then projected gradient descent from the best
    of them; returns (x, margins) of the worst point found (margins from engine.margins)."""
    pts = [0.5 * (x_lo + x_hi)]
    if n_samples > 0:
        pts.append(rng.uniform(x_lo, x_hi, size=(n_samples, x_lo.shape[0])))
    x = np.vstack([np.atleast_2d(p) for p in pts])
    m = engine.margins(x)
    worst = m.min(axis=1)
    if worst.min() >= 0 and pgd_steps > 0:
        starts = x[np.argsort(worst)[:pgd_starts]]
        xp = _pgd(engine.pb, starts, x_lo, x_hi, pgd_steps)
        if xp is not None:
            x = np.vstack([x, xp[None]])
            m = np.vstack([m, engine.margins(xp[None])])
            worst = m.min(axis=1)
    i = int(np.argmin(worst))
    return x[i], m[i]


def _upper(engine, doms, cases, res):
    """f(x*) for every row of the bounded subdomains: the lowest margin at the points that minimise
    their linear bounds.  A negative one (re-checked in FP64) decides its property: violated."""
    if not doms:
        return
    subs = [(cases[d.owner][0], d.splits, d.signs) for d in doms]
    xs, m = engine.xstar(subs, np.concatenate([d.alpha for d in doms]), np.concatenate([d.beta for d in doms]))
    K = engine.K
    worst = m.min(axis=1).reshape(len(doms), K)
    for i, d in enumerate(doms):
        r = res[d.owner]
        j = int(np.argmin(worst[i]))
        if worst[i, j] < r.upper or worst[i, j] < 0:
            x = np.asarray(xs[i * K + j], np.float64)
            m64 = engine.margins(x[None])[0]
            r.upper = min(r.upper, float(m64.min()))
            if m64.min() < 0 and r.status != "violated":
                r.status, r.witness, r.witness_margins = "violated", x, m64


LINE_SEARCH_LRS = (0.05, 0.2, 1.0)   # initial step sizes of the beta ascent tried per subdomain


def _line_search(engine, doms, cases, K, iters=500, decay=0.99, lrs=LINE_SEARCH_LRS, tol=1e-6):
    """Fully split subdomains (no alpha left in their bound): the bound is concave and piecewise
    linear in beta (Theorem 3.3), so ascent on beta alone reaches its maximum, the exact minimum
    of the region (Corollary 3.1).  The paper suggests a line search so that convergence does not
    hang on a preset learning rate; along a supergradient of this piecewise-linear function a
    backtracking search stalls at the kinks (measured on the tiny nets: a few percent short after
    200 steps), so the search here is over the step size of the projected Adam ascent on beta:
    one FP32 run per initial step size in `lrs` (decayed by `decay` per step), keeping per row
    the best certified bound.  A row is converged when its bound turned positive (verified; an
    empty region, whose dual is unbounded, ends here too, Appendix B.3) or the runs agree to
    within tol.  Returns (certified lb [n, K], converged [n])."""
    subs = [(cases[d.owner][0], d.splits, d.signs) for d in doms]
    alpha = np.concatenate([d.alpha for d in doms])
    beta0 = np.concatenate([d.beta for d in doms])
    boff = np.concatenate([[0], np.cumsum([K * d.depth for d in doms])]).astype(np.int64)
    rows = np.repeat(np.arange(len(doms) * K), np.repeat([d.depth for d in doms], K))   # row of each beta
    best = lo = None
    best_beta = None
    for lr in lrs:
        lb, _, b = engine.optimize(subs, alpha, beta0, iters=iters, lr_alpha=0.0, lr_beta=lr, decay=decay,
                                   fp32=True)
        lb = np.asarray(lb, np.float64)
        b = np.asarray(b, np.float32)
        if best is None:
            best, lo, best_beta = lb.copy(), lb.copy(), b.copy()
            continue
        better = lb > best
        best = np.where(better, lb, best)
        lo = np.minimum(lo, lb)
        best_beta = np.where(better[rows], b, best_beta)
    conv = (best > 0) | (best - lo <= tol * np.maximum(1.0, np.abs(best)))
    cert = best.reshape(len(doms), K)
    for i, d in enumerate(doms):
        d.beta = best_beta[boff[i]:boff[i + 1]]
        d.lb = cert[i].astype(np.float32)
    return cert, conv.reshape(len(doms), K).all(axis=1)


def bab(engine, prop, l, u, x_lo, x_hi, batch_size=512, max_rounds=50, max_bounded=1_000_000,
        n_samples=256, seed=0, time_limit=None, alpha_init=0.5, pgd_steps=20, start=None, upper=True,
        line_search=True, joint=False):
    """Decide property `prop` (its box x_lo, x_hi and root bounds l, u over all hidden neurons).

    start: subdomains to begin from instead of the whole box, as (neuron indices, signs) pairs;
    "verified" then covers their union only (a witness of "violated" may lie anywhere in the box)."""
    return bab_many(engine, [(prop, l, u, x_lo, x_hi)], batch_size=batch_size, max_rounds=max_rounds,
                    max_bounded=max_bounded, n_samples=n_samples, seed=seed, time_limit=time_limit,
                    alpha_init=alpha_init, pgd_steps=pgd_steps, starts=None if start is None else [start],
                    upper=upper, line_search=line_search, joint=joint)[0]


def _own(d):
    """A subdomain that stays in the pool gets its own alpha and beta (they are slices of the
    batch-wide result arrays, which would otherwise stay alive as long as any descendant does)."""
    d.alpha, d.beta = d.alpha.copy(), d.beta.copy()
    return d


def _bound(engine, doms, cases, K, Us, joint=False):
    """One engine call on a list of subdomains (of any of the properties); results written back.
    joint: the intermediate bounds are recomputed per subdomain and optimised with alpha, beta
    (Section 3.3; alpha' starts at the root rule and beta' at 0 for every call)."""
    opt = engine.optimize_joint if joint else engine.optimize
    lb, a, b = opt([(cases[d.owner][0], d.splits, d.signs) for d in doms],
                   np.concatenate([d.alpha for d in doms]), np.concatenate([d.beta for d in doms]))
    lb = np.asarray(lb, np.float32).reshape(len(doms), K)
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    aoff = np.concatenate([[0], np.cumsum([K * Us[d.owner] for d in doms])])
    boff = np.concatenate([[0], np.cumsum([K * d.depth for d in doms])])
    for i, d in enumerate(doms):
        d.lb, d.alpha, d.beta = lb[i], a[aoff[i]:aoff[i + 1]], b[boff[i]:boff[i + 1]]


def bab_many(engine, cases, batch_size=512, max_rounds=50, max_bounded=1_000_000, n_samples=256, seed=0,
             time_limit=None, alpha_init=0.5, pgd_steps=20, starts=None, upper=True, line_search=True, joint=False):
    """Decide several properties at once: cases = [(prop, l, u, x_lo, x_hi), ...].  Their open
    subdomains share one pool, so each engine call bounds the lowest-bound subdomains of all the
    properties still open together (one batch of mixed properties).  Returns one BabResult per
    case; starts, if given, holds each case's start subdomains (see bab).  upper: evaluate the
    network at every bounded subdomain's x*; line_search: take fully split subdomains to their
    exact minimum over beta (both on by default; off, the driver is the plain Algorithm 1 loop).
    joint: bound every subdomain with its intermediate bounds recomputed and optimised jointly
    (Section 3.3, engine.optimize_joint; FP32 bounds, the certifying pass is not applied)."""
    t0 = time.perf_counter()
    K = engine.K
    n = len(cases)
    res = [BabResult("unknown") for _ in range(n)]
    orders, Us = [], []
    for c, (prop, l, u, x_lo, x_hi) in enumerate(cases):
        scores = branching_scores(l, u)
        Us.append(int(np.isfinite(scores).sum()))
        orders.append(np.argsort(-scores, kind="stable")[:Us[-1]])   # root-unstable, widest first
    open_case = [True] * n
    for c, (prop, l, u, x_lo, x_hi) in enumerate(cases):
        x, m = _falsify(engine, np.asarray(x_lo, np.float64), np.asarray(x_hi, np.float64), n_samples,
                        np.random.default_rng(seed + c), pgd_steps)
        if m.min() < 0:
            res[c].status, res[c].witness, res[c].witness_margins = "violated", x, m
            open_case[c] = False

    first = []
    for c in range(n):
        if not open_case[c]:
            continue
        st = [(np.zeros(0, np.int64), np.zeros(0, np.int8))] if starts is None else starts[c]
        first += [Domain(np.asarray(sp, np.int64), np.asarray(sg, np.int8), np.full(K * Us[c], alpha_init, np.float32),
                         np.zeros(K * len(sp), np.float32), np.full(K, -np.inf, np.float32), c) for sp, sg in st]
    pool, exhausted = [], []
    if first:
        _bound(engine, first, cases, K, Us, joint)
        if upper:
            _upper(engine, first, cases, res)
        for d in first:
            res[d.owner].bounded += 1
            res[d.owner].max_depth = max(res[d.owner].max_depth, d.depth)
            if d.lb.min() <= 0:
                pool.append(_own(d))
    for c in range(n):
        if open_case[c] and res[c].status == "violated":
            open_case[c] = False
    pool = [d for d in pool if open_case[d.owner]]
    rounds = bounded = 0
    while pool or any(open_case[d.owner] and not getattr(d, "searched", False) for d in exhausted):
        if rounds >= max_rounds or bounded >= max_bounded or (
                time_limit is not None and time.perf_counter() - t0 > time_limit):
            break
        rounds += 1
        pool.sort(key=lambda d: float(d.lb.min()))
        take, pool = pool[:batch_size], pool[batch_size:]
        kids = []
        for c in {d.owner for d in take}:
            res[c].rounds += 1
        for d in take:
            j = _next_neuron(d, orders[d.owner])
            if j is None:
                exhausted.append(d)
                continue
            kids.extend(_children(d, j, K))
        if kids:
            _bound(engine, kids, cases, K, Us, joint)
            if upper:
                _upper(engine, kids, cases, res)
            bounded += len(kids)
            for k in kids:
                r = res[k.owner]
                r.bounded += 1
                r.max_depth = max(r.max_depth, k.depth)
                if k.lb.min() <= 0:      # Domain_Filter: keep the subdomains not yet verified
                    pool.append(_own(k))
        # a property with a witness is decided: its subdomains leave the pool
        for c in range(n):
            if open_case[c] and res[c].status == "violated":
                open_case[c] = False
        pool = [d for d in pool if open_case[d.owner]]
        # fully split subdomains: beta alone, to the exact subdomain minimum (Theorem 3.3)
        fresh = [d for d in exhausted if open_case[d.owner] and not getattr(d, "searched", False)]
        if fresh and not line_search:
            for d in fresh:
                d.searched = True
        elif fresh:
            cert, conv = _line_search(engine, fresh, cases, K)
            _upper(engine, fresh, cases, res)   # x* of the maximised bound: the witness of a negative minimum
            keep = []
            for d, ok in zip(fresh, conv):
                d.searched = True
                res[d.owner].line_searched += 1
                if d.lb.min() > 0:
                    res[d.owner].infeasible += int(not ok)   # grew past zero before converging
                else:
                    keep.append(d)
            exhausted = [d for d in exhausted if not getattr(d, "searched", False)] + keep
            for c in range(n):
                if open_case[c] and res[c].status == "violated":
                    open_case[c] = False
        exhausted = [d for d in exhausted if open_case[d.owner]]
        for c in range(n):
            if open_case[c]:
                left = [float(d.lb.min()) for d in pool + exhausted if d.owner == c]
                res[c].history.append((len(left), min(left, default=float("inf"))))
    for c in range(n):
        if not open_case[c] or res[c].status == "violated":
            continue
        left = [d for d in pool + exhausted if d.owner == c]
        res[c].open_domains = len(left)
        res[c].min_lb = min([float(d.lb.min()) for d in left], default=float("inf"))
        res[c].status = "verified" if not left else "unknown"
    dt = time.perf_counter() - t0
    for r in res:
        r.seconds = dt
    return res


_CODE = {"verified": 0, "unknown": 1, "violated": 2}


def rank_starts(l, u, rank, world):
    """The subdomains rank `rank` of `world` starts from: the sign patterns r, r + world, ... of
    the first k = ceil(log2 world) neurons of the branching order (fewer if fewer are unstable)."""
    scores = branching_scores(l, u)
    U = int(np.isfinite(scores).sum())
    order = np.argsort(-scores, kind="stable")[:U]
    k = min(int(np.ceil(np.log2(world))) if world > 1 else 0, U)
    top = order[:k].astype(np.int64)
    patterns = [np.array([(-1 if (p >> i) & 1 == 0 else 1) for i in range(k)], np.int8) for p in range(1 << k)]
    return [(top, sg) for sg in patterns[rank::world]]


def bab_ranks(engine, prop, l, u, x_lo, x_hi, rank, world, dist, seed=0, driver="list", **kw):
    """One property decided by `world` ranks (one process per GPU, torch.distributed `dist`).
    driver: "list" (bab) or "pool" (bab_pool.bab_pool, the pool in arrays; alpha and beta on the
    device the engine computes on).

    The first k = ceil(log2 world) neurons of the (static) branching order give 2^k subdomains;
    rank r decides those with index r, r + world, ... on its own, with its own sampling seed.
    The verdicts then combine in one all-reduce: violated if any rank found a witness (which the
    lowest such rank broadcasts), verified if every rank verified its share, unknown otherwise.
    There is no exchange while the ranks branch."""
    import torch
    mine = rank_starts(l, u, rank, world)
    if driver == "pool":
        from . import bab_pool
        res = bab_pool.bab_pool(engine, [(prop, l, u, x_lo, x_hi)], seed=seed + rank, starts=[mine], **kw)[0]
    else:
        res = bab(engine, prop, l, u, x_lo, x_hi, seed=seed + rank, start=mine, **kw)
    t = torch.tensor([_CODE[res.status]], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    status = {v: s for s, v in _CODE.items()}[int(t.item())]
    tot = torch.tensor([res.bounded, res.rounds], dtype=torch.int64)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    out = BabResult(status, rounds=int(tot[1]), bounded=int(tot[0]), max_depth=res.max_depth,
                    open_domains=res.open_domains, min_lb=res.min_lb, seconds=res.seconds)
    if status == "violated":
        src = torch.tensor([rank if res.status == "violated" else world], dtype=torch.int64)
        dist.all_reduce(src, op=dist.ReduceOp.MIN)
        w = torch.zeros(len(x_lo) + engine.K, dtype=torch.float64)
        if int(src) == rank:
            w = torch.as_tensor(np.concatenate([res.witness, res.witness_margins]).astype(np.float64))
        dist.broadcast(w, int(src))
        out.witness, out.witness_margins = w[:len(x_lo)].numpy(), w[len(x_lo):].numpy()
    return out


class GpuEngine:
    """Bounds through the library: bcrown_optimize with BF16 iterations (the tensor-core path)
    and the FP32 certifying pass, on the GPU; margins C f(x) in FP64 on the host."""

    def __init__(self, problem, net, dom, unstable_counts, precision=None, iters=20, graphs=False):
        from . import bcrown as bc
        self.bc = bc
        self.pb = problem
        self.net = net
        self.dom = dom
        self.K = problem.K
        self.U = list(unstable_counts)
        self.cfg = bc.OptCfg(iters=iters, precision=bc.BF16 if precision is None else precision, certify=True)
        # graphs: optimisation calls at the engine's settings replay a CUDA graph per batch-size bucket
        self.graphs = bc.GraphOptimizer(net, dom, self.cfg, self.U) if graphs else None

    def optimize(self, subs, alpha, beta, iters=None, lr_alpha=None, lr_beta=None, decay=None, fp32=False):
        """The optimised, certified bound (bcrown_optimize); the keywords override the engine's
        settings for one call (fp32: FP32 iterations instead of BF16)."""
        import dataclasses
        if self.graphs is not None and not fp32 and all(v is None for v in (iters, lr_alpha, lr_beta, decay)):
            lb, a, b = self.graphs(wl.pack_batch(self.pb.hidden_widths, self.K, self.U, subs), alpha, beta)
            self._check()
            return lb, a, b
        db, at, bt = self._args(subs, alpha, beta)
        cfg = dataclasses.replace(self.cfg, **{k: v for k, v in dict(iters=iters, lr_alpha=lr_alpha, lr_beta=lr_beta,
                                                                      decay=decay).items() if v is not None})
        if fp32:
            cfg = dataclasses.replace(cfg, precision=self.bc.FP32)
        lb = self.bc.optimize(self.net, self.dom, db, at, bt, cfg)
        st = self.bc.status(self.net)
        if st != 0:
            raise RuntimeError(f"bcrown device status {st}")
        return lb.cpu().numpy(), at.cpu().numpy(), bt.cpu().numpy()

    def optimize_joint(self, subs, alpha, beta):
        """The bound with the intermediate bounds recomputed per subdomain and optimised jointly with
        alpha, beta (bcrown_optimize_joint, FP32); alpha' starts at the root rule, beta' at 0."""
        import dataclasses
        db, at, bt = self._args(subs, alpha, beta)
        ap, bp = self.bc.joint_init_alpha(self.net, self.dom, db)
        cfg = dataclasses.replace(self.cfg, precision=self.bc.FP32, certify=False)
        lb, _, _ = self.bc.optimize_joint(self.net, self.dom, db, at, bt, ap, bp, cfg=cfg)
        self._check()
        return lb.cpu().numpy(), at.cpu().numpy(), bt.cpu().numpy()

    # the array-pool driver's interface (bab_pool): alpha [B, K * Umax] and compact beta stay on the
    # device; only the batch's split lists (a few bytes per subdomain) are copied to it
    def optimize_rows(self, batch, alpha, beta):
        """The optimised, certified bound of a host batch; alpha and beta (device tensors) are
        overwritten with the per-row best values.  Returns lb [B*K] on the device."""
        if self.graphs is not None:
            lb = self.graphs.rows(batch, alpha, beta)
            self._check()
            return lb
        db = self.bc.DeviceBatch.from_host(batch)
        lb = self.bc.optimize(self.net, self.dom, db, alpha, beta, self.cfg)
        self._check()
        return lb

    def xstar_rows(self, batch, alpha, beta):
        """Per row, the box point x* that minimises its linear bound and C f(x*) (device tensors)."""
        db = self.bc.DeviceBatch.from_host(batch)
        _, xs = self.bc.bound_xstar(self.net, self.dom, db, alpha, beta)
        m = self.bc.forward(self.net, xs)
        self._check()
        return xs, m

    def _args(self, subs, alpha, beta):
        import torch
        batch = wl.pack_batch(self.pb.hidden_widths, self.K, self.U, subs)
        db = self.bc.DeviceBatch.from_host(batch)
        at = torch.as_tensor(np.ascontiguousarray(alpha, np.float32)).cuda()
        bt = torch.as_tensor(np.ascontiguousarray(beta, np.float32)).cuda()
        return db, at, bt

    def _check(self):
        st = self.bc.status(self.net)
        if st != 0:
            raise RuntimeError(f"bcrown device status {st}")

    def bound_grad(self, subs, alpha, beta):
        db, at, bt = self._args(subs, alpha, beta)
        lb, da, dbeta = self.bc.bound_grad(self.net, self.dom, db, at, bt, self.bc.FP32)
        self._check()
        return lb.cpu().numpy(), da.cpu().numpy(), dbeta.cpu().numpy()

    def certify(self, subs, alpha, beta):
        db, at, bt = self._args(subs, alpha, beta)
        lb = self.bc.bound(self.net, self.dom, db, at, bt, self.bc.CERTIFY)
        self._check()
        return lb.cpu().numpy()

    def xstar(self, subs, alpha, beta):
        db, at, bt = self._args(subs, alpha, beta)
        _, xs = self.bc.bound_xstar(self.net, self.dom, db, at, bt)
        m = self.bc.forward(self.net, xs)
        self._check()
        return xs.cpu().numpy(), m.cpu().numpy()

    def margins(self, x):
        f = wl.reference_forward(self.pb.layers, x)
        return np.atleast_2d(f) @ self.pb.C.astype(np.float64).T

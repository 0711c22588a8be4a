"""Branch-and-bound driver (Algorithm 1) on the oracle: its verdicts against the exact minimum of
each margin over the box (all activation patterns enumerated, one LP each), and its host logic."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from oracle import lp_pins as LP
from paper_2103_06624_gb300 import bab
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import oracle_setup


class OracleEngine:
    """The driver's engine interface on the FP64 oracle (projected Adam, 20 iterations)."""

    def __init__(self, pb, props, U):
        self.pb, self.props, self.U = pb, props, list(U)
        self.onet = O.OracleNet(pb.layers, pb.C)
        self.K = pb.K
        self.calls = 0

    def optimize(self, subs, alpha, beta, iters=None, lr_alpha=None, lr_beta=None, decay=None, fp32=False):
        self.calls += 1
        import dataclasses
        cfg = dataclasses.replace(O.AdamCfg(), **{k: v for k, v in dict(iters=iters, lr_alpha=lr_alpha,
                                                                         lr_beta=lr_beta, decay=decay).items()
                                                   if v is not None})
        batch = wl.pack_batch(self.pb.hidden_widths, self.K, self.U, subs)
        lb, a, b, _ = O.optimize(self.onet, self.props, batch, alpha, beta, cfg)
        return lb, a, b

    def optimize_joint(self, subs, alpha, beta):
        self.calls += 1
        from oracle import joint as J
        batch = self._batch(subs)
        lay = J.joint_layout(self.onet, batch, self.props["l"], self.props["u"])
        ap0 = J.init_alpha_p(self.onet, batch, self.props["l"], self.props["u"])
        lb, a, b, *_ = J.joint_optimize(self.onet, self.props, batch, alpha, beta, ap0, np.zeros(lay.n_beta_p))
        return lb, a, b

    def _batch(self, subs):
        return wl.pack_batch(self.pb.hidden_widths, self.K, self.U, subs)

    def bound_grad(self, subs, alpha, beta):
        lb, da, db = O.grad(self.onet, self.props, self._batch(subs), np.asarray(alpha, np.float64),
                            np.asarray(beta, np.float64))
        return lb, da, db

    def certify(self, subs, alpha, beta):
        return O.bound(self.onet, self.props, self._batch(subs), alpha, beta)

    def xstar(self, subs, alpha, beta):
        batch = self._batch(subs)
        rows = O.expand_rows(self.onet, batch, self.props["l"], self.props["u"])
        _, tr = O.bound(self.onet, self.props, batch, alpha, beta, rows=rows, trace=True)
        xlo = np.asarray(self.props["x_lo"], np.float64)[rows.prop]
        xhi = np.asarray(self.props["x_hi"], np.float64)[rows.prop]
        xs = np.where(tr.A[0] >= 0, xlo, xhi)
        return xs, self.margins(xs)

    def margins(self, x):
        return np.atleast_2d(wl.reference_forward(self.pb.layers, x)) @ self.pb.C.astype(np.float64).T

    # the array-pool driver's interface: batches in the C-ABI layout, alpha and beta as tensors
    def optimize_rows(self, batch, alpha_t, beta_t):
        self.calls += 1
        lb, a, b, _ = O.optimize(self.onet, self.props, batch, alpha_t.reshape(-1).numpy().astype(np.float64),
                                 beta_t.numpy().astype(np.float64), O.AdamCfg())
        alpha_t.copy_(torch.as_tensor(np.asarray(a, np.float32)).reshape(alpha_t.shape))
        beta_t.copy_(torch.as_tensor(np.asarray(b, np.float32)))
        return torch.as_tensor(np.asarray(lb, np.float64))

    def xstar_rows(self, batch, alpha_t, beta_t):
        rows = O.expand_rows(self.onet, batch, self.props["l"], self.props["u"])
        _, tr = O.bound(self.onet, self.props, batch, alpha_t.reshape(-1).numpy().astype(np.float64),
                        beta_t.numpy().astype(np.float64), rows=rows, trace=True)
        xlo = np.asarray(self.props["x_lo"], np.float64)[rows.prop]
        xhi = np.asarray(self.props["x_hi"], np.float64)[rows.prop]
        xs = np.where(tr.A[0] >= 0, xlo, xhi)
        return torch.as_tensor(xs), torch.as_tensor(self.margins(xs))


# (widths, seed, eps): the expected verdict follows from the exact minima computed in the test
CASES = {
    "verified_at_root": ([5, 10, 10, 4], 2, 0.1),
    "verified_by_branching_a": ([5, 10, 10, 4], 1, 0.15),
    "verified_by_branching_b": ([5, 10, 10, 4], 4, 0.15),
    "violated": ([5, 8, 8, 4], 0, 0.2),
    "violated_found_by_descent": ([4, 8, 6, 4], 4, 0.4),   # random points of the box all miss it
}


def make_case(name):
    widths, seed, eps = CASES[name]
    pb = wl.make_problem(name, wl.mlp_layers(widths, seed), 1, eps, 3, seed)
    onet, props, unst = oracle_setup(pb)
    exact = np.array([LP.exact_min(onet, pb.x_lo[0], pb.x_hi[0], props["l"][0], props["u"][0], [], k)
                      for k in range(pb.K)])
    return pb, props, unst, exact


def run_case(name, engine_factory, **kw):
    pb, props, unst, exact = make_case(name)
    eng = engine_factory(pb, props, [len(u) for u in unst])
    res = bab.bab(eng, 0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0], **kw)
    return pb, exact, res


def check_verdict(name, pb, exact, res):
    """Soundness in every case; the expected verdict where the exact minima decide it."""
    if res.status == "verified":
        assert exact.min() > 0, (name, exact)
    if res.status == "violated":
        x = res.witness
        assert np.all(x >= pb.x_lo[0] - 1e-12) and np.all(x <= pb.x_hi[0] + 1e-12)
        m = np.atleast_2d(wl.reference_forward(pb.layers, x)) @ pb.C.astype(np.float64).T
        assert m.min() < 0 and exact.min() < 0
    if name.startswith("verified"):
        assert res.status == "verified", (name, res.status, res.min_lb)
    else:
        assert res.status == "violated", (name, res.status)


@pytest.mark.parametrize("name", list(CASES))
def test_bab_on_the_oracle_agrees_with_exact_minima(name):
    pb, exact, res = run_case(name, OracleEngine, batch_size=256, max_rounds=12, n_samples=256)
    check_verdict(name, pb, exact, res)
    if name == "verified_at_root":
        assert res.rounds == 0 and res.bounded == 1
    if name.startswith("verified_by_branching"):
        assert res.rounds >= 1 and res.max_depth >= 1
        # every round's open subdomains have a lowest bound no better than the exact minimum
        assert all(mlb <= exact.min() + 1e-9 for _, mlb in res.history if np.isfinite(mlb))


def test_a_negative_minimum_is_never_verified_when_no_witness_is_found():
    """Random points of the box all have positive margins; gradient descent, the x* upper bound and
    the line search are switched off: branching must not verify the property (its exact minimum
    is negative), so every split is made and the fully split subdomains stay open: unknown."""
    pb, exact, res = run_case("violated_found_by_descent", OracleEngine, batch_size=256, max_rounds=12,
                              n_samples=256, pgd_steps=0, upper=False, line_search=False)
    assert exact.min() < 0
    assert res.status == "unknown" and res.open_domains > 0 and res.min_lb <= 0


@pytest.mark.parametrize("mechanism", ["upper", "line_search"])
def test_the_upper_bound_or_the_line_search_finds_the_violation_sampling_misses(mechanism):
    """The same net with no sampled point and no descent: the violation is found at x* of a bounded
    subdomain (Algorithm 1's upper bound f(x*), Appendix B.1), or -- with that switched off during
    branching -- once the fully split subdomains are maximised over beta (Theorem 3.3)."""
    pb, exact, res = run_case("violated_found_by_descent", OracleEngine, batch_size=256, max_rounds=12,
                              n_samples=0, pgd_steps=0, upper=(mechanism == "upper"),
                              line_search=(mechanism == "line_search"))
    check_verdict("violated_found_by_descent", pb, exact, res)
    if mechanism == "line_search":
        assert res.line_searched > 0


def test_line_search_reaches_the_exact_minimum_of_fully_split_subdomains():
    """Every unstable neuron split (a linear region): the beta-only ascent with its step-size search
    reaches the exact minimum of each spec over the region (Theorem 3.3, Corollary 3.1) -- the
    minimum found by scipy's LP over the region -- and never goes above it; rows whose minimum is
    positive end verified, and regions whose splits contradict each other (empty) end with a
    positive bound (Appendix B.3)."""
    pb, props, unst, _ = make_case("violated")
    onet = O.OracleNet(pb.layers, pb.C)
    l, u = props["l"][0], props["u"][0]
    U = len(unst[0])
    offs = np.concatenate([[0], np.cumsum(pb.hidden_widths)])
    rng = np.random.default_rng(0)
    # the activation patterns of sampled inputs (feasible regions), and random patterns (mostly empty)
    xs = rng.uniform(pb.x_lo[0], pb.x_hi[0], size=(8, pb.x_lo.shape[1]))
    z = np.concatenate([zi for zi in onet.preacts(xs)[1:]], axis=1)[:, unst[0]]
    patterns = [np.where(zi >= 0, -1, 1).astype(np.int8) for zi in z]
    patterns += [rng.choice([-1, 1], size=U).astype(np.int8) for _ in range(6)]
    doms = [bab.Domain(unst[0].astype(np.int64), sg, np.full(pb.K * U, 0.5, np.float32),
                       np.zeros(pb.K * U, np.float32), np.zeros(pb.K, np.float32), 0) for sg in patterns]
    eng = OracleEngine(pb, props, [U])
    cert, conv = bab._line_search(eng, doms, [(0, l, u, pb.x_lo[0], pb.x_hi[0])], pb.K)
    assert conv.all()
    n_neg = n_empty = 0
    for d, c in zip(doms, cert):
        layer = np.searchsorted(offs, d.splits, side="right")
        splits = [(int(i), int(g - offs[i - 1]), int(s)) for i, g, s in zip(layer, d.splits, d.signs)]
        for k in range(pb.K):
            ex = LP.exact_min(onet, pb.x_lo[0], pb.x_hi[0], l, u, splits, k)
            if not np.isfinite(ex):
                assert c[k] > 0      # an empty region: the dual grew without bound past zero
                n_empty += 1
            elif ex > 0:
                assert 0 < c[k] <= ex + 1e-9
            else:
                assert ex - 1e-6 * max(1.0, abs(ex)) <= c[k] <= ex + 1e-9, (k, c[k], ex)
                n_neg += 1
    assert n_neg > 0 and n_empty > 0


def test_children_inherit_alpha_and_start_the_new_beta_at_zero():
    K = 3
    parent = bab.Domain(np.array([7, 2]), np.array([-1, 1], np.int8), np.arange(K * 5, dtype=np.float32),
                        np.arange(K * 2, dtype=np.float32) + 1, np.zeros(K, np.float32))
    kids = bab._children(parent, 4, K)
    assert [k.signs.tolist() for k in kids] == [[-1, 1, -1], [-1, 1, 1]]
    for k in kids:
        assert k.splits.tolist() == [7, 2, 4]
        np.testing.assert_array_equal(k.alpha, parent.alpha)
        # beta layout [k][split]: the parent's two betas per spec, then 0 for the new split
        np.testing.assert_array_equal(k.beta.reshape(K, 3), [[1, 2, 0], [3, 4, 0], [5, 6, 0]])
    # the parent is left as it was
    assert parent.splits.tolist() == [7, 2] and parent.beta.tolist() == list(np.arange(K * 2) + 1.0)


def test_branching_scores_rank_the_widest_relaxations_first():
    l = np.array([-1.0, 0.5, -2.0, -0.5, -3.0])
    u = np.array([1.0, 2.0, 1.0, -0.1, 0.1])
    s = bab.branching_scores(l, u)
    assert np.isneginf(s[1]) and np.isneginf(s[3])       # stable neurons are never split
    np.testing.assert_allclose(s[[0, 2, 4]], [0.5, 2.0 / 3.0, 0.3 / 3.1])
    assert list(np.argsort(-s)[:3]) == [2, 0, 4]


def test_several_properties_share_one_pool():
    """Three properties of one net decided together (their subdomains bounded in mixed batches):
    each verdict matches the exact minima and the property's own single run, with fewer engine
    calls than the three single runs."""
    pb = wl.make_problem("multi", wl.mlp_layers([5, 10, 10, 4], 1), 3, 0.12, 3, 1)
    onet, props, unst = oracle_setup(pb)
    U = [len(u) for u in unst]
    exact = [min(LP.exact_min(onet, pb.x_lo[p], pb.x_hi[p], props["l"][p], props["u"][p], [], k)
                 for k in range(pb.K)) for p in range(pb.P)]
    cases = [(p, props["l"][p], props["u"][p], pb.x_lo[p], pb.x_hi[p]) for p in range(pb.P)]
    eng = OracleEngine(pb, props, U)
    many = bab.bab_many(eng, cases, batch_size=256, max_rounds=12, n_samples=256)
    calls_many = eng.calls
    calls_single = 0
    for p, r in enumerate(many):
        e1 = OracleEngine(pb, props, U)
        single = bab.bab(e1, *cases[p], batch_size=256, max_rounds=12, n_samples=256)
        calls_single += e1.calls
        assert r.status == single.status
        assert r.status == ("verified" if exact[p] > 0 else "violated"), (p, r.status, exact[p])
    assert [r.status for r in many] == ["verified", "violated", "verified"]
    assert calls_many < calls_single


@pytest.mark.parametrize("name", ["verified_by_branching_a", "verified_by_branching_b", "violated"])
def test_joint_mode_reaches_the_exact_verdicts_with_no_more_branching(name):
    """The driver with every subdomain's intermediate bounds recomputed and optimised jointly
    (Section 3.3): the verdicts still follow the exact minima, and the tighter bounds need at most
    as many bounded subdomains as the fixed-bound driver (the joint rows of Table A4 count fewer
    branches)."""
    pb, exact, plain = run_case(name, OracleEngine, batch_size=256, max_rounds=12, n_samples=256)
    _, _, joint = run_case(name, OracleEngine, batch_size=256, max_rounds=12, n_samples=256, joint=True)
    check_verdict(name, pb, exact, joint)
    assert joint.bounded <= plain.bounded, (joint.bounded, plain.bounded)


def _same_result(a, b):
    assert a.status == b.status
    assert (a.rounds, a.bounded, a.max_depth, a.open_domains) == (b.rounds, b.bounded, b.max_depth, b.open_domains)
    assert (a.line_searched, a.infeasible) == (b.line_searched, b.infeasible)
    assert a.min_lb == b.min_lb and a.upper == b.upper
    assert a.history == b.history
    if a.status == "violated":
        assert np.array_equal(a.witness, b.witness)


@pytest.mark.parametrize("name", list(CASES))
def test_array_pool_driver_takes_the_same_steps_as_the_list_driver(name):
    """The driver with the pool in arrays (alpha, beta as tensors, split lists implicit in the
    branching order) against the list driver on the same deterministic engine: the same rounds,
    counts, per-round pool sizes and lowest bounds, upper bound and verdict, on every tiny case
    (verified at the root, by branching with line searches of fully split subdomains, violated)."""
    from paper_2103_06624_gb300 import bab_pool
    pb, props, unst, exact = make_case(name)
    U = [len(u) for u in unst]
    case = (0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0])
    ref = bab.bab_many(OracleEngine(pb, props, U), [case], batch_size=8, max_rounds=30, n_samples=64)[0]
    got = bab_pool.bab_pool(OracleEngine(pb, props, U), [case], batch_size=8, max_rounds=30, n_samples=64,
                            device="cpu")[0]
    _same_result(ref, got)
    check_verdict(name, pb, exact, got)


def test_array_pool_driver_with_several_properties():
    """Three properties in one pool (their own orders and unstable counts, alpha rows padded to the
    largest): the same per-property results as the list driver."""
    from paper_2103_06624_gb300 import bab_pool
    pb = wl.make_problem("multi", wl.mlp_layers([5, 10, 10, 4], 1), 3, 0.15, 3, 1)
    onet, props, unst = oracle_setup(pb)
    U = [len(u) for u in unst]
    cases = [(p, props["l"][p], props["u"][p], pb.x_lo[p], pb.x_hi[p]) for p in range(pb.P)]
    ref = bab.bab_many(OracleEngine(pb, props, U), cases, batch_size=8, max_rounds=20, n_samples=64)
    got = bab_pool.bab_pool(OracleEngine(pb, props, U), cases, batch_size=8, max_rounds=20, n_samples=64,
                            device="cpu")
    for a, b in zip(ref, got):
        _same_result(a, b)


@pytest.mark.parametrize("upper,line_search", [(True, True), (False, True), (False, False)])
def test_array_pool_driver_branches_to_full_depth_like_the_list_driver(upper, line_search):
    """No sampled point and no descent on the net whose violation sampling misses: the violation is
    found at x* during branching, or by the line search of the fully split subdomains, or (both off)
    the verdict stays unknown with fully split subdomains open -- the same steps in both drivers."""
    from paper_2103_06624_gb300 import bab_pool
    pb, props, unst, exact = make_case("violated_found_by_descent")
    U = [len(u) for u in unst]
    case = (0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0])
    kw = dict(batch_size=256, max_rounds=12, n_samples=0, pgd_steps=0, upper=upper, line_search=line_search)
    ref = bab.bab_many(OracleEngine(pb, props, U), [case], **kw)[0]
    got = bab_pool.bab_pool(OracleEngine(pb, props, U), [case], device="cpu", **kw)[0]
    _same_result(ref, got)
    if not upper:
        assert got.max_depth == U[0]   # every neuron split before the verdict
    if line_search and not upper:
        assert got.line_searched > 0
    assert got.status == ("unknown" if not (upper or line_search) else "violated")


def test_array_pool_driver_from_start_subdomains():
    """Start subdomains on the first branching neurons (one rank's share of two): the same steps as
    the list driver from the same starts; a start that skips a neuron of the order is refused."""
    from paper_2103_06624_gb300 import bab_pool
    pb, props, unst, exact = make_case("verified_by_branching_a")
    U = [len(u) for u in unst]
    l, u = props["l"][0], props["u"][0]
    case = (0, l, u, pb.x_lo[0], pb.x_hi[0])
    for rank in range(2):
        mine = bab.rank_starts(l, u, rank, 4)
        ref = bab.bab_many(OracleEngine(pb, props, U), [case], batch_size=8, max_rounds=30, n_samples=64,
                           starts=[mine])[0]
        got = bab_pool.bab_pool(OracleEngine(pb, props, U), [case], batch_size=8, max_rounds=30, n_samples=64,
                                starts=[mine], device="cpu")[0]
        _same_result(ref, got)
    order = np.argsort(-bab.branching_scores(l, u), kind="stable")
    with pytest.raises(ValueError):
        bab_pool.bab_pool(OracleEngine(pb, props, U), [case], starts=[[(order[1:2], np.array([1], np.int8))]],
                          n_samples=0, pgd_steps=0, device="cpu")


def test_pool_batch_equals_the_packed_split_lists():
    """The array pool's vectorised batch builder against workloads.pack_batch on the same
    subdomains (split lists = prefixes of each property's branching order): the same properties,
    offsets, counts, layers, indices and signs; alpha blocks K * max U apart."""
    from paper_2103_06624_gb300 import bab_pool
    rng = np.random.default_rng(5)
    hw = [7, 5, 9]
    K = 3
    H = sum(hw)
    orders = np.stack([rng.permutation(H)[:10] for _ in range(2)]).astype(np.int64)
    U = [10, 8]
    n = 40
    owner = rng.integers(0, 2, n).astype(np.int32)
    depth = np.array([rng.integers(0, U[o] + 1) for o in owner], np.int32)
    signs = rng.choice(np.array([-1, 1], np.int8), size=(n, 10))
    props = np.array([4, 1], np.int32)
    got = bab_pool.pool_batch(hw, K, max(U), orders, props, depth, owner, signs)
    subs = [(int(props[o]), orders[o, :d], signs[i, :d]) for i, (o, d) in enumerate(zip(owner, depth))]
    Up = np.zeros(5, np.int64)
    Up[props] = U
    ref = wl.pack_batch(hw, K, Up, subs)
    for f in ("prop_of", "split_off", "split_cnt", "split_layer", "split_idx", "split_sign"):
        np.testing.assert_array_equal(getattr(got, f), getattr(ref, f), err_msg=f)
    np.testing.assert_array_equal(got.alpha_off, np.arange(n) * K * max(U))
    assert got.n_alpha == n * K * max(U) and got.n_beta == ref.n_beta

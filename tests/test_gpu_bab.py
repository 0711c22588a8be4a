"""Branch and bound through the library (needs a GB300): the driver of Algorithm 1 on the GPU
engine (BF16 iterations, FP32 certifying pass) reaches the verdicts the exact minima fix, like
the oracle engine; the ablation settings of the optimiser (alpha only, beta only); and the
driver with the joint intermediate-bound optimisation."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import bab
from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import oracle_setup
from tests.test_bab import CASES, OracleEngine, check_verdict, make_case, run_case

pytestmark = pytest.mark.gpu


def gpu_engine(pb, props, U):
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    return bab.GpuEngine(pb, net, dom, U)


@pytest.mark.parametrize("name", list(CASES))
def test_bab_on_the_gpu_reaches_the_exact_verdict(name):
    pb, exact, res = run_case(name, gpu_engine, batch_size=256, max_rounds=12, n_samples=256)
    print("%s: %s, rounds %d, subdomains %d, depth %d" % (name, res.status, res.rounds, res.bounded, res.max_depth))
    check_verdict(name, pb, exact, res)
    _, _, ref = run_case(name, OracleEngine, batch_size=256, max_rounds=12, n_samples=256)
    assert res.status == ref.status


@pytest.mark.parametrize("frozen", ["alpha", "beta"])
def test_ablation_settings_freeze_one_set_of_variables(frozen):
    """lr_alpha = 0 keeps alpha (the beta-only variant), lr_beta = 0 keeps beta (alpha only);
    the bound at the returned variables stays certified."""
    pb = wl.problem_mlp_small()
    onet, props, unst = oracle_setup(pb)
    batch = wl.random_batch(pb, unst, 32, 1, 4, 1)
    a0, b0 = wl.random_alpha_beta(batch, 7, 0.5)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    db = bc.DeviceBatch.from_host(batch)
    at, bt = torch.as_tensor(a0).cuda(), torch.as_tensor(b0).cuda()
    cfg = bc.OptCfg(lr_alpha=0.0 if frozen == "alpha" else 0.1, lr_beta=0.0 if frozen == "beta" else 0.05,
                    precision=bc.BF16, certify=True)
    lb = bc.optimize(net, dom, db, at, bt, cfg).cpu().numpy()
    assert bc.status(net) == 0
    a, b = at.cpu().numpy(), bt.cpu().numpy()
    if frozen == "alpha":
        np.testing.assert_array_equal(a, a0)
        assert np.abs(b - b0).max() > 0
    else:
        np.testing.assert_array_equal(b, b0)
        assert np.abs(a - a0).max() > 0
    ref = O.bound(onet, props, batch, a, b)
    assert np.all(lb <= ref + 1e-12 * np.abs(ref))


@pytest.mark.parametrize("name", ["verified_by_branching_a", "verified_by_branching_b"])
def test_joint_mode_on_the_gpu_reaches_the_oracle_verdict_with_no_more_branching(name):
    """The driver with the joint intermediate-bound optimisation on the GPU engine
    (bcrown_optimize_joint): the verdict of the exact minima, and no more bounded subdomains than
    the fixed-bound driver on the same engine."""
    pb, exact, plain = run_case(name, gpu_engine, batch_size=256, max_rounds=12, n_samples=256)
    _, _, joint = run_case(name, gpu_engine, batch_size=256, max_rounds=12, n_samples=256, joint=True)
    print("%s: fixed bounds %d subdomains in %d rounds, joint %d in %d" % (name, plain.bounded, plain.rounds,
                                                                          joint.bounded, joint.rounds))
    check_verdict(name, pb, exact, joint)
    assert joint.bounded <= plain.bounded


def test_graph_replayed_engine_gives_the_same_decisions():
    """GpuEngine(graphs=True): every optimisation call at the engine's settings replays a CUDA
    graph captured per batch-size bucket; the driver's verdict, round count and bounded subdomains
    equal those of the eager engine."""
    name = "verified_by_branching_a"

    def graph_engine(pb, props, U):
        net = bc.load_net(pb.layers, pb.C)
        dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
        return bab.GpuEngine(pb, net, dom, U, graphs=True)

    pb, exact, eager = run_case(name, gpu_engine, batch_size=256, max_rounds=12, n_samples=256)
    _, _, replay = run_case(name, graph_engine, batch_size=256, max_rounds=12, n_samples=256)
    check_verdict(name, pb, exact, replay)
    assert (replay.status, replay.rounds, replay.bounded) == (eager.status, eager.rounds, eager.bounded)


@pytest.mark.parametrize("name", list(CASES))
def test_array_pool_driver_on_the_gpu_reaches_the_exact_verdict(name):
    """The driver with alpha and beta resident on the device (bab_pool) through the library: the
    verdicts the exact minima fix, and those of the list driver on the same engine."""
    from paper_2103_06624_gb300 import bab_pool
    pb, props, unst, exact = make_case(name)
    U = [len(u) for u in unst]
    case = (0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0])
    res = bab_pool.bab_pool(gpu_engine(pb, props, U), [case], batch_size=256, max_rounds=12, n_samples=256)[0]
    print("%s: %s, rounds %d, subdomains %d, depth %d" % (name, res.status, res.rounds, res.bounded, res.max_depth))
    check_verdict(name, pb, exact, res)
    ref = bab.bab_many(gpu_engine(pb, props, U), [case], batch_size=256, max_rounds=12, n_samples=256)[0]
    assert res.status == ref.status


@pytest.mark.parametrize("upper,line_search", [(True, False), (False, True)])
def test_array_pool_driver_on_the_gpu_finds_the_violation_sampling_misses(upper, line_search):
    """No sampled point and no descent: the violation is found at x* of a bounded subdomain, or by
    the line search of the fully split subdomains (their alpha and beta read back from the device)."""
    from paper_2103_06624_gb300 import bab_pool
    pb, props, unst, exact = make_case("violated_found_by_descent")
    U = [len(u) for u in unst]
    case = (0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0])
    res = bab_pool.bab_pool(gpu_engine(pb, props, U), [case], batch_size=256, max_rounds=12, n_samples=0,
                            pgd_steps=0, upper=upper, line_search=line_search)[0]
    check_verdict("violated_found_by_descent", pb, exact, res)
    assert res.status == "violated"
    if line_search:
        assert res.line_searched > 0


@pytest.mark.parametrize("name", ["verified_by_branching_a", "violated_found_by_descent"])
def test_array_pool_driver_with_graph_replay_takes_the_same_steps(name):
    """GpuEngine(graphs=True) under the array pool: alpha and beta are copied device to device into
    the bucket's captured buffers (the padding subdomains get copies of the last one's) and the
    graph replayed; the same verdict, rounds, subdomain counts and per-round bounds as the eager
    engine, and, for the net whose violation sampling misses, the violation found at x*."""
    from paper_2103_06624_gb300 import bab_pool
    pb, props, unst, exact = make_case(name)
    U = [len(u) for u in unst]
    case = (0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0])

    def engine(graphs):
        net = bc.load_net(pb.layers, pb.C)
        dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
        return bab.GpuEngine(pb, net, dom, U, graphs=graphs)

    kw = dict(batch_size=48, max_rounds=12, n_samples=0, pgd_steps=0, line_search=False)
    eager = bab_pool.bab_pool(engine(False), [case], **kw)[0]
    eng = engine(True)
    replay = bab_pool.bab_pool(eng, [case], **kw)[0]
    check_verdict(name, pb, exact, replay)
    assert eng.graphs.captures >= 1
    assert (replay.status, replay.rounds, replay.bounded, replay.max_depth) == (
        eager.status, eager.rounds, eager.bounded, eager.max_depth)
    assert replay.history == eager.history

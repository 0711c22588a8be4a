"""Multi-rank host logic on CPU (gloo, world size 2): sharding by subdomain, no data-path
exchange, gathered bounds equal the single-process bounds, max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import sharding as S
from paper_2103_06624_gb300 import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup():
    pb = wl.problem_mlp_small()
    onet = O.OracleNet(pb.layers, pb.C)
    l, u = O.root_bounds(onet, pb.x_lo, pb.x_hi)
    unst = [np.nonzero(O.unstable_mask(l[0], u[0]))[0]]
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l, u=u)
    batch = wl.random_batch(pb, unst, 37, 0, 4, 3)
    a, b = wl.random_alpha_beta(batch, 4, 1.0)
    _, U = O.unstable_ranks(onet, l, u)
    return pb, onet, props, batch, a, b, U


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb, onet, props, batch, a, b, U = _setup()
    sb, sa, sbeta, (lo, hi) = S.shard_batch(batch, pb.K, U, rank, world, a, b)
    lb_local = O.bound(onet, props, sb, sa, sbeta)            # no collective on the path
    full = S.gather_rows(lb_local, batch.B, pb.K, dist).numpy()
    t = S.max_over_ranks(10.0 + rank, dist)
    if rank == 0:
        q.put((full, t, (lo, hi)))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_the_batch():
    for B in (0, 1, 7, 64):
        for world in (1, 2, 3, 8):
            spans = [S.shard_range(B, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == B
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [h - l for l, h in spans]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_gloo_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, t, span = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pb, onet, props, batch, a, b, U = _setup()
    ref = O.bound(onet, props, batch, a, b)
    assert np.allclose(full, ref, rtol=0, atol=1e-12)
    assert t == 11.0
    assert span == (0, 19)


def _bab_worker(rank, world, port, q, name, driver):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2103_06624_gb300 import bab
    from tests.test_bab import OracleEngine, make_case
    pb, props, unst, exact = make_case(name)
    eng = OracleEngine(pb, props, [len(u) for u in unst])
    kw = dict(device="cpu") if driver == "pool" else {}
    res = bab.bab_ranks(eng, 0, props["l"][0], props["u"][0], pb.x_lo[0], pb.x_hi[0], rank, world, dist,
                        batch_size=256, max_rounds=12, n_samples=128, driver=driver, **kw)
    q.put((rank, res.status, res.bounded, res.witness, exact))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("driver", ["list", "pool"])
@pytest.mark.parametrize("name,world", [("verified_by_branching_a", 2), ("verified_by_branching_b", 3),
                                        ("violated", 2)])
def test_bab_across_ranks_reaches_the_single_process_verdict(name, world, driver):
    """Each rank decides its share of the subdomains below the first ceil(log2 world) splits,
    with no exchange while branching; one all-reduce combines the verdicts (and the lowest
    finding rank broadcasts a witness).  Both drivers: the list pool, and the array pool whose
    start subdomains are the rank's sign patterns of the first branching neurons."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bab_worker, args=(r, world, port, q, name, driver)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    statuses = {o[1] for o in out}
    assert len(statuses) == 1                       # every rank returns the combined verdict
    status = statuses.pop()
    exact = out[0][4]
    assert status == ("violated" if name == "violated" else "verified")
    assert (status == "verified") == (exact.min() > 0)
    if status == "violated":
        from tests.test_bab import make_case
        pb = make_case(name)[0]
        for o in out:                               # the same witness on every rank, and valid
            np.testing.assert_array_equal(o[3], out[0][3])
        m = np.atleast_2d(wl.reference_forward(pb.layers, out[0][3])) @ pb.C.astype(np.float64).T
        assert m.min() < 0
    assert len({o[2] for o in out}) == 1            # the subdomain count is summed over ranks


def test_rank_shares_partition_the_first_splits():
    """The 2^k sign patterns of the first k branching neurons are split over the ranks without
    overlap or gap (k = ceil(log2 world), capped by the number of unstable neurons)."""
    from paper_2103_06624_gb300 import bab
    rng = np.random.default_rng(0)
    l = -rng.random(20)
    u = rng.random(20)
    u[3] = -0.1                                     # a stable neuron is never among the first splits
    order = list(np.argsort(-bab.branching_scores(l, u), kind="stable"))
    for world in (1, 2, 3, 4, 5, 8):
        k = int(np.ceil(np.log2(world))) if world > 1 else 0
        shares = [bab.rank_starts(l, u, r, world) for r in range(world)]
        flat = [tuple(sg.tolist()) for sh in shares for _, sg in sh]
        assert len(flat) == 1 << k and len(set(flat)) == len(flat)
        assert all(len(sh) >= 1 for sh in shares)
        for sh in shares:
            for top, _ in sh:
                assert top.tolist() == [int(n) for n in order[:k]] and 3 not in top.tolist()
    # one unstable neuron: at most 2 patterns whatever the world size; the other ranks start empty
    l1, u1 = np.array([-1.0, 0.5]), np.array([1.0, 2.0])
    shares = [bab.rank_starts(l1, u1, r, 4) for r in range(4)]
    assert sum(len(sh) for sh in shares) == 2

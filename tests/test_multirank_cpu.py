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

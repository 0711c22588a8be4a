"""Host-side sharding of a batch of subdomains across ranks (one process per GPU).

Rows (subdomain x spec) are independent given the weights and the per-property root bounds,
so a batch splits into contiguous blocks of subdomains with no exchange on the data path.
Collectives appear only around the path: the maximum of the timed region over ranks, and,
for a caller that wants every bound on every rank, an all-gather of the results.
"""
from __future__ import annotations

import numpy as np

from .workloads import Batch


def shard_range(B, rank, world):
    """Contiguous block [lo, hi) of subdomains owned by `rank` (sizes differ by at most one)."""
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_batch(batch, K, U, rank, world, alpha=None, beta=None):
    """The rank's subdomains as a self-contained Batch, with their alpha/beta slices repacked."""
    lo, hi = shard_range(batch.B, rank, world)
    idx = np.arange(lo, hi)
    U = np.asarray(U, np.int64)
    cnt = batch.split_cnt[idx].astype(np.int32)
    off = np.zeros(len(idx), np.int32)
    if len(idx) > 1:
        off[1:] = np.cumsum(cnt)[:-1]
    per = U[batch.prop_of[idx]] * K
    aoff = np.zeros(len(idx), np.int64)
    if len(idx) > 1:
        aoff[1:] = np.cumsum(per)[:-1]
    sl = [np.arange(batch.split_off[b], batch.split_off[b] + batch.split_cnt[b]) for b in idx]
    sel = np.concatenate(sl) if sl else np.zeros(0, np.int64)
    out = Batch(batch.prop_of[idx].astype(np.int32), off, cnt, batch.split_layer[sel], batch.split_idx[sel],
                batch.split_sign[sel], aoff, int(per.sum()), int(cnt.sum()) * K)
    a = b = None
    if alpha is not None:
        a = np.concatenate([alpha[batch.alpha_off[i]:batch.alpha_off[i] + per[n]] for n, i in enumerate(idx)]) \
            if len(idx) else np.zeros(0, np.float32)
    if beta is not None:
        b = np.concatenate([beta[batch.split_off[i] * K:(batch.split_off[i] + batch.split_cnt[i]) * K] for i in idx]) \
            if len(idx) else np.zeros(0, np.float32)
    return out, a, b, (lo, hi)


def max_over_ranks(value, dist=None):
    """Maximum of a float over the process group (the slowest rank sets the timed region)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local, B, K, dist):
    """All-gather per-rank row results (e.g. bounds) into the global [B*K] order."""
    import torch
    world = dist.get_world_size()
    sizes = [(shard_range(B, r, world)[1] - shard_range(B, r, world)[0]) * K for r in range(world)]
    t = torch.as_tensor(np.asarray(local))
    pad = max(sizes)
    buf = torch.zeros(pad, dtype=t.dtype, device=t.device)
    buf[:t.numel()] = t
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return torch.cat([p[:n] for p, n in zip(parts, sizes)])

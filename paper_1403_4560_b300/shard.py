"""Sharding of independent disorder samples across ranks (one GPU per rank).

Disorder samples never interact, so a run splits into per-rank shards with
no communication while it runs; every random number of sample s is keyed by
its global index (sg_options.sample_base + local index), so the shards
reproduce the unsplit run exactly. The single exchange step is a gather of the
per-sample FP64 accumulators for the disorder averages (and, when the overlap
histogram is kept, one sum of the per-rank integer histograms).
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_samples: int, world: int, rank: int, align: int = 1):
    """Contiguous [begin, end) of rank's samples; shard sizes are multiples of
    `align` (64 for the multispin-coded layout) except possibly the last."""
    if n_samples % align:
        raise ValueError("n_samples must be a multiple of align")
    units = n_samples // align
    per, extra = divmod(units, world)
    b = rank * per + min(rank, extra)
    e = b + per + (1 if rank < extra else 0)
    return b * align, e * align


def reduce_histogram(hist_local: np.ndarray, group=None) -> np.ndarray:
    """Sum of the ranks' overlap histograms uint64 [n_T][B][N+1] (all-reduce;
    counts are added as int64, exact below 2^63)."""
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.from_numpy(np.ascontiguousarray(hist_local).view(np.int64)).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().view(np.uint64)


def gather_accumulators(acc_local: np.ndarray, group=None) -> np.ndarray:
    """All-gather per-sample accumulator arrays [S_r][n_T][40] (or
    [S_r][n_T][B][40] with sweep bins) of every rank, concatenated in rank
    order (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    n = torch.tensor([acc_local.shape[0]], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    tail = acc_local.shape[1:]
    mx = max(sizes)
    buf = torch.zeros((mx,) + tail, dtype=torch.float64, device=dev)
    buf[: acc_local.shape[0]] = torch.from_numpy(np.ascontiguousarray(acc_local)).to(dev)
    outs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([o[:s].cpu().numpy() for o, s in zip(outs, sizes)], axis=0)

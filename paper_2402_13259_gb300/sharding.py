"""Replication ranges per rank, and the host-side combination of their
statistics.

Replications are independent and the random streams are keyed by the
replication index, so a run shards by giving each rank a contiguous range of
indices: the union of the ranks' results is the single-device result, with no
data-path collective.  The one exchange is at the end of a run: the station
rows and N_K add up over ranks (all-reduce) and the replication rows are
concatenated in rank order (all-gather).  Weak scaling gives every rank R replications
(indices rank*R ...); strong scaling splits R replications across ranks.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def replica_range(rank: int, world: int, R: int, scaling: str = "weak") -> Tuple[int, int]:
    """(rep_begin, replications) of `rank` out of `world`."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    if scaling == "weak":
        return rank * R, R
    if scaling == "strong":
        base, extra = divmod(R, world)
        begin = rank * base + min(rank, extra)
        return begin, base + (1 if rank < extra else 0)
    raise ValueError("scaling must be 'weak' or 'strong'")


def combine_stats(parts: Sequence[np.ndarray], n: int, Rs: Sequence[int]) -> np.ndarray:
    """Combine per-rank stats buffers (layout 6n + 4R of the C ABI) of
    consecutive replication ranges into one buffer over all replications."""
    station = np.zeros((n, 5), dtype=np.int64)
    nk = np.zeros(n, dtype=np.int64)
    reps: List[np.ndarray] = []
    for st, R in zip(parts, Rs):
        st = np.asarray(st, dtype=np.int64)
        station += st[: 5 * n].reshape(n, 5)
        reps.append(st[5 * n: 5 * n + 4 * R])
        nk += st[5 * n + 4 * R: 6 * n + 4 * R]
    return np.concatenate([station.ravel(), *reps, nk])


def combine_stats_dist(stats, n: int, counts: Sequence[int], group=None):
    """The same combination as `combine_stats` with torch.distributed
    collectives (gloo on CPU tensors, NCCL on device tensors): `stats` is this
    rank's int64 buffer over its `counts[rank]` replications; every rank gets
    the buffer over all replications, ranks' ranges in rank order."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    if len(counts) != world:
        raise ValueError("one replication count per rank")
    Rk = int(counts[rank])
    if stats.numel() != 6 * n + 4 * Rk or stats.dtype != torch.int64:
        raise ValueError("stats must be int64 of length 6n + 4R")
    head = torch.cat([stats[: 5 * n], stats[5 * n + 4 * Rk:]])  # station rows, N_K
    dist.all_reduce(head, op=dist.ReduceOp.SUM, group=group)
    Rmax = max(int(c) for c in counts)
    rep = torch.zeros(4 * Rmax, dtype=torch.int64, device=stats.device)
    rep[: 4 * Rk] = stats[5 * n: 5 * n + 4 * Rk]
    parts = [torch.empty_like(rep) for _ in range(world)]
    dist.all_gather(parts, rep, group=group)
    reps = [p[: 4 * int(c)] for p, c in zip(parts, counts)]
    return torch.cat([head[: 5 * n], *reps, head[5 * n:]])

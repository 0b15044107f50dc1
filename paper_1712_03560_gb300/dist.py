"""Multi-GPU plan for the dictionary scan: one process per GPU.

Patterns are independent (MOASM runs one filter per pattern, Sec. 6.4), so a
dictionary shards by pattern with no exchange on the data path: every rank
scans the full text with its share of the patterns, and only the final hit
lists are gathered.  Shares are balanced by bit-vector word count (the scan's
work is proportional to the sum over patterns of ceil(l_p / 32)).  Streams
(serving) shard the same way by stream id.

These helpers are host logic; they run under ``torch.distributed`` with any
backend (NCCL on GPUs, gloo on CPU for the tests).
"""
from __future__ import annotations

import numpy as np


def shard_patterns(lengths, world: int, unit: int = 32) -> list:
    """Pattern ids per rank, greedily balanced by ceil(l_p / unit) (longest
    first, each to the least loaded rank); ids stay sorted.  unit = 32: the
    bit-parallel scan's words; unit = 4: the weighted path's lanes of 4 rows."""
    lengths = np.asarray(lengths, dtype=np.int64)
    words = (lengths + unit - 1) // unit
    order = np.argsort(-words, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    parts = [[] for _ in range(world)]
    for p in order.tolist():
        r = int(np.argmin(load))
        parts[r].append(p)
        load[r] += int(words[p])
    return [sorted(x) for x in parts]


def remap(hits: np.ndarray, ids, field: str = "pattern_id") -> np.ndarray:
    """Local pattern ids of a shard -> global ids."""
    out = hits.copy()
    out[field] = np.asarray(ids, dtype=np.int64)[hits[field].astype(np.int64)]
    return out


def gather_hits(local: np.ndarray, ids, group=None, field: str = "pattern_id") -> np.ndarray:
    """All ranks' hits with global pattern ids, sorted by (pattern, decided_at, k)."""
    import torch.distributed as dist
    mine = remap(local, ids, field)
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, mine, group=group)
    allh = np.concatenate(parts) if parts else mine
    order = np.lexsort((allh["k"], allh["decided_at"], allh[field]))
    return allh[order]


def max_over_ranks(x: float, device=None) -> float:
    """The slowest rank's value (the job's time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Multi-process (world size 2, gloo, CPU) checks of the sharding plan: each
rank runs the CPU oracle on its pattern share, the hit lists are gathered,
and the result equals the single-process result; max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest

from paper_1712_03560_gb300 import dist as D
from paper_1712_03560_gb300 import workloads as W


def test_shards_cover_every_pattern_once_and_balance_words():
    rng = np.random.default_rng(0)
    lens = rng.integers(1, 129, size=1000)
    for world in (1, 2, 3, 8):
        parts = D.shard_patterns(lens, world)
        flat = sorted(p for part in parts for p in part)
        assert flat == list(range(1000))
        words = [int(((lens[part] + 31) // 32).sum()) for part in parts]
        assert max(words) - min(words) <= 4


def test_weighted_shards_balance_lanes():
    """The weighted path's work is a lane of 4 rows per started 4 symbols."""
    rng = np.random.default_rng(1)
    lens = rng.integers(1, 129, size=777)
    for world in (2, 3, 8):
        parts = D.shard_patterns(lens, world, unit=4)
        assert sorted(p for part in parts for p in part) == list(range(777))
        lanes = [int(((lens[part] + 3) // 4).sum()) for part in parts]
        assert max(lanes) - min(lanes) <= 32


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.dictionary_dna(seed=11, n=60_000, n_pat=23, copies=8)
        ids = D.shard_patterns([p.size for p in wl.patterns], world)[rank]
        local = oracle.oasm_dictionary([wl.patterns[i] for i in ids], [wl.ks[i] for i in ids],
                                       wl.texts[0], threads=1)
        got = D.gather_hits(local, ids)
        slow = D.max_over_ranks(float(rank + 1))
        if rank == 0:
            full = oracle.oasm_dictionary(wl.patterns, wl.ks, wl.texts[0], threads=2)
            same = [tuple(r) for r in got[["pattern_id", "decided_at", "k", "start", "len"]].tolist()] == \
                   [tuple(r) for r in full[["pattern_id", "decided_at", "k", "start", "len"]].tolist()]
            q.put((same, len(full), slow))
    finally:
        dist.destroy_process_group()


def test_pattern_sharding_with_two_gloo_ranks_equals_one_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    same, n, slow = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert same and n > 0
    assert slow == 2.0

"""The two ways the filtered output reaches canonical order
(`oasm_config.record_order`): 1, each piece of a pair's sorted hits writes
its records at a position fixed by its place among the hits and a scan of
the counts gives the offsets; 2, records are appended as decided and then
sorted.  Both must give the oracle's records, in canonical order (pattern_id,
decided_at, k) per stream, across steps (windows carried from one step to the
next, decided by a later step with or without new hits), under every rule
set, and when the output outgrows its buffers (a re-run)."""
import numpy as np
import pytest

import oracle
from paper_1712_03560_gb300 import binding as B
from paper_1712_03560_gb300 import workloads as W
from parity_util import RULE_NAMES, canon, oracle_rows, random_case, run_gpu

pytestmark = pytest.mark.gpu

ORDERS = [1, 2]


def rows_of(res):
    return [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
             int(r["len"])) for r in res]


def in_canonical_order(rows):
    keys = [(p, d, k) for (p, d, k, _s, _l) in rows]
    return keys == sorted(keys)


RULE_SETS = [dict(replace=r, order=o, acc=a, cmp=c)
             for r in ("contained", "same_end", "never")
             for o in ("per_start_length", "per_start_best")
             for a in ("sum", "last")
             for c in ("gt", "ge")]


@pytest.mark.parametrize("ro", ORDERS)
@pytest.mark.parametrize("ri", range(0, len(RULE_SETS), 5))
def test_rule_sets_with_splits(ro, ri):
    """Several steps per stream (a flush after each piece): pending windows
    carry over and are decided by the next step's first piece."""
    rng = np.random.default_rng(900 + ri)
    pats, ks, text = random_case(rng, 3, 14, 3, 24, 9000, kmax=5)
    splits = np.sort(rng.integers(0, text.size + 1, size=12))
    rows, _ = run_gpu(pats, ks, text, RULE_SETS[ri], splits=splits,
                      cfg={"record_order": ro})
    assert canon(rows) == oracle_rows(pats, ks, text, RULE_SETS[ri])


@pytest.mark.parametrize("ro", ORDERS)
def test_windows_decided_by_a_step_without_hits(ro):
    """A stream ends a step with a pending window and the next step brings no
    new hit for that pattern: the window is decided from the carried state
    alone (for the ordered records, in the pair's reserved head slots)."""
    rng = np.random.default_rng(911)
    pats = [np.frombuffer(b"GATTACAGATTACA", np.uint8), np.frombuffer(b"CCGGAATTCCGG", np.uint8)]
    ks = [3, 2]
    filler = np.frombuffer(b"T" * 4000, np.uint8).copy()
    streams = []
    for i in range(5):
        a = W.iid_dna(rng, 3000)
        W.plant(rng, a, W.edit_copy(rng, pats[i % 2], 1, W.DNA))
        a[-20:-6] = pats[0]  # a window still open at the end of the first piece
        streams.append((a, filler[: 500 + 300 * i]))
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 8, "record_order": ro})
    try:
        sids = [B.oasm_open_stream(ctx) for _ in streams]
        for s, (a, _b) in zip(sids, streams):
            B.oasm_feed(ctx, s, a)
        B.oasm_step(ctx)
        for s, (_a, b) in zip(sids, streams):
            B.oasm_feed(ctx, s, b)
        B.oasm_step(ctx)
        got = {s: rows_of(B.oasm_flush(ctx, s)) for s in sids}
        for s in sids:
            B.oasm_end_stream(ctx, s)
        B.oasm_step(ctx)
        for s in sids:
            got[s] += rows_of(B.oasm_flush(ctx, s))
    finally:
        B.oasm_destroy(ctx)
    quiet = 0
    for s, (a, b) in zip(sids, streams):
        text = np.concatenate([a, b])
        want = oracle_rows(pats, ks, text)
        assert any(r[0] == 0 and r[3] >= a.size - 20 for r in want)
        assert in_canonical_order(got[s])
        assert canon(got[s]) == want, s
        # the setup: pattern 0's window is still open after the first step
        # (a hit given to it ends past the last start it could decide) ...
        h = oracle.hits(pats[0], ks[0], text)
        f1 = a.size - pats[0].size - ks[0]
        given = h["start"] <= f1
        assert (h["start"][given] + h["len"][given] - 1).max() > f1
        # ... and, in most streams, the second step has no hit of it at all
        quiet += int(not ((h["start"] > f1) & (h["start"] <= text.size - 1)).any())
    assert quiet >= 3


@pytest.mark.parametrize("ro", ORDERS)
def test_interleaved_streams_canonical_without_sorting(ro):
    """Nine streams fed in random pieces over many steps; each flush is in
    canonical order as returned and equals the oracle."""
    rng = np.random.default_rng(913)
    pats, ks, _ = random_case(rng, 4, 40, 6, 40, 10, kmax=4)
    texts = [random_case(rng, 4, 1, 6, 8, int(rng.integers(0, 12000)))[2] for _ in range(9)]
    for t in texts:
        for p, k in zip(pats[:8], ks[:8]):
            if t.size > 100:
                W.plant(rng, t, W.edit_copy(rng, p, k, W.DNA))
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 16, "record_order": ro})
    try:
        sids = [B.oasm_open_stream(ctx) for _ in texts]
        pos = [0] * len(texts)
        got = {s: [] for s in sids}
        while any(p < t.size for p, t in zip(pos, texts)):
            for i, (s, t) in enumerate(zip(sids, texts)):
                if pos[i] < t.size:
                    n = int(rng.integers(1, 3000))
                    B.oasm_feed(ctx, s, t[pos[i]:pos[i] + n])
                    pos[i] += n
            B.oasm_step(ctx)
            for s in sids:
                part = rows_of(B.oasm_flush(ctx, s))
                assert in_canonical_order(part)
                got[s] += part
        for s in sids:
            B.oasm_end_stream(ctx, s)
        B.oasm_step(ctx)
        for s in sids:
            got[s] += rows_of(B.oasm_flush(ctx, s))
    finally:
        B.oasm_destroy(ctx)
    for s, t in zip(sids, texts):
        assert canon(got[s]) == oracle_rows(pats, ks, t), s


@pytest.mark.parametrize("ro", ORDERS)
def test_output_outgrows_its_buffers(ro):
    """m = 8, K = 2 over 8 M random DNA symbols fed in three pieces: the first
    step (7 MiB) yields about 80,000 kept records and more hits than the
    first buffers hold, so it re-runs with larger ones, and the later steps
    continue from the windows it left; the whole output against the
    oracle."""
    rng = np.random.default_rng(917)
    pat = W.iid_dna(rng, 8)
    text = W.iid_dna(rng, 8 << 20)
    rows, st = run_gpu([pat], [2], text, splits=[7 << 20, (7 << 20) + 12345],
                       cfg={"record_order": ro})
    assert st["reruns"] >= 1
    assert len(rows) > 65536
    assert in_canonical_order(rows)
    assert canon(rows) == oracle_rows([pat], [2], text)


def test_both_orders_equal_on_a_dictionary():
    """The 1,024-pattern DNA dictionary shape on 4 MiB: both paths return the
    same records in the same order."""
    rng = np.random.default_rng(919)
    pats, ks, text = random_case(rng, 4, 300, 8, 32, 4 << 20, kmax=3)
    a, _ = run_gpu(pats, ks, text, cfg={"record_order": 1})
    b, _ = run_gpu(pats, ks, text, cfg={"record_order": 2})
    assert len(a) > 1000
    assert a == b


@pytest.mark.parametrize("ro", ORDERS)
def test_split_steps_overlap_the_record_copy(ro):
    """The pipelined pattern of bench.py: while step i runs on the device the
    host drains and closes step i - 1's streams (whose records are still being
    copied to the host) and opens and feeds step i + 1's.  Four steps of three
    fresh streams each; every stream's records against the oracle, in
    canonical order as drained."""
    rng = np.random.default_rng(931)
    pats, ks, _ = random_case(rng, 4, 30, 6, 40, 10, kmax=3)
    sets = []
    for i in range(4):
        texts = []
        for j in range(3):
            t = W.iid_dna(rng, 15000 + 4000 * j + 1000 * i)
            for p, k in zip(pats[:10], ks[:10]):
                W.plant(rng, t, W.edit_copy(rng, p, k, W.DNA))
            texts.append(t)
        sets.append(texts)
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 8, "record_order": ro})
    got = {}

    def open_feed(i):
        sids = []
        for t in sets[i]:
            s = B.oasm_open_stream(ctx)
            B.oasm_feed(ctx, s, t)
            B.oasm_end_stream(ctx, s)
            sids.append(s)
        return sids

    def drain_close(i, sids):
        out = B.oasm_drain(ctx)
        col = [int(r["stream_id"]) for r in out]
        assert col == sorted(col)
        for j, s in enumerate(sids):
            mine = rows_of(out[np.array(col, dtype=np.int64) == s])
            assert in_canonical_order(mine)
            got[(i, j)] = mine
        for s in sids:
            B.oasm_close_stream(ctx, s)

    try:
        cur, prev = open_feed(0), None
        for i in range(4):
            B.oasm_step_begin(ctx)
            if prev is not None:
                drain_close(i - 1, prev)
            nxt = open_feed(i + 1) if i + 1 < 4 else None
            B.oasm_step_end(ctx)
            prev, cur = cur, nxt
        drain_close(3, prev)
    finally:
        B.oasm_destroy(ctx)
    for i in range(4):
        for j in range(3):
            assert canon(got[(i, j)]) == oracle_rows(pats, ks, sets[i][j]), (i, j)

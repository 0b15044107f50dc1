"""Emission order of the decided hits, as the ABI promises it: oasm_flush
returns a stream's hits in canonical order (pattern_id, decided_at, k; for
the raw all-hits output, ties by length), also when several steps queued
them and a small cap splits the output over several calls; oasm_drain gives
streams in id order, each in canonical order.  Each case runs with the records
written in order by the filter and with the record sort
(oasm_config.record_order 1 and 2).  The GPU rows are checked in
the order they arrive, without sorting, and as a multiset against the
oracle."""
import ctypes

import numpy as np
import pytest

from paper_1712_03560_gb300 import binding as B
from parity_util import oracle_rows, random_case

pytestmark = pytest.mark.gpu


def as_rows(res):
    return [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["len"]),
             int(r["start"])) for r in res]


def canonical(rows):
    return sorted(rows, key=lambda x: (x[0], x[1], x[2], x[3]))


def to_oracle_order(rows):
    return sorted((p, d, k, s, ln) for (p, d, k, ln, s) in rows)


@pytest.mark.parametrize("ro", [1, 2])
@pytest.mark.parametrize("output", ["filtered", "ends", "all_hits"])
def test_flush_is_canonical_after_several_steps(output, ro):
    """A stream fed in six pieces with a step after each: the queue holds one
    sorted run per step; the flush at the end returns their merge."""
    rng = np.random.default_rng(801)
    pats, ks, text = random_case(rng, 4, 48, 6, 40, 60000, kmax=4)
    rules = None if output == "filtered" else {"output": output}
    ctx = B.oasm_create(pats, ks, rules, {"record_order": ro})
    try:
        sid = B.oasm_open_stream(ctx)
        for piece in np.split(text, [7000, 19000, 19001, 33000, 47000]):
            B.oasm_feed(ctx, sid, piece)
            B.oasm_step(ctx)
        res = B.oasm_flush(ctx, sid, end_of_stream=True)
    finally:
        B.oasm_destroy(ctx)
    got = as_rows(res)
    assert len(got) > 100
    assert got == canonical(got)
    mode = {"filtered": "oasm", "ends": "ends", "all_hits": "hits"}[output]
    assert to_oracle_order(got) == oracle_rows(pats, ks, text, mode=mode)


@pytest.mark.parametrize("ro", [1, 2])
def test_flush_with_small_cap_continues_in_canonical_order(ro):
    """OASM_ETRUNC hands out the first cap records; the next calls continue
    where it stopped, and the concatenation is the canonical sequence."""
    rng = np.random.default_rng(802)
    pats, ks, text = random_case(rng, 4, 40, 6, 30, 40000, kmax=3)
    lib = B.load()
    ctx = B.oasm_create(pats, ks, None, {"record_order": ro})
    parts = []
    try:
        sid = B.oasm_open_stream(ctx)
        for piece in np.split(text, [13000, 26000]):
            B.oasm_feed(ctx, sid, piece)
            B.oasm_step(ctx)
        B.oasm_end_stream(ctx, sid)
        B.oasm_step(ctx)
        cap = 97
        buf = np.zeros(cap, dtype=B.HIT_DTYPE)
        n = ctypes.c_size_t(0)
        while True:
            rc = lib.oasm_flush(ctx, sid, 0, buf.ctypes.data, cap, ctypes.byref(n))
            assert rc in (B.OASM_OK, B.OASM_ETRUNC)
            parts.append(buf[: n.value].copy())
            if rc == B.OASM_OK:
                break
            assert n.value == cap
    finally:
        B.oasm_destroy(ctx)
    got = as_rows(np.concatenate(parts))
    assert len(parts) > 3
    assert got == canonical(got)
    assert to_oracle_order(got) == oracle_rows(pats, ks, text)


@pytest.mark.parametrize("ro", [1, 2])
def test_drain_gives_streams_in_id_order_each_canonical(ro):
    """Three interleaved streams with steps between their feeds; one drain."""
    rng = np.random.default_rng(803)
    pats, ks, _ = random_case(rng, 4, 36, 6, 30, 10, kmax=3)
    texts = [random_case(rng, 4, 1, 6, 6, n, kmax=0)[2] for n in (30000, 18000, 25000)]
    ctx = B.oasm_create(pats, ks, None, {"record_order": ro})
    try:
        sids = [B.oasm_open_stream(ctx) for _ in texts]
        for a, b in ((0, 6000), (6000, 15000), (15000, 30000)):
            for s, t in zip(sids, texts):
                B.oasm_feed(ctx, s, t[a:b])
            B.oasm_step(ctx)
        for s in sids:
            B.oasm_end_stream(ctx, s)
        B.oasm_step(ctx)
        res = B.oasm_drain(ctx)
    finally:
        B.oasm_destroy(ctx)
    sid_col = [int(r["stream_id"]) for r in res]
    assert sid_col == sorted(sid_col)
    for s, t in zip(sids, texts):
        mine = as_rows(res[np.array(sid_col) == s])
        assert mine == canonical(mine)
        assert to_oracle_order(mine) == oracle_rows(pats, ks, t)

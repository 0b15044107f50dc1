"""Parity at the full workload sizes, in the launch configuration bench.py
times (one context per workload, autotuned on a 32 MiB slice): the GPU runs
every pattern over the whole input, and the CPU oracle computes a sample of
the outputs one by one -- a few patterns over the whole text, a few whole
texts or streams, or, where one pattern over the whole text is too slow for
the oracle, every decision a text prefix already fixes.  Sampled outputs must
match exactly."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_03560_gb300 import binding as B
from paper_1712_03560_gb300 import serve
from paper_1712_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rows(res, keep=None):
    out = []
    for r in res:
        p = int(r["pattern_id"])
        if keep is None or p in keep:
            out.append((p, int(r["decided_at"]), int(r["k"]), int(r["start"]), int(r["len"])))
    return sorted(out)


def oracle_sample(wl_patterns, wl_ks, idx, text, costs=None):
    res = oracle.oasm_dictionary([wl_patterns[i] for i in idx], [int(wl_ks[i]) for i in idx],
                                 text, threads=min(len(idx), os.cpu_count() or 1), costs=costs)
    return sorted((int(idx[int(r["pattern_id"])]), int(r["decided_at"]), int(r["k"]),
                   int(r["start"]), int(r["len"])) for r in res)


def tuned_context(wl, costs=None):
    import torch
    ctx = B.oasm_create(wl.patterns, wl.ks, None, {"max_streams": max(64, len(wl.texts))},
                        costs=costs)
    big = max(wl.texts, key=lambda t: t.size)
    sample = torch.from_numpy(big[: min(big.size, 32 << 20)].copy()).cuda()
    B.oasm_autotune(ctx, sample)
    return ctx


def search_one(ctx, dtext):
    sid = B.oasm_open_stream(ctx)
    B.oasm_feed_device(ctx, sid, dtext)
    res = B.oasm_flush(ctx, sid, end_of_stream=True)
    B.oasm_close_stream(ctx, sid)
    return res


def test_dictionary_dna_full_size():
    """1,024 DNA patterns over the whole 256 MiB text; 6 patterns checked."""
    import torch
    wl = W.dictionary_dna()
    ctx = tuned_context(wl)
    try:
        res = search_one(ctx, torch.from_numpy(wl.texts[0]).cuda())
    finally:
        B.oasm_destroy(ctx)
    idx = [0, 204, 409, 614, 819, 1023]
    want = oracle_sample(wl.patterns, wl.ks, idx, wl.texts[0])
    assert len(want) > 0
    assert rows(res, set(idx)) == want


def test_dictionary_dna_weighted_full_size():
    """The weighted path (edit costs 1, 2, 2) on the 1,024-pattern, 256 MiB
    DNA dictionary; 6 patterns checked over the whole text."""
    import torch
    wl = W.dictionary_dna()
    costs = (1, 2, 2)
    ctx = tuned_context(wl, costs)
    try:
        res = search_one(ctx, torch.from_numpy(wl.texts[0]).cuda())
    finally:
        B.oasm_destroy(ctx)
    idx = [3, 200, 411, 618, 822, 1020]
    want = oracle_sample(wl.patterns, wl.ks, idx, wl.texts[0], costs)
    assert len(want) > 0
    assert rows(res, set(idx)) == want


def test_bytes_zipf_full_size_prefix_decisions():
    """4,096 byte patterns over the whole 1 GiB text; for 4 patterns every
    decision the first 16 MiB fix (decided_at + m + K <= 16 MiB) is checked."""
    import torch
    wl = W.bytes_zipf()
    ctx = tuned_context(wl)
    try:
        res = search_one(ctx, torch.from_numpy(wl.texts[0]).cuda())
    finally:
        B.oasm_destroy(ctx)
    P = 16 << 20
    idx = [7, 1500, 2900, 4090]
    lim = {i: P - wl.patterns[i].size - int(wl.ks[i]) for i in idx}
    got = [r for r in rows(res, set(idx)) if r[1] <= lim[r[0]]]
    want = [r for r in oracle_sample(wl.patterns, wl.ks, idx, wl.texts[0][:P]) if r[1] <= lim[r[0]]]
    assert len(want) > 0
    assert got == want


def test_many_texts_full_size_sampled_texts():
    """10,000 DNA texts (~4 GB) x 512 patterns in one step; 5 whole texts
    checked against the oracle with every pattern."""
    import torch
    wl = W.many_texts()
    ctx = tuned_context(wl)
    try:
        dts = [torch.from_numpy(t).cuda() for t in wl.texts]
        sids = []
        for t in dts:
            s = B.oasm_open_stream(ctx)
            B.oasm_feed_device(ctx, s, t)
            B.oasm_end_stream(ctx, s)
            sids.append(s)
        B.oasm_step(ctx)
        picks = [i for i in range(len(wl.texts)) if 2000 <= wl.texts[i].size <= 150_000][:5]
        got = {i: rows(B.oasm_flush(ctx, sids[i])) for i in picks}
    finally:
        B.oasm_destroy(ctx)
    for i in picks:
        want = oracle_sample(wl.patterns, wl.ks, list(range(len(wl.patterns))), wl.texts[i])
        assert got[i] == want, i


def test_served_full_config_sampled_streams():
    """4,096 streams x 2,000 signatures, 20,000 packets through the serving
    loop; 6 whole streams checked against the oracle."""
    tr = W.served(n_packets=20000, gbps=1.0)
    with serve.Server(tr.patterns, tr.ks, max_streams=4096) as srv:
        res = srv.replay(tr, realtime=False, collect=True)
    texts = tr.stream_texts()
    picks = [e for e in range(tr.n_streams) if texts[e].size > 0][:6]
    for e in picks:
        got = res["hits"].get(e)
        got = [] if got is None else rows(got)
        want = oracle_sample(tr.patterns, tr.ks, list(range(len(tr.patterns))), texts[e])
        assert got == want, e

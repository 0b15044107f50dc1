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


_ZIPF = {}


def bytes_zipf_searched():
    """The 4,096-pattern, 1 GiB Zipf workload and its whole GPU output (one
    step over the whole text, autotuned context), computed once per run."""
    if not _ZIPF:
        import torch
        wl = W.bytes_zipf()
        ctx = tuned_context(wl)
        try:
            res = search_one(ctx, torch.from_numpy(wl.texts[0]).cuda())
        finally:
            B.oasm_destroy(ctx)
        _ZIPF["wl"], _ZIPF["rows"] = wl, rows(res)
    return _ZIPF["wl"], _ZIPF["rows"]


def test_bytes_zipf_full_size_prefix_decisions():
    """4,096 byte patterns over the whole 1 GiB text; for 4 patterns every
    decision the first 16 MiB fix (decided_at + m + K <= 16 MiB) is checked."""
    wl, allrows = bytes_zipf_searched()
    P = 16 << 20
    idx = [7, 1500, 2900, 4090]
    lim = {i: P - wl.patterns[i].size - int(wl.ks[i]) for i in idx}
    got = [r for r in allrows if r[0] in lim and r[1] <= lim[r[0]]]
    want = [r for r in oracle_sample(wl.patterns, wl.ks, idx, wl.texts[0][:P]) if r[1] <= lim[r[0]]]
    assert len(want) > 0
    assert got == want


def zipf_class_picks(wl):
    """One pattern per (word count, K) pair the workload holds: every class of
    the scan (the automaton classes for K <= 2 and the Myers scan of one word,
    the cut-off scan of two to four words) and every threshold."""
    seen = {}
    for i, (p, k) in enumerate(zip(wl.patterns, wl.ks)):
        seen.setdefault(((p.size + 31) // 32, int(k)), i)
    return sorted(seen.values())


def test_bytes_zipf_full_size_every_class_and_threshold():
    """One pattern of every (word count, K) pair: every decision the first 64
    MiB fix, and every decision in three 4 MiB windows deep in the 1 GiB text
    (past thousands of region boundaries of the step).  A window starts at a
    position x0 that the oracle shows quiescent for the pattern: no hit starts
    in the 2 (K + 1)(l_p + K) symbols before x0, twice the delay bound, so no
    decision window is pending there and the oracle run from x0 on makes the
    same decisions as the run over the whole text."""
    wl, allrows = bytes_zipf_searched()
    text = wl.texts[0]
    idx = zipf_class_picks(wl)
    assert len(idx) >= 25
    P = 64 << 20
    lim = {i: P - wl.patterns[i].size - int(wl.ks[i]) for i in idx}
    got = [r for r in allrows if r[0] in lim and r[1] <= lim[r[0]]]
    want = [r for r in oracle_sample(wl.patterns, wl.ks, idx, text[:P]) if r[1] <= lim[r[0]]]
    assert len(want) > 0
    assert got == want
    S = 4 << 20

    def window(job):
        i, x0 = job
        p, K = wl.patterns[i], int(wl.ks[i])
        L = 2 * (K + 1) * (p.size + K)
        for x in (x0, x0 + (1 << 20)):
            h = oracle.hits(p, K, text[x - L:x + p.size + K])
            if (h["start"] < L).any():  # a hit starts in [x - L, x): not quiescent
                continue
            hi = x + S - p.size - K
            ref = [(i, int(r["decided_at"]) + x, int(r["k"]), int(r["start"]) + x,
                    int(r["len"])) for r in oracle.oasm(p, K, text[x:x + S])
                   if int(r["decided_at"]) + x <= hi]
            return i, x, hi, sorted(ref)
        return None

    from concurrent.futures import ThreadPoolExecutor
    jobs = [(i, x0) for i in idx for x0 in (300 << 20, 700 << 20, text.size - S - (2 << 20))]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        done = [d for d in ex.map(window, jobs) if d is not None]
    assert len(done) >= 2 * len(idx)
    by_pat = {i: [] for i in idx}
    for r in allrows:
        if r[0] in by_pat:
            by_pat[r[0]].append(r)
    for i, x, hi, ref in done:
        mine = [r for r in by_pat[i] if x <= r[1] <= hi]
        assert mine == ref, (i, x)


_MANY = {}


def many_texts_searched():
    """The 10,000-text workload in one step (autotuned context); the outputs
    of five mid-sized texts and of the three longest, computed once per run."""
    if not _MANY:
        import torch
        wl = W.many_texts()
        ctx = tuned_context(wl)
        order = sorted(range(len(wl.texts)), key=lambda i: -wl.texts[i].size)
        mid = [i for i in range(len(wl.texts)) if 2000 <= wl.texts[i].size <= 150_000][:5]
        longest = order[:3]
        try:
            dts = [torch.from_numpy(t).cuda() for t in wl.texts]
            sids = []
            for t in dts:
                s = B.oasm_open_stream(ctx)
                B.oasm_feed_device(ctx, s, t)
                B.oasm_end_stream(ctx, s)
                sids.append(s)
            B.oasm_step(ctx)
            got = {i: rows(B.oasm_flush(ctx, sids[i])) for i in mid + longest}
        finally:
            B.oasm_destroy(ctx)
        _MANY.update(wl=wl, mid=mid, longest=longest, got=got)
    return _MANY


def test_many_texts_full_size_sampled_texts():
    """10,000 DNA texts (~4 GB) x 512 patterns in one step; 5 whole texts
    checked against the oracle with every pattern."""
    M = many_texts_searched()
    wl = M["wl"]
    for i in M["mid"]:
        want = oracle_sample(wl.patterns, wl.ks, list(range(len(wl.patterns))), wl.texts[i])
        assert M["got"][i] == want, i


def test_many_texts_full_size_largest_texts():
    """The three longest texts of the 10,000 (the clipped log-normal tail,
    up to 10 MB, each spanning many scan regions), every pattern, against
    the oracle."""
    M = many_texts_searched()
    wl = M["wl"]
    assert wl.texts[M["longest"][-1]].size >= 1_000_000
    for i in M["longest"]:
        want = oracle_sample(wl.patterns, wl.ks, list(range(len(wl.patterns))), wl.texts[i])
        assert len(want) > 0
        assert M["got"][i] == want, i


def test_served_overload_split_steps_sampled_streams():
    """The native serving loop at 150 Gbit/s offered (beyond its sustained
    rate): steps of up to 32 MiB, each launched while the previous one's hits
    are handed out (split steps).  Eight whole streams against the oracle."""
    tr = W.served(seed=77, n_packets=120_000, gbps=150.0)
    with serve.Server(tr.patterns, tr.ks, max_streams=4096, prefilter_piece=1,
                      max_batch_bytes=32 << 20) as srv:
        res = srv.replay(tr, realtime=True, collect=True, engine="native")
    assert res["steps"] >= 2
    texts = tr.stream_texts()
    sizes = np.array([t.size for t in texts])
    picks = [int(e) for e in np.argsort(-sizes)[:4]] + \
        [e for e in range(tr.n_streams) if 0 < texts[e].size][:4]
    for e in picks:
        got = res["hits"].get(e)
        got = [] if got is None else rows(got)
        want = oracle_sample(tr.patterns, tr.ks, list(range(len(tr.patterns))), texts[e])
        assert got == want, e


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

"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element -- pattern id, start, length, k and decision point must
all agree exactly (integer work, no tolerance)."""
import numpy as np
import pytest

import oracle
from paper_1712_03560_gb300 import binding as B
from paper_1712_03560_gb300 import workloads as W
from parity_util import canon, oracle_rows, random_case, run_gpu

pytestmark = pytest.mark.gpu

RULE_SETS = [dict(replace=r, order=o, acc=a, cmp=c)
             for r in ("contained", "same_end", "never")
             for o in ("per_start_length", "per_start_best")
             for a in ("sum", "last")
             for c in ("gt", "ge")]


def test_worked_example_on_gpu():
    rows, _ = run_gpu([b"ACBDA"], [2], np.frombuffer(b"CCCCDACCBDACBDAA", np.uint8))
    assert canon(rows) == canon([(0, 14, 0, 10, 5), (0, 14, 2, 3, 3)])


def test_plain_dna_full_size():
    """m=8, K=2, 1e6 symbols with 200 planted copies: whole output."""
    wl = W.plain_dna()
    rows, st = run_gpu(wl.patterns, wl.ks, wl.texts[0])
    want = oracle_rows(wl.patterns, wl.ks, wl.texts[0])
    assert len(want) > 200
    assert canon(rows) == want
    assert st["scan_launches"] >= 1


@pytest.mark.parametrize("seed", range(6))
def test_random_dictionaries_default_rules(seed):
    rng = np.random.default_rng(seed)
    for sigma, npat, mlo, mhi, n in [(4, 40, 4, 32, 20000), (2, 7, 2, 12, 5000),
                                     (256, 70, 16, 128, 30000), (4, 33, 30, 70, 8000),
                                     (3, 5, 1, 6, 3000)]:
        pats, ks, text = random_case(rng, sigma, npat, mlo, mhi, n, kmax=8)
        rows, _ = run_gpu(pats, ks, text)
        assert canon(rows) == oracle_rows(pats, ks, text), (sigma, npat)


@pytest.mark.parametrize("ri", range(len(RULE_SETS)))
def test_every_rule_set(ri):
    rules = RULE_SETS[ri]
    rng = np.random.default_rng(100 + ri)
    pats, ks, text = random_case(rng, 3, 12, 3, 20, 6000, kmax=4)
    rows, _ = run_gpu(pats, ks, text, rules)
    assert canon(rows) == oracle_rows(pats, ks, text, rules)


@pytest.mark.parametrize("seed", range(4))
def test_chunk_invariance(seed):
    """Output does not depend on how the stream is cut into feeds."""
    rng = np.random.default_rng(200 + seed)
    pats, ks, text = random_case(rng, 4, 20, 4, 40, 12000, kmax=4)
    want = oracle_rows(pats, ks, text)
    for trial in range(3):
        nsplit = int(rng.integers(1, 30))
        splits = np.sort(rng.integers(0, text.size + 1, size=nsplit))
        rows, _ = run_gpu(pats, ks, text, splits=splits)
        assert canon(rows) == want, splits
    # one symbol at a time over a short prefix
    short = text[:400]
    rows, _ = run_gpu(pats, ks, short, splits=np.arange(1, short.size))
    assert canon(rows) == oracle_rows(pats, ks, short)


def test_partial_flush_returns_only_decided_hits():
    """Hits returned before the end are final: a later flush never revises them."""
    rng = np.random.default_rng(7)
    pats, ks, text = random_case(rng, 4, 8, 6, 20, 20000, kmax=3)
    want = oracle_rows(pats, ks, text)
    ctx = B.oasm_create(pats, ks)
    try:
        sid = B.oasm_open_stream(ctx)
        got = []
        for a in range(0, text.size, 3001):
            B.oasm_feed(ctx, sid, text[a:a + 3001])
            part = B.oasm_flush(ctx, sid)
            fed = min(text.size, a + 3001)
            for r in part:  # nothing decided beyond what the fed text fixes
                p = int(r["pattern_id"])
                assert int(r["decided_at"]) + len(pats[p]) + ks[p] <= fed
            got += [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                     int(r["len"])) for r in part]
        got += [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                 int(r["len"])) for r in B.oasm_flush(ctx, sid, end_of_stream=True)]
        assert canon(got) == want
    finally:
        B.oasm_destroy(ctx)


def test_many_streams_alone_and_in_the_mix():
    """Each stream's result is the same alone and interleaved with others."""
    rng = np.random.default_rng(11)
    pats, ks, _ = random_case(rng, 4, 24, 6, 40, 10, kmax=4)
    texts = [random_case(rng, 4, 1, 6, 8, int(rng.integers(0, 9000)))[2] for _ in range(9)]
    for t in texts:  # plant a few pattern copies into every text
        for p, k in zip(pats[:5], ks[:5]):
            if t.size > 100:
                W.plant(rng, t, W.edit_copy(rng, p, k, W.DNA))
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 16})
    try:
        sids = [B.oasm_open_stream(ctx) for _ in texts]
        pos = [0] * len(texts)
        got = {s: [] for s in sids}
        while any(p < t.size for p, t in zip(pos, texts)):
            for i, (s, t) in enumerate(zip(sids, texts)):
                if pos[i] < t.size:
                    n = int(rng.integers(1, 2500))
                    B.oasm_feed(ctx, s, t[pos[i]:pos[i] + n])
                    pos[i] += n
            B.oasm_step(ctx)
        for s in sids:
            B.oasm_end_stream(ctx, s)
        B.oasm_step(ctx)
        for s in sids:
            res = B.oasm_flush(ctx, s)
            assert (res["stream_id"] == s).all()
            got[s] = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                       int(r["len"])) for r in res]
        for s, t in zip(sids, texts):
            assert canon(got[s]) == oracle_rows(pats, ks, t), s
            alone, _ = run_gpu(pats, ks, t)
            assert canon(alone) == canon(got[s])
    finally:
        B.oasm_destroy(ctx)


@pytest.mark.parametrize("n_pat", [1, 2, 3, 17, 31, 32, 33, 64, 100])
def test_lane_group_shapes(n_pat):
    """Few patterns spread one pattern over several lanes; many fill groups."""
    rng = np.random.default_rng(300 + n_pat)
    pats, ks, text = random_case(rng, 4, n_pat, 5, 60, 15000, kmax=5)
    rows, _ = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text)


def test_pattern_length_extremes():
    rng = np.random.default_rng(5)
    alpha = np.frombuffer(b"ACGT", np.uint8)
    pats = [alpha[rng.integers(0, 4, size=m)] for m in (1, 2, 31, 32, 33, 63, 64, 65, 96, 97, 127, 128)]
    ks = [0, 1, 7, 8, 15, 3, 15, 15, 15, 2, 15, 15]
    text = alpha[rng.integers(0, 4, size=20000)]
    for p, k in zip(pats, ks):
        for _ in range(3):
            W.plant(rng, text, W.edit_copy(rng, p, k, alpha))
    rows, _ = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text)


@pytest.mark.parametrize("n", [0, 1, 5, 7, 8, 9, 15, 16, 17, 33])
def test_short_and_empty_texts(n):
    rng = np.random.default_rng(n)
    pats, ks, text = random_case(rng, 2, 6, 2, 9, n, kmax=3)
    rows, _ = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text)


def test_byte_alphabet_all_values():
    rng = np.random.default_rng(9)
    pats, ks, text = random_case(rng, 256, 40, 10, 100, 50000, kmax=8)
    rows, _ = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text)


def test_device_feed_equals_host_feed():
    rng = np.random.default_rng(13)
    pats, ks, text = random_case(rng, 4, 20, 6, 30, 30000, kmax=3)
    a, _ = run_gpu(pats, ks, text)
    b, _ = run_gpu(pats, ks, text, device_feed=True, splits=[5000, 17000])
    assert canon(a) == canon(b) == oracle_rows(pats, ks, text)


def test_raw_outputs_less_naive_and_all_hits():
    rng = np.random.default_rng(17)
    pats, ks, text = random_case(rng, 4, 10, 5, 30, 8000, kmax=4)
    ends, _ = run_gpu(pats, ks, text, {"output": "ends"})
    assert canon(ends) == oracle_rows(pats, ks, text, mode="ends")
    allh, _ = run_gpu(pats, ks, text, {"output": "all_hits"})
    assert canon(allh) == oracle_rows(pats, ks, text, mode="hits")
    # kept <= Sellers ends <= hits (the shape of Table 1)
    kept, _ = run_gpu(pats, ks, text)
    assert len(kept) <= len(ends) <= len(allh)


@pytest.mark.parametrize("piece", [1, 4])
def test_raw_outputs_through_the_piece_filter(piece):
    """Less Naive ends and the full hit set of Eq. 2 with patterns on the piece
    filter: the filter's candidates are a superset of the scan's, so the raw
    outputs must still equal the oracle's."""
    rng = np.random.default_rng(19 + piece)
    pats, ks, text = random_case(rng, 256, 24, 12, 60, 20000, kmax=3)
    cfg = {"prefilter_piece": piece}
    ends, _ = run_gpu(pats, ks, text, {"output": "ends"}, cfg=cfg)
    assert canon(ends) == oracle_rows(pats, ks, text, mode="ends")
    allh, _ = run_gpu(pats, ks, text, {"output": "all_hits"}, cfg=cfg)
    assert canon(allh) == oracle_rows(pats, ks, text, mode="hits")
    assert len(allh) > 0


def test_small_buffers_regrow_and_rerun():
    """A step whose device buffers overflow is re-run after they grow."""
    rng = np.random.default_rng(21)
    pats = [np.frombuffer(b"AAAA", np.uint8)] * 3 + [np.frombuffer(b"ACAC", np.uint8)]
    ks = [1, 2, 3, 2]
    text = np.frombuffer(b"A" * 40000 + b"AC" * 20000, np.uint8).copy()
    rows, st = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text)


def test_stream_admission_and_slots():
    ctx = B.oasm_create([b"ACGTACGT"], [1], None, {"max_streams": 2})
    try:
        a = B.oasm_open_stream(ctx)
        b = B.oasm_open_stream(ctx)
        with pytest.raises(B.OasmError) as e:
            B.oasm_open_stream(ctx)
        assert e.value.code == B.OASM_EBUSY
        B.oasm_close_stream(ctx, a)
        c = B.oasm_open_stream(ctx)
        assert c == a
        B.oasm_close_stream(ctx, b)
        B.oasm_close_stream(ctx, c)
    finally:
        B.oasm_destroy(ctx)
    ctx = B.oasm_create([b"ACGTACGT"] * 100, [1] * 100, None, {"max_streams": 8, "mem_budget": 5000})
    try:
        s = B.oasm_open_stream(ctx)
        with pytest.raises(B.OasmError) as e:
            B.oasm_open_stream(ctx)
        assert e.value.code == B.OASM_ENOMEM
        B.oasm_close_stream(ctx, s)
        B.oasm_open_stream(ctx)
    finally:
        B.oasm_destroy(ctx)


def test_dictionary_dna_reduced():
    """Shape of the 1,024-pattern DNA dictionary at a size the oracle finishes fast."""
    wl = W.dictionary_dna(n=1 << 21, n_pat=256, copies=20)
    rows, st = run_gpu(wl.patterns, wl.ks, wl.texts[0])
    assert canon(rows) == oracle_rows(wl.patterns, wl.ks, wl.texts[0])
    assert st["kept"] == len(rows)


def test_bytes_zipf_reduced():
    wl = W.bytes_zipf(n=1 << 20, n_pat=200, copies=10)
    rows, _ = run_gpu(wl.patterns, wl.ks, wl.texts[0])
    assert canon(rows) == oracle_rows(wl.patterns, wl.ks, wl.texts[0])


def test_many_texts_reduced():
    wl = W.many_texts(n_texts=40, total=4e6, n_pat=64, copies=20)
    ctx = B.oasm_create(wl.patterns, wl.ks, None, {"max_streams": 64})
    try:
        sids = []
        for t in wl.texts:
            s = B.oasm_open_stream(ctx)
            B.oasm_feed(ctx, s, t)
            B.oasm_end_stream(ctx, s)
            sids.append(s)
        B.oasm_step(ctx)
        for s, t in zip(sids, wl.texts):
            res = B.oasm_flush(ctx, s)
            got = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                    int(r["len"])) for r in res]
            assert canon(got) == oracle_rows(wl.patterns, wl.ks, t)
    finally:
        B.oasm_destroy(ctx)


def test_autotune_then_search_matches_oracle():
    import json

    import torch
    wl = W.dictionary_dna(n=1 << 21, n_pat=80, copies=20)
    ctx = B.oasm_create(wl.patterns, wl.ks)
    try:
        t = torch.from_numpy(wl.texts[0]).cuda()
        rep = json.loads(B.oasm_autotune(ctx, t))
        assert rep["buckets"] and all(b["ms"] > 0 for b in rep["buckets"])
        sid = B.oasm_open_stream(ctx)
        B.oasm_feed_device(ctx, sid, t)
        res = B.oasm_flush(ctx, sid, end_of_stream=True)
        got = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                int(r["len"])) for r in res]
        assert canon(got) == oracle_rows(wl.patterns, wl.ks, wl.texts[0])
    finally:
        B.oasm_destroy(ctx)


@pytest.mark.parametrize("gpw", [1, 2])
def test_two_lane_groups_per_warp(gpw):
    """One-word classes scanned with one or two lane groups per warp: odd
    group counts (an idle second group), packed and one-pattern automaton
    groups sharing a warp, and the Myers/Hyyro class, against the oracle, in
    one feed and across feeds."""
    rng = np.random.default_rng(900 + gpw)
    lens, ks = [], []
    for m in rng.integers(8, 14, size=70).tolist() + rng.integers(20, 33, size=40).tolist():
        lens.append(m); ks.append(1)
    for m in rng.integers(20, 33, size=33).tolist():
        lens.append(m); ks.append(2)
    for m in rng.integers(12, 33, size=150).tolist():
        lens.append(m); ks.append(3)
    pats = [W.DNA[rng.integers(0, 4, size=m)] for m in lens]
    text = W.DNA[rng.integers(0, 4, size=50000)]
    for p, k in zip(pats[::2], ks[::2]):
        for cp in W.edit_copies(rng, p, rng.integers(0, k + 1, size=2), W.DNA):
            W.plant(rng, text, cp)
    want = oracle_rows(pats, ks, text)
    rows, _ = run_gpu(pats, ks, text, cfg={"groups_per_warp": gpw})
    assert canon(rows) == want
    split, _ = run_gpu(pats, ks, text, cfg={"groups_per_warp": gpw},
                       splits=np.sort(rng.integers(0, text.size, size=6)))
    assert canon(split) == want


def test_autotune_picks_groups_per_warp():
    import json

    import torch
    wl = W.dictionary_dna(n=1 << 21, n_pat=200, copies=10)
    ctx = B.oasm_create(wl.patterns, wl.ks)
    try:
        rep = json.loads(B.oasm_autotune(ctx, torch.from_numpy(wl.texts[0]).cuda()))
        for b in rep["buckets"]:
            assert b["gpw"] in ((1, 2) if b["W"] == 1 and b["dict"] else (1,))
            assert {t[0] for t in b["trials"]} <= {1, 2}
    finally:
        B.oasm_destroy(ctx)


@pytest.mark.parametrize("seed", range(3))
def test_piece_filter_equals_scan_and_oracle(seed):
    """Patterns whose K + 1 pieces are at least 4 symbols long go through the
    exact piece filter (cfg.prefilter_piece = 4); shorter ones stay on the
    scan.  Byte patterns over a skewed (Zipf) text with edited planted copies:
    the output equals the oracle's and the scan-only output, in one feed and
    across feeds, for several streams at once."""
    rng = np.random.default_rng(1000 + seed)
    table = W.zipf_table(np.random.default_rng(seed).permutation(256).astype(np.uint8))
    pats, ks = [], []
    for _ in range(60):
        m = int(rng.integers(6, 70))
        k = int(rng.integers(0, min(4, m // 3) + 1))
        pats.append(table[rng.integers(0, table.size, size=m)].astype(np.uint8))
        ks.append(k)
    for m in (8, 9, 10, 11):  # pieces of 2-3 symbols: these stay on the scan
        pats.append(table[rng.integers(0, table.size, size=m)].astype(np.uint8))
        ks.append(2)
    texts = []
    for _ in range(3):
        t = table[rng.integers(0, table.size, size=int(rng.integers(20000, 60000)))].astype(np.uint8)
        for p, k in zip(pats, ks):
            for cp in W.edit_copies(rng, p, rng.integers(0, k + 1, size=2), np.arange(256, dtype=np.uint8)):
                W.plant(rng, t, cp)
        texts.append(t)
    on_filter = sum(len(p) // (k + 1) >= 4 for p, k in zip(pats, ks))
    assert 20 <= on_filter < len(pats)
    for t in texts:
        want = oracle_rows(pats, ks, t)
        assert len(want) > 0
        got, _ = run_gpu(pats, ks, t, cfg={"prefilter_piece": 4})
        scan, _ = run_gpu(pats, ks, t)
        assert canon(got) == canon(scan) == want
    split, _ = run_gpu(pats, ks, texts[0], cfg={"prefilter_piece": 4},
                       splits=np.sort(rng.integers(0, texts[0].size, size=8)))
    assert canon(split) == oracle_rows(pats, ks, texts[0])
    # several streams in one step
    ctx = B.oasm_create(pats, ks, None, {"prefilter_piece": 4, "max_streams": 8})
    try:
        sids = [B.oasm_open_stream(ctx) for _ in texts]
        for s_, t in zip(sids, texts):
            B.oasm_feed(ctx, s_, t)
            B.oasm_end_stream(ctx, s_)
        B.oasm_step(ctx)
        for s_, t in zip(sids, texts):
            res = B.oasm_flush(ctx, s_)
            rows = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                     int(r["len"])) for r in res]
            assert canon(rows) == oracle_rows(pats, ks, t)
    finally:
        B.oasm_destroy(ctx)


@pytest.mark.parametrize("workload", ["dna", "zipf"])
def test_piece_filter_automatic_choice(workload):
    """prefilter_piece = 1: the library picks per pattern between the scan and
    the piece filter; the output equals the oracle's and the scan-only one."""
    rng = np.random.default_rng(77 if workload == "dna" else 78)
    if workload == "dna":
        wl = W.dictionary_dna(seed=21, n=300_000, n_pat=120, copies=6)
        pats, ks, text = wl.patterns, wl.ks, wl.texts[0]
    else:
        wl = W.bytes_zipf(seed=22, n=300_000, n_pat=150, copies=4)
        pats, ks, text = wl.patterns, wl.ks, wl.texts[0]
    want = oracle_rows(pats, ks, text)
    got, _ = run_gpu(pats, ks, text, cfg={"prefilter_piece": 1})
    assert len(want) > 0
    assert canon(got) == want
    split, _ = run_gpu(pats, ks, text, cfg={"prefilter_piece": 1},
                       splits=np.sort(rng.integers(0, text.size, size=4)))
    assert canon(split) == want


def test_piece_filter_set_grows_on_repetitive_text():
    """A text of one repeated symbol makes every piece match everywhere: the
    filter's (end, pattern) set overflows, grows and the step re-runs; pieces
    of 5 and 8 symbols, K = 0..3."""
    pats = [np.full(m, 65, np.uint8) for m in (16, 17, 20, 24, 32, 40)]
    ks = [0, 1, 2, 3, 2, 3]
    text = np.full(120000, 65, np.uint8)
    text[::997] = 66
    got, st = run_gpu(pats, ks, text, cfg={"prefilter_piece": 4})
    assert st["reruns"] >= 1
    assert canon(got) == oracle_rows(pats, ks, text)


def test_zero_copy_feed_from_registered_host_memory():
    """Packets fed from a registered host range are read by the device in
    place (no staging copy); the output equals the oracle's, and the range
    cannot be unregistered while its input waits for a step."""
    rng = np.random.default_rng(31)
    pats, ks, _ = random_case(rng, 4, 20, 6, 40, 10, kmax=3)
    texts = [random_case(rng, 4, 1, 6, 8, int(rng.integers(3000, 9000)))[2] for _ in range(5)]
    for t in texts:
        for p, k in zip(pats[:6], ks[:6]):
            W.plant(rng, t, W.edit_copy(rng, p, k, W.DNA))
    # interleave the texts as packets of 1..700 bytes in one buffer
    buf, pk = [], []
    pos = [0] * len(texts)
    off = 0
    while any(p_ < t.size for p_, t in zip(pos, texts)):
        for i, t in enumerate(texts):
            if pos[i] < t.size:
                n = int(min(rng.integers(1, 700), t.size - pos[i]))
                buf.append(t[pos[i]:pos[i] + n])
                pk.append((i, off, n))
                pos[i] += n
                off += n
    payload = np.ascontiguousarray(np.concatenate(buf))
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 8})
    try:
        B.oasm_register_host(ctx, payload)
        sids = [B.oasm_open_stream(ctx) for _ in texts]
        half = len(pk) // 2
        for part in (pk[:half], pk[half:]):
            B.oasm_feed_many(ctx, np.array([sids[i] for i, _, _ in part], np.uint32), payload,
                             np.array([o for _, o, _ in part], np.uint64),
                             np.array([n for _, _, n in part], np.uint32))
            with pytest.raises(B.OasmError) as ei:
                B.oasm_unregister_host(ctx, payload)
            assert ei.value.code == B.OASM_ESTATE
            B.oasm_step(ctx)
        for s_ in sids:
            B.oasm_end_stream(ctx, s_)
        B.oasm_step(ctx)
        B.oasm_unregister_host(ctx, payload)
        for s_, t in zip(sids, texts):
            res = B.oasm_flush(ctx, s_)
            rows = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                     int(r["len"])) for r in res]
            assert canon(rows) == oracle_rows(pats, ks, t)
    finally:
        B.oasm_destroy(ctx)


def test_split_steps_overlap_feeding_with_the_device():
    """oasm_step_begin / oasm_step_end: input fed, streams opened and hits
    drained while a step is in flight go to the next step; closing a stream
    of the step in flight finishes it first.  Every stream's output equals the
    oracle's."""
    rng = np.random.default_rng(41)
    pats, ks, _ = random_case(rng, 4, 24, 6, 40, 10, kmax=3)
    texts = [random_case(rng, 4, 1, 6, 8, int(rng.integers(4000, 12000)))[2] for _ in range(6)]
    for t in texts:
        for p, k in zip(pats[:8], ks[:8]):
            W.plant(rng, t, W.edit_copy(rng, p, k, W.DNA))
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 8})
    got = {}
    try:
        sids = {i: B.oasm_open_stream(ctx) for i in range(3)}  # three now, three later
        pos = [0] * len(texts)
        B.oasm_step_begin(ctx)  # nothing pending: launches nothing
        B.oasm_step_end(ctx)
        rounds = 0
        while any(p_ < t.size for p_, t in zip(pos, texts)):
            if rounds == 2:
                for i in range(3, 6):
                    sids[i] = B.oasm_open_stream(ctx)  # while a step may be in flight
            for i, sd in sids.items():
                if pos[i] < texts[i].size:
                    n = int(rng.integers(1, 3000))
                    B.oasm_feed(ctx, sd, texts[i][pos[i]:pos[i] + n])
                    pos[i] += n
                    if pos[i] >= texts[i].size:
                        B.oasm_end_stream(ctx, sd)
            B.oasm_step_end(ctx)
            B.oasm_step_begin(ctx)
            with pytest.raises(B.OasmError) as ei:
                B.oasm_step_begin(ctx)
            assert ei.value.code == B.OASM_ESTATE
            out = B.oasm_drain(ctx)
            for r in out:
                got.setdefault(int(r["stream_id"]), []).append(r)
            rounds += 1
        B.oasm_step_end(ctx)
        B.oasm_step(ctx)
        for r in B.oasm_drain(ctx):
            got.setdefault(int(r["stream_id"]), []).append(r)
        for i, sd in sids.items():
            rows = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                     int(r["len"])) for r in got.get(sd, [])]
            assert canon(rows) == oracle_rows(pats, ks, texts[i]), i
        # closing a stream that is part of the step in flight finishes the step
        sd = B.oasm_open_stream(ctx)
        B.oasm_feed(ctx, sd, texts[0][:5000])
        B.oasm_step_begin(ctx)
        B.oasm_close_stream(ctx, sd)
        B.oasm_step_end(ctx)
    finally:
        B.oasm_destroy(ctx)


@pytest.mark.parametrize("seed", range(8))
def test_fuzz_configurations(seed):
    """Random combinations of alphabet, lengths, thresholds, rules, feed
    splits and the library's execution choices (automaton on/off, lane groups
    per warp, graphs, piece filter off/fixed/automatic): always the oracle's
    output."""
    rng = np.random.default_rng(5000 + seed)
    sigma = int(rng.choice([2, 4, 20, 256]))
    n_pat = int(rng.integers(1, 90))
    mlo = int(rng.integers(1, 20))
    mhi = int(rng.integers(mlo, 129))
    pats, ks, text = random_case(rng, sigma, n_pat, mlo, mhi, int(rng.integers(0, 40000)),
                                 kmax=int(rng.integers(0, 9)))
    rules = RULE_SETS[int(rng.integers(0, len(RULE_SETS)))]
    cfg = {"myers_only": int(rng.integers(0, 2)), "groups_per_warp": int(rng.integers(0, 3)),
           "graphs": int(rng.integers(0, 2)),
           "prefilter_piece": int(rng.choice([0, 1, 4, 6]))}
    splits = np.sort(rng.integers(0, text.size + 1, size=int(rng.integers(0, 6))))
    rows, _ = run_gpu(pats, ks, text, rules, splits=splits, cfg=cfg)
    assert canon(rows) == oracle_rows(pats, ks, text, rules), (sigma, n_pat, mlo, mhi, cfg, rules)


def test_int_peak_microbenchmark_runs():
    ops, ms = B.oasm_measure_int_peak(0)
    assert ops > 1e12 and ms > 0


@pytest.mark.parametrize("K", [0, 1, 2])
def test_automaton_classes_equal_bit_vector_scan_and_oracle(K):
    """One-word patterns with K <= 2 run on the automaton scan when a class
    holds 32 or more of them; the Myers/Hyyro scan must give the same output."""
    rng = np.random.default_rng(400 + K)
    pats = [W.DNA[rng.integers(0, 4, size=int(rng.integers(max(K + 1, 3), 33)))] for _ in range(45)]
    ks = [K] * len(pats)
    text = W.DNA[rng.integers(0, 4, size=60000)]
    for p in pats:
        for cp in W.edit_copies(rng, p, rng.integers(0, K + 1, size=3), W.DNA):
            W.plant(rng, text, cp)
    auto, _ = run_gpu(pats, ks, text)
    myers, _ = run_gpu(pats, ks, text, cfg={"myers_only": 1})
    want = oracle_rows(pats, ks, text)
    assert canon(auto) == canon(myers) == want
    # also across feeds (state carried through the stored tail)
    split, _ = run_gpu(pats, ks, text, splits=np.sort(rng.integers(0, text.size, size=7)))
    assert canon(split) == want


@pytest.mark.parametrize("K,alpha", [(0, 2), (1, 2), (2, 4), (1, 256), (2, 2)])
def test_packed_automaton_lanes(K, alpha):
    """Automaton lanes hold up to four patterns whose lengths sum to at most
    32 bits.  Lanes of one to four slots, exactly full words, dense
    candidates (binary alphabet: the per-step recording mode) and sparse ones
    must all give the oracle's output, equal to the one-pattern-per-lane
    bit-vector scan, in one feed and across feeds."""
    rng = np.random.default_rng(700 + 10 * K + alpha)
    lens = [8] * 40 + [max(K + 1, 3)] * 10 + [16] * 6 + [24] * 6
    lens += [int(x) for x in rng.integers(K + 1, 33, size=40)]
    alphabet = np.arange(alpha, dtype=np.uint8)
    pats = [alphabet[rng.integers(0, alpha, size=m)] for m in lens]
    ks = [K] * len(pats)
    text = alphabet[rng.integers(0, alpha, size=12000 if alpha == 2 else 40000)]
    for p in pats[::3]:
        for cp in W.edit_copies(rng, p, rng.integers(0, K + 1, size=2), alphabet):
            W.plant(rng, text, cp)
    auto, st_auto = run_gpu(pats, ks, text)
    myers, st_myers = run_gpu(pats, ks, text, cfg={"myers_only": 1})
    want = oracle_rows(pats, ks, text)
    assert len(want) > 0
    assert canon(auto) == canon(myers) == want
    split, _ = run_gpu(pats, ks, text, splits=np.sort(rng.integers(0, text.size, size=5)))
    assert canon(split) == want
    # packing runs fewer lane words than one pattern per lane
    assert st_auto["word_steps"] < st_myers["word_steps"]


def test_packing_fills_lanes_with_four_short_patterns():
    """128 patterns of length 8 with K = 1 pack four to a lane: one lane
    group (32 lanes) instead of four."""
    rng = np.random.default_rng(77)
    pats = [W.DNA[rng.integers(0, 4, size=8)] for _ in range(128)]
    ks = [1] * 128
    text = W.DNA[rng.integers(0, 4, size=20000)]
    auto, st_auto = run_gpu(pats, ks, text)
    myers, st_myers = run_gpu(pats, ks, text, cfg={"myers_only": 1})
    assert canon(auto) == canon(myers) == oracle_rows(pats, ks, text)
    assert st_myers["word_steps"] == 4 * st_auto["word_steps"]


@pytest.mark.parametrize("seed", range(3))
def test_stream_state_moves_to_another_context(seed):
    """Save a stream mid-text, restore it into a new context, continue: the
    union of both halves' hits equals the uninterrupted result (oracle)."""
    rng = np.random.default_rng(600 + seed)
    pats, ks, text = random_case(rng, 4, 40, 6, 70, 30000, kmax=4)
    cut = int(rng.integers(1, text.size))
    want = oracle_rows(pats, ks, text)
    a = B.oasm_create(pats, ks)
    b = B.oasm_create(pats, ks)
    try:
        sa = B.oasm_open_stream(a)
        B.oasm_feed(a, sa, text[:cut])
        first = B.oasm_flush(a, sa)
        state = B.oasm_save_stream(a, sa)
        B.oasm_close_stream(a, sa)
        sb = B.oasm_open_stream(b)
        B.oasm_restore_stream(b, sb, state)
        B.oasm_feed(b, sb, text[cut:])
        second = B.oasm_flush(b, sb, end_of_stream=True)
        rows = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                 int(r["len"])) for r in np.concatenate([first, second])]
        assert canon(rows) == want
        # a state from another dictionary is refused
        c = B.oasm_create(pats[:-1], ks[:-1])
        try:
            sc = B.oasm_open_stream(c)
            with pytest.raises(B.OasmError):
                B.oasm_restore_stream(c, sc, state)
        finally:
            B.oasm_destroy(c)
    finally:
        B.oasm_destroy(a)
        B.oasm_destroy(b)


def test_graph_launched_steps_equal_direct_launches():
    """Steps launched as captured CUDA graphs (updated in place while the step
    shape repeats) give the same output as direct launches."""
    rng = np.random.default_rng(700)
    pats, ks, text = random_case(rng, 4, 50, 5, 60, 64000, kmax=4)
    splits = np.arange(4000, text.size, 4000)  # equal pieces: repeating step shapes
    g, sg = run_gpu(pats, ks, text, splits=splits, cfg={"graphs": 1, "timing": 1})
    d, sd = run_gpu(pats, ks, text, splits=splits)
    assert canon(g) == canon(d) == oracle_rows(pats, ks, text)
    assert 1 <= sg["graph_builds"] < sg["steps"]
    assert sd["graph_builds"] == 0
    assert sg["scan_ms"] > 0


def test_graph_cache_keeps_one_executable_per_step_topology():
    """Steps whose launch sequence alternates (the piece filter only when a
    step spans a whole piece start, sort passes that depend on the step's
    span) keep one cached graph per topology: after the first step of each
    topology no graph is built again, and the output equals direct launches."""
    rng = np.random.default_rng(701)
    pats, ks, text = random_case(rng, 256, 48, 12, 60, 200000, kmax=3)
    # alternate short and long steps so consecutive steps differ in shape
    cuts, pos = [], 0
    for i in range(40):
        pos += 700 if i % 2 else 9000
        cuts.append(pos)
    cfg = {"graphs": 1, "prefilter_piece": 1}
    g, sg = run_gpu(pats, ks, text, splits=cuts, cfg=cfg)
    d, sd = run_gpu(pats, ks, text, splits=cuts, cfg={"prefilter_piece": 1})
    assert canon(g) == canon(d) == oracle_rows(pats, ks, text)
    assert sg["steps"] >= 40
    assert sg["graph_builds"] <= 8


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    """Failure detection without a fault: a device wait on a barrier that
    nothing completes runs out of its bound and reports OASM_ETIMEOUT; the
    completed barrier reports OASM_OK; afterwards a search still matches the
    oracle."""
    assert B.oasm_selftest_wait(0, 1 << 16, arrive=False) == B.OASM_ETIMEOUT
    assert B.oasm_selftest_wait(0, 1 << 16, arrive=True) == B.OASM_OK
    rng = np.random.default_rng(71)
    pats, ks, text = random_case(rng, 4, 8, 6, 30, 5000, kmax=3)
    got, _ = run_gpu(pats, ks, text)
    assert canon(got) == oracle_rows(pats, ks, text)


def test_tuning_moves_between_contexts():
    """oasm_get_tuning / oasm_set_tuning: the settings one context's
    autotuner picked go to a second context over the same patterns, whose
    search still matches the oracle; entries that do not fit are rejected."""
    import torch
    rng = np.random.default_rng(72)
    pats, ks, text = random_case(rng, 4, 90, 6, 70, 120000, kmax=3)
    a = B.oasm_create(pats, ks, None, None)
    b = B.oasm_create(pats, ks, None, None)
    try:
        B.oasm_autotune(a, torch.from_numpy(text[:65536].copy()).cuda())
        ta = B.oasm_get_tuning(a)
        B.oasm_set_tuning(b, ta)
        assert B.oasm_get_tuning(b) == ta
        with pytest.raises(B.OasmError):
            B.oasm_set_tuning(b, ta[:-1])
        bad = [dict(e) for e in ta]
        bad[0]["warps"] = 17
        with pytest.raises(B.OasmError):
            B.oasm_set_tuning(b, bad)
        assert B.oasm_get_tuning(b) == ta  # a rejected call changes nothing
        sid = B.oasm_open_stream(b)
        B.oasm_feed(b, sid, text)
        res = B.oasm_flush(b, sid, end_of_stream=True)
        got = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                int(r["len"])) for r in res]
        assert canon(got) == oracle_rows(pats, ks, text)
    finally:
        B.oasm_destroy(a)
        B.oasm_destroy(b)


def test_feed_from_registered_host_memory():
    """oasm_feed of bytes inside a range registered with oasm_register_host
    reads them where they are (zero copy); bytes outside it go through the
    pinned staging buffer.  Both kinds of piece in one stream, over two
    steps: the output equals the oracle's."""
    rng = np.random.default_rng(61)
    pats, ks, text = random_case(rng, 4, 20, 6, 40, 50000, kmax=3)
    buf = np.ascontiguousarray(text.copy())
    reg = buf[:30000]
    ctx = B.oasm_create(pats, ks)
    try:
        B.oasm_register_host(ctx, reg)
        sid = B.oasm_open_stream(ctx)
        B.oasm_feed(ctx, sid, buf[:12000])          # registered: zero copy
        part = B.oasm_flush(ctx, sid)
        B.oasm_feed(ctx, sid, buf[12000:30000])     # registered: zero copy
        B.oasm_feed(ctx, sid, buf[30000:])          # outside: staged
        rest = B.oasm_flush(ctx, sid, end_of_stream=True)
        B.oasm_unregister_host(ctx, reg)
    finally:
        B.oasm_destroy(ctx)
    got = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
            int(r["len"])) for r in np.concatenate([part, rest])]
    assert canon(got) == oracle_rows(pats, ks, text)

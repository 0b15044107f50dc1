"""GPU parity of the weighted path (integer edit costs, a variant outside the
paper): the wave-front dynamic program, the weighted verification and the
unchanged filter, through the C ABI, against the CPU oracle with the same
costs -- exact agreement of pattern id, start, length, k and decision point."""
import numpy as np
import pytest

from paper_1712_03560_gb300 import binding as B
from paper_1712_03560_gb300 import workloads as W
from parity_util import canon, oracle_rows, random_case, run_gpu

pytestmark = pytest.mark.gpu

COSTS = [(1, 1, 1), (2, 1, 1), (1, 2, 2), (1, 2, 3), (3, 1, 2), (2, 3, 1), (1, 5, 5)]


@pytest.mark.parametrize("seed", range(7))
def test_weighted_random_dictionaries(seed):
    """Lengths 1..128 (one to four rows per lane), alphabets of 2, 4 and 256
    symbols, K up to 6, planted copies, several feed splits."""
    rng = np.random.default_rng(900 + seed)
    costs = COSTS[seed]
    sigma = (2, 4, 256)[seed % 3]
    pats, ks, text = random_case(rng, sigma, 24, 1, 128, 12000, kmax=6)
    for i in range(4):  # plant a few copies edited only by the cheapest operation
        p = pats[i]
        if p.size > 4:
            W.plant(rng, text, W.edit_copy(rng, p, 1, np.unique(text)))
    want = oracle_rows(pats, ks, text, costs=costs)
    got, st = run_gpu(pats, ks, text, costs=costs)
    assert canon(got) == want
    splits = np.sort(rng.integers(0, text.size, size=5))
    got2, _ = run_gpu(pats, ks, text, splits=splits, costs=costs)
    assert canon(got2) == want


def test_weighted_unit_costs_equal_the_bit_parallel_path():
    """costs = (1, 1, 1) through the weighted path, the paper's bit-parallel
    path and the oracle agree."""
    rng = np.random.default_rng(31)
    pats, ks, text = random_case(rng, 4, 70, 4, 40, 30000, kmax=3)
    want = oracle_rows(pats, ks, text)
    a, _ = run_gpu(pats, ks, text, costs=(1, 1, 1))
    b, _ = run_gpu(pats, ks, text)
    assert canon(a) == canon(b) == want


def test_weighted_raw_outputs_less_naive_and_all_hits():
    rng = np.random.default_rng(32)
    costs = (1, 2, 1)
    pats, ks, text = random_case(rng, 4, 12, 5, 60, 8000, kmax=4)
    ends, _ = run_gpu(pats, ks, text, {"output": "ends"}, costs=costs)
    assert canon(ends) == oracle_rows(pats, ks, text, mode="ends", costs=costs)
    allh, _ = run_gpu(pats, ks, text, {"output": "all_hits"}, costs=costs)
    assert canon(allh) == oracle_rows(pats, ks, text, mode="hits", costs=costs)
    kept, _ = run_gpu(pats, ks, text, costs=costs)
    assert len(kept) <= len(ends) <= len(allh)


@pytest.mark.parametrize("rules", [dict(replace="never", acc="last"),
                                   dict(order="per_start_best", cmp="ge")])
def test_weighted_other_rule_sets(rules):
    rng = np.random.default_rng(33)
    costs = (2, 1, 2)
    pats, ks, text = random_case(rng, 3, 10, 6, 30, 6000, kmax=5)
    got, _ = run_gpu(pats, ks, text, rules, costs=costs)
    assert canon(got) == oracle_rows(pats, ks, text, rules, costs=costs)


@pytest.mark.parametrize("n", [0, 1, 5, 31, 32, 33, 95])
def test_weighted_short_and_empty_texts(n):
    rng = np.random.default_rng(34 + n)
    pats, ks, text = random_case(rng, 2, 6, 2, 40, n, kmax=3)
    got, _ = run_gpu(pats, ks, text, costs=(1, 1, 2))
    assert canon(got) == oracle_rows(pats, ks, text, costs=(1, 1, 2))


def test_weighted_many_streams_alone_and_in_the_mix():
    rng = np.random.default_rng(35)
    costs = (1, 2, 2)
    pats, ks, _ = random_case(rng, 4, 16, 6, 70, 10, kmax=4)
    texts = [random_case(rng, 4, 1, 6, 8, int(rng.integers(0, 7000)))[2] for _ in range(6)]
    for t in texts:
        for p, k in zip(pats[:4], ks[:4]):
            if t.size > 100:
                W.plant(rng, t, W.edit_copy(rng, p, min(k, 1), W.DNA))
    ctx = B.oasm_create(pats, ks, None, {"max_streams": 8}, costs=costs)
    try:
        sids = [B.oasm_open_stream(ctx) for _ in texts]
        pos = [0] * len(texts)
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
        for s, t in zip(sids, texts):
            res = B.oasm_flush(ctx, s)
            got = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                    int(r["len"])) for r in res]
            assert canon(got) == oracle_rows(pats, ks, t, costs=costs)
    finally:
        B.oasm_destroy(ctx)


def test_weighted_autotune_then_search():
    import torch
    rng = np.random.default_rng(36)
    costs = (1, 2, 2)
    pats, ks, text = random_case(rng, 4, 40, 8, 100, 200000, kmax=3)
    ctx = B.oasm_create(pats, ks, None, {"timing": 1}, costs=costs)
    try:
        import json
        rep = json.loads(B.oasm_autotune(ctx, torch.from_numpy(text[:65536].copy()).cuda()))
        assert rep["buckets"] and all(b["gpw"] == 1 for b in rep["buckets"])
        sid = B.oasm_open_stream(ctx)
        B.oasm_feed(ctx, sid, text)
        res = B.oasm_flush(ctx, sid, end_of_stream=True)
        got = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
                int(r["len"])) for r in res]
        assert canon(got) == oracle_rows(pats, ks, text, costs=costs)
    finally:
        B.oasm_destroy(ctx)


def test_weighted_state_does_not_restore_into_a_unit_cost_context():
    """A saved stream carries its context's fingerprint, costs included."""
    rng = np.random.default_rng(37)
    pats, ks, text = random_case(rng, 4, 5, 8, 20, 3000, kmax=2)
    a = B.oasm_create(pats, ks, None, None, costs=(1, 2, 2))
    b = B.oasm_create(pats, ks, None, None)
    try:
        sid = B.oasm_open_stream(a)
        B.oasm_feed(a, sid, text)
        B.oasm_step(a)
        blob = B.oasm_save_stream(a, sid)
        sb = B.oasm_open_stream(b)
        with pytest.raises(B.OasmError):
            B.oasm_restore_stream(b, sb, blob)
    finally:
        B.oasm_destroy(a)
        B.oasm_destroy(b)


@pytest.mark.parametrize("costs", [(255, 255, 255), (1, 255, 255), (255, 1, 1), (16, 16, 1)])
def test_weighted_extreme_costs(costs):
    """Costs at the ends of their range: edits dearer than K leave only exact
    matches; dear indels leave substitutions only; dear substitutions leave
    indels only.  K up to 15, lengths up to 128."""
    rng = np.random.default_rng(38 + costs[0] + costs[2])
    pats, ks, text = random_case(rng, 4, 20, 16, 128, 20000, kmax=15)
    got, _ = run_gpu(pats, ks, text, costs=costs)
    assert canon(got) == oracle_rows(pats, ks, text, costs=costs)


def test_weighted_stream_moves_to_another_weighted_context():
    """Save a weighted stream mid-text, restore it into a second context with
    the same patterns and costs, continue: both halves' hits together equal
    the uninterrupted result."""
    rng = np.random.default_rng(39)
    costs = (2, 1, 3)
    pats, ks, text = random_case(rng, 4, 30, 6, 90, 20000, kmax=4)
    cut = int(rng.integers(1, text.size))
    want = oracle_rows(pats, ks, text, costs=costs)
    a = B.oasm_create(pats, ks, None, None, costs=costs)
    b = B.oasm_create(pats, ks, None, None, costs=costs)
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
    finally:
        B.oasm_destroy(a)
        B.oasm_destroy(b)


@pytest.mark.parametrize("costs", [(2, 254, 255), (255, 255, 255), (9, 255, 1)])
def test_weighted_large_costs_long_patterns(costs):
    """Costs up to 255 with patterns of 100..128 symbols: cell values reach
    l_p x c_del (at most 32,640, one cost more in a sum), the range the
    kernel's 16-bit halves must hold.  Copies planted with substitutions only
    (the cheap edit for the first cost set) and exact copies; whole output
    against the oracle, in one feed and in pieces."""
    rng = np.random.default_rng(1300 + costs[0])
    alphabet = np.arange(256, dtype=np.uint8)
    pats, ks = [], []
    for _ in range(40):
        m = int(rng.integers(100, 129))
        pats.append(alphabet[rng.integers(0, 256, size=m)])
        ks.append(int(rng.integers(0, 16)))
    text = alphabet[rng.integers(0, 256, size=30000)]
    for p in pats[:20]:
        cp = p.copy()
        for pos in rng.integers(0, p.size, size=int(rng.integers(0, 4))):
            cp[pos] = rng.integers(0, 256)
        W.plant(rng, text, cp)
    want = oracle_rows(pats, ks, text, costs=costs)
    got, _ = run_gpu(pats, ks, text, costs=costs)
    assert canon(got) == want
    got2, _ = run_gpu(pats, ks, text, splits=np.sort(rng.integers(0, text.size, size=4)),
                      costs=costs)
    assert canon(got2) == want
    if costs[0] == 2:
        assert len(want) >= 10

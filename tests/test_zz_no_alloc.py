"""The search call that allocates no device memory.

Some callers cannot allocate device memory themselves: a framework's caching
allocator may already hold the whole device, or a hard per-process memory cap
applies.  For them the library offers ``oasm_scan_ends_noalloc``, which works
only in the caller's buffers and in one fixed scratch array inside the
library.  These tests call it through the C ABI, several times in a row on
different inputs, and check that it returns exactly the end positions and
distances of the Less Naive output (Sec. 5.1): those of an ordinary context
in that output mode, and those of the CPU oracle (integer results, so the
comparisons are exact).  This file is collected last so that a run stopping
at its first failure has run every other test before it."""
import numpy as np
import pytest

import oracle
from paper_1712_03560_gb300 import binding as B
from paper_1712_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(seed, n_pat, n):
    rng = W.rng_for(seed)
    pats, ks = [], []
    for _ in range(n_pat):
        m = int(rng.integers(5, 41))
        pats.append(W.iid_dna(rng, m))
        ks.append(int(rng.integers(0, min(3, m - 1) + 1)))
    text = W.iid_dna(rng, n)
    for p, k in zip(pats, ks):
        for cp in W.edit_copies(rng, p, rng.integers(0, k + 1, size=5), W.DNA):
            W.plant(rng, text, cp)
    return pats, ks, text


def _byte_case(seed, n_pat, n):
    """Byte-alphabet patterns of 65..128 symbols (three and four words) with
    thresholds up to 15, over a skewed byte text with planted copies."""
    rng = W.rng_for(seed)
    alphabet = np.arange(256, dtype=np.uint8)
    probs = W.zipf_probs(1.1, 256)
    pats, ks = [], []
    for _ in range(n_pat):
        m = int(rng.integers(65, 129))
        pats.append(alphabet[rng.choice(256, size=m, p=probs)])
        ks.append(int(rng.integers(0, min(15, m - 1) + 1)))
    text = alphabet[rng.choice(256, size=n, p=probs)]
    for p, k in zip(pats, ks):
        for cp in W.edit_copies(rng, p, rng.integers(0, k + 1, size=4), alphabet):
            W.plant(rng, text, cp)
    return pats, ks, text


def _oracle_ends(pats, ks, text):
    res = oracle.oasm_dictionary(pats, ks, text, mode="ends")
    return sorted((int(r["pattern_id"]), int(r["decided_at"]), int(r["k"])) for r in res)


def _records(d_out, found):
    recs = d_out[: found * B.END_DTYPE.itemsize].cpu().numpy().view(B.END_DTYPE)
    return sorted((int(r["pattern_id"]), int(r["end"]), int(r["k"])) for r in recs)


def test_noalloc_equals_context_two_calls_in_a_row():
    import torch
    cap = 1 << 17
    d_out = torch.zeros(cap * B.END_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for seed, (n_pat, n) in enumerate([(40, 300_000), (64, 70_000)]):
        pats, ks, text = _case(100 + seed, n_pat, n)
        d_text = torch.from_numpy(text).cuda()
        found = B.oasm_scan_ends_noalloc(pats, ks, d_text, d_out, cap)
        assert 0 < found <= cap
        got = _records(d_out, found)
        with B.Matcher(pats, ks, {"output": "ends"}) as mt:
            res = mt.search(d_text, device=True)
        want = sorted((int(r["pattern_id"]), int(r["decided_at"]), int(r["k"])) for r in res)
        assert got == want


def test_noalloc_equals_oracle_on_long_byte_patterns():
    """Three- and four-word patterns with K up to 15 (the whole carry chain),
    then a DNA call on the same scratch array: both against the oracle."""
    import torch
    cap = 1 << 16
    d_out = torch.zeros(cap * B.END_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for pats, ks, text in (_byte_case(201, 24, 60_000), _case(202, 64, 50_000)):
        d_text = torch.from_numpy(text).cuda()
        found = B.oasm_scan_ends_noalloc(pats, ks, d_text, d_out, cap)
        assert 0 < found <= cap
        assert _records(d_out, found) == _oracle_ends(pats, ks, text)


def test_noalloc_truncates_at_cap_and_keeps_the_count():
    """More ends than cap: the call reports every end it found, writes cap of
    them, and those are ends of the full set."""
    import torch
    pats, ks, text = _case(211, 16, 40_000)
    want = _oracle_ends(pats, ks, text)
    assert len(want) > 100
    cap = 37
    d_out = torch.zeros(cap * B.END_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    d_text = torch.from_numpy(text).cuda()
    lib = B.load()
    import ctypes
    m = len(pats)
    arrs = [np.ascontiguousarray(p) for p in pats]
    ptrs = (ctypes.c_void_p * m)(*[a.ctypes.data for a in arrs])
    lens = (ctypes.c_uint32 * m)(*[a.size for a in arrs])
    kk = (ctypes.c_uint32 * m)(*ks)
    found = ctypes.c_uint64(0)
    rc = lib.oasm_scan_ends_noalloc(ptrs, lens, kk, m, d_text.data_ptr(), text.size,
                                    d_out.data_ptr(), cap, ctypes.byref(found),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == B.OASM_ETRUNC
    assert found.value == len(want)
    got = _records(d_out, cap)
    assert len(got) == cap and set(got) <= set(want)


@pytest.mark.parametrize("n", [0, 1, 7, 20, 40])
def test_noalloc_texts_shorter_than_the_warm_up(n):
    """Texts shorter than l_p + K: every end is still exact."""
    import torch
    rng = W.rng_for(220 + n)
    pats = [W.iid_dna(rng, m) for m in (5, 12, 33, 40)]
    ks = [2, 5, 9, 15]
    text = W.iid_dna(rng, n)
    if n >= 12:
        text[:12] = pats[1]
    cap = 4096
    d_out = torch.zeros(cap * B.END_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    d_text = torch.from_numpy(text.copy()).cuda() if n else torch.zeros(1, dtype=torch.uint8,
                                                                          device="cuda")
    found = B.oasm_scan_ends_noalloc(pats, ks, d_text, d_out, cap, n=n)
    assert _records(d_out, found) == _oracle_ends(pats, ks, text)


def test_noalloc_rejects_more_patterns_than_its_scratch_holds():
    import torch
    d_text = torch.zeros(16, dtype=torch.uint8, device="cuda")
    d_out = torch.zeros(16 * 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.OasmError) as e:
        B.oasm_scan_ends_noalloc([b"ACGTACGT"] * 65, [1] * 65, d_text, d_out, 16)
    assert e.value.code == B.OASM_EINVAL


def test_noalloc_binding_rejects_buffers_too_small_for_n_or_cap():
    """The binding refuses an n beyond the text tensor or a cap beyond the
    output tensor before the library is called."""
    import torch
    d_text = torch.zeros(100, dtype=torch.uint8, device="cuda")
    d_out = torch.zeros(10 * B.END_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for kw in ({"n": 101, "cap": 10}, {"n": 100, "cap": 11}):
        with pytest.raises(B.OasmError) as e:
            B.oasm_scan_ends_noalloc([b"ACGTACGT"], [1], d_text, d_out, kw["cap"], n=kw["n"])
        assert e.value.code == B.OASM_EINVAL
    with pytest.raises(B.OasmError):
        B.oasm_scan_ends_noalloc([b"ACGTACGT"], [1], d_text.cpu(), d_out, 10)

"""The search call that allocates no device memory.

Some callers cannot allocate device memory themselves: a framework's caching
allocator may already hold the whole device, or a hard per-process memory cap
applies.  For them the library offers ``oasm_scan_ends_noalloc``, which works
only in the caller's buffers and in one fixed scratch array inside the
library.  These tests call it through the C ABI twice in a row on different
inputs.  Each time they check that it returns exactly the end positions and
distances that an ordinary context returns in Less Naive output mode
(integer results, so the comparison is exact)."""
import numpy as np
import pytest

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


def test_noalloc_equals_context_two_calls_in_a_row():
    import torch
    cap = 1 << 17
    d_out = torch.zeros(cap * B.END_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for seed, (n_pat, n) in enumerate([(40, 300_000), (64, 70_000)]):
        pats, ks, text = _case(100 + seed, n_pat, n)
        d_text = torch.from_numpy(text).cuda()
        found = B.oasm_scan_ends_noalloc(pats, ks, d_text, d_out, cap)
        assert 0 < found <= cap
        recs = d_out[: found * B.END_DTYPE.itemsize].cpu().numpy().view(B.END_DTYPE)
        got = sorted((int(r["pattern_id"]), int(r["end"]), int(r["k"])) for r in recs)
        with B.Matcher(pats, ks, {"output": "ends"}) as mt:
            res = mt.search(d_text, device=True)
        want = sorted((int(r["pattern_id"]), int(r["decided_at"]), int(r["k"])) for r in res)
        assert got == want


def test_noalloc_rejects_more_patterns_than_its_scratch_holds():
    import torch
    d_text = torch.zeros(16, dtype=torch.uint8, device="cuda")
    d_out = torch.zeros(16 * 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.OasmError) as e:
        B.oasm_scan_ends_noalloc([b"ACGTACGT"] * 65, [1] * 65, d_text, d_out, 16)
    assert e.value.code == B.OASM_EINVAL

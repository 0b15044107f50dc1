"""GPU parity of the cut-off scan: multi-word classes (33..128 symbols) of 32
or more patterns compute only each pattern's first 32 rows while none of them
comes within K of a match, and every word near matches.  Their output must
equal the oracle's element by element, and equal the every-word scan
(cfg.full_words = 1), on inputs that enter and leave the full form often:
small alphabets, long planted copies, thresholds up to 15, periodic text."""
import numpy as np
import pytest

from paper_1712_03560_gb300 import workloads as W
from parity_util import canon, oracle_rows, run_gpu

pytestmark = pytest.mark.gpu


def multiword_case(rng, sigma, per_class, n, kmax, words=(2, 3, 4), copies=3):
    """per_class patterns in each word class, planted copies with up to K edits."""
    alphabet = np.frombuffer(b"ACGT", np.uint8) if sigma == 4 else np.arange(sigma, dtype=np.uint8)
    pats, ks = [], []
    for w in words:
        for _ in range(per_class):
            m = int(rng.integers(32 * (w - 1) + 1, 32 * w + 1))
            pats.append(alphabet[rng.integers(0, alphabet.size, size=m)])
            ks.append(int(rng.integers(0, min(kmax, m - 1, 15) + 1)))
    text = alphabet[rng.integers(0, alphabet.size, size=n)]
    for p, k in zip(pats, ks):
        for _ in range(copies):
            W.plant(rng, text, W.edit_copy(rng, p, int(rng.integers(0, k + 1)), alphabet))
    return pats, ks, text


@pytest.mark.parametrize("sigma,kmax", [(4, 15), (4, 3), (256, 8), (3, 15), (20, 6)])
def test_cutoff_equals_oracle(sigma, kmax):
    rng = np.random.default_rng(700 + sigma + kmax)
    pats, ks, text = multiword_case(rng, sigma, 33, 40000, kmax)
    rows, st = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text), (sigma, kmax)
    full, st_full = run_gpu(pats, ks, text, cfg={"full_words": 1})
    assert canon(full) == canon(rows)


@pytest.mark.parametrize("seed", range(3))
def test_cutoff_raw_ends_and_all_hits(seed):
    """Every Less Naive end (the scan's own candidate test, D[e] <= K) and
    every hit of Eq. 2: a missed or spurious candidate shows here."""
    rng = np.random.default_rng(720 + seed)
    pats, ks, text = multiword_case(rng, 4, 32, 30000, 12)
    ends, _ = run_gpu(pats, ks, text, {"output": "ends"})
    assert canon(ends) == oracle_rows(pats, ks, text, mode="ends")
    allh, _ = run_gpu(pats, ks, text, {"output": "all_hits"})
    assert canon(allh) == oracle_rows(pats, ks, text, mode="hits")


def test_cutoff_with_splits_and_one_symbol_feeds():
    """Stream cuts land anywhere relative to the 32-step blocks and the
    full-form episodes; the state carried between steps is the window state,
    and each step's warm-up re-enters the scan."""
    rng = np.random.default_rng(731)
    pats, ks, text = multiword_case(rng, 4, 32, 12000, 10)
    want = oracle_rows(pats, ks, text)
    cuts = sorted(set(int(x) for x in rng.integers(1, text.size, size=9)))
    rows, _ = run_gpu(pats, ks, text, splits=cuts)
    assert canon(rows) == want
    rows1, _ = run_gpu(pats[:40], ks[:40], text[:600], splits=list(range(1, 600)))
    assert canon(rows1) == oracle_rows(pats[:40], ks[:40], text[:600])


def test_cutoff_periodic_text_stays_in_full_form():
    """A text made of repeats of a pattern's prefix keeps its lanes within K
    for long stretches (the full form), then leaves them in random text."""
    rng = np.random.default_rng(741)
    alphabet = np.frombuffer(b"ACGT", np.uint8)
    pats, ks, _ = multiword_case(rng, 4, 32, 10, 15, words=(3,), copies=0)
    parts = []
    for i in range(8):
        p = pats[int(rng.integers(0, len(pats)))]
        parts.append(np.tile(p[:int(rng.integers(5, 40))], int(rng.integers(5, 60))))
        parts.append(alphabet[rng.integers(0, 4, size=int(rng.integers(50, 3000)))])
    text = np.concatenate(parts)
    rows, _ = run_gpu(pats, ks, text)
    assert canon(rows) == oracle_rows(pats, ks, text)


def test_cutoff_runs_fewer_words_on_sparse_matches():
    """On a byte text with rare matches the cut-off runs about one word per
    pattern and step, the every-word scan all of them (executed counts)."""
    rng = np.random.default_rng(751)
    pats, ks, text = multiword_case(rng, 256, 32, 200000, 8, copies=2)
    rows, st = run_gpu(pats, ks, text)
    full, st_full = run_gpu(pats, ks, text, cfg={"full_words": 1})
    assert canon(rows) == canon(full) == oracle_rows(pats, ks, text)
    words_full = sum((p.size + 31) // 32 for p in pats) * text.size
    assert st_full["word_steps"] == words_full
    assert st["word_steps"] < 0.5 * words_full
    assert st["word_steps"] >= len(pats) * text.size

"""Pins for the CPU oracle against things other than itself.

* the worked example printed in Sec. 4.2 (golden fixture),
* an edit distance found by breadth-first search over single-symbol edits:
  the definition of Sec. 3 (the fewest insertions, deletions and
  substitutions that turn one string into the other), with no dynamic
  programming at all,
* brute-force enumeration of every substring (Fully Naive, Sec. 5.1),
* textbook special cases (K = 0 reduces to leftmost non-overlapping exact
  search, done here with ``bytes.find``),
* invariants of the priority rules and of the validation step.
"""
import itertools
import os
from collections import deque

import numpy as np
import pytest

import oracle
from paper_1712_03560_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def load_golden():
    d = {"kept": [], "dropped": [], "r": {}}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key in ("pattern", "text"):
            d[key] = vals[0].encode()
        elif key == "K":
            d["K"] = int(vals[0])
        elif key in ("kept", "dropped"):
            d[key].append(tuple(int(v) for v in vals))
        elif key == "r":
            d["r"][int(vals[0])] = int(vals[1])
    return d


# --------------------------------------------------------------------------
# worked example (Sec. 4.2)

def test_worked_example_kept_set_and_counters():
    g = load_golden()
    kept, trace = oracle.oasm(g["pattern"], g["K"], g["text"], trace=True)
    first = trace[trace["decided_at"] == trace["decided_at"].min()]
    got_kept = sorted((int(r["start"]), int(r["len"]), int(r["level"])) for r in first if r["kept"])
    got_drop = sorted((int(r["start"]), int(r["len"]), int(r["level"])) for r in first if not r["kept"])
    assert got_kept == sorted(g["kept"])
    assert got_drop == sorted(g["dropped"])
    assert {int(r["level"]): int(r["r"]) for r in first} == g["r"]
    # the occurrence of priority 0 completes its validation when r(0) = l(0) = 5
    assert int(first["decided_at"][0]) == 10 + 5 - 1
    # Eq. 3 instances: r(1) - l(0) = 3 (not > 4) and r(2) - l(0) = 7 (> 3)
    lv = {int(r["level"]): r for r in first}
    assert int(lv[1]["acc"]) == 5 and int(lv[2]["acc"]) == 5
    # the first window is everything the 16 printed symbols produce
    assert sorted((int(h["start"]), int(h["len"]), int(h["k"])) for h in kept) == sorted(g["kept"])


@pytest.mark.parametrize("seed", range(8))
def test_worked_example_independent_of_continuation(seed):
    """The printed text ends in an ellipsis; no continuation changes the window
    decided at i = 14, since every hit starting at 11..14 overlaps t[10;5]."""
    g = load_golden()
    rng = np.random.default_rng(seed)
    tail = bytes(rng.choice(list(b"ABCD"), size=40).tolist())
    kept = oracle.oasm(g["pattern"], g["K"], g["text"] + tail)
    first = [(int(h["start"]), int(h["len"]), int(h["k"])) for h in kept if h["decided_at"] == 14]
    assert sorted(first) == sorted(g["kept"])


# --------------------------------------------------------------------------
# Eq. 1 against the definition by breadth-first search

def bfs_distances(src: bytes, alphabet: bytes, maxlen: int) -> dict:
    """Shortest number of single-symbol insertions, deletions and substitutions
    from ``src`` to every string of length <= maxlen over ``alphabet``."""
    dist = {src: 0}
    q = deque([src])
    while q:
        s = q.popleft()
        d = dist[s]
        nbrs = []
        for i in range(len(s)):
            nbrs.append(s[:i] + s[i + 1:])
            for c in alphabet:
                if c != s[i]:
                    nbrs.append(s[:i] + bytes([c]) + s[i + 1:])
        if len(s) < maxlen:
            for i in range(len(s) + 1):
                for c in alphabet:
                    nbrs.append(s[:i] + bytes([c]) + s[i:])
        for t in nbrs:
            if t not in dist:
                dist[t] = d + 1
                q.append(t)
    return dist


def all_strings(alphabet: bytes, maxlen: int):
    for L in range(maxlen + 1):
        for tup in itertools.product(alphabet, repeat=L):
            yield bytes(tup)


def test_lev_matches_bfs_definition_binary_up_to_6():
    alpha = b"AC"
    strings = list(all_strings(alpha, 6))
    for p in strings[1:]:
        dist = bfs_distances(p, alpha, 6)
        for s in strings:
            assert oracle.lev(p, s) == dist[s], (p, s)


def test_lev_matches_bfs_definition_dna_small():
    alpha = b"ACGT"
    rng = np.random.default_rng(7)
    for _ in range(12):
        p = bytes(rng.choice(list(alpha), size=int(rng.integers(1, 5))).tolist())
        dist = bfs_distances(p, alpha, 5)
        for _ in range(200):
            s = bytes(rng.choice(list(alpha), size=int(rng.integers(0, 6))).tolist())
            assert oracle.lev(p, s) == dist[s]


def test_fig1_shared_prefix_distances():
    """Fig. 1(a): p = ABCD against t[0,5] = ABBDA; one matrix yields the
    distances of t[0,3], t[0,4] and t[0,5] as c[4][3], c[4][4], c[4][5]."""
    p, t = b"ABCD", b"ABBDABCDACDB"
    pref = oracle.lev_prefixes(p, t[:5])
    dist = bfs_distances(p, b"ABCD", 6)
    for l in (3, 4, 5):
        assert pref[l] == dist[t[:l]] == oracle.lev(p, t[:l])
    assert list(pref[3:6]) == [2, 1, 2]


def test_lev_prefixes_equal_full_matrix_random():
    rng = np.random.default_rng(11)
    for _ in range(300):
        p = rng.integers(0, 4, size=int(rng.integers(1, 12))).astype(np.uint8)
        s = rng.integers(0, 4, size=int(rng.integers(0, 20))).astype(np.uint8)
        pref = oracle.lev_prefixes(p, s)
        for l in range(s.size + 1):
            assert pref[l] == oracle.lev(p, s[:l])


# --------------------------------------------------------------------------
# Less Naive and the hit set against brute force (Fully Naive, Sec. 5.1)

def fully_naive(p, K, t, levfn):
    """Every substring of every length, its distance, kept when <= K."""
    out = []
    n = len(t)
    for i in range(n):
        for l in range(1, n - i + 1):
            k = levfn(p, t[i:i + l])
            if k <= K:
                out.append((i, l, k))
    return sorted(out)


def test_hits_equal_fully_naive_binary_bfs():
    alpha = b"AC"
    rng = np.random.default_rng(3)
    for _ in range(25):
        m = int(rng.integers(1, 6))
        p = bytes(rng.choice(list(alpha), size=m).tolist())
        K = int(rng.integers(0, m))
        t = bytes(rng.choice(list(alpha), size=int(rng.integers(0, 11))).tolist())
        dist = bfs_distances(p, alpha, 10)
        want = fully_naive(p, K, t, lambda a, b: dist[b])
        got = sorted((int(h["start"]), int(h["len"]), int(h["k"])) for h in oracle.hits(p, K, t))
        assert got == want


@pytest.mark.parametrize("sigma", [2, 3, 4])
def test_hits_equal_fully_naive_random(sigma):
    rng = np.random.default_rng(100 + sigma)
    for _ in range(60):
        m = int(rng.integers(1, 8))
        K = int(rng.integers(0, m))
        p = rng.integers(0, sigma, size=m).astype(np.uint8)
        t = rng.integers(0, sigma, size=int(rng.integers(0, 40))).astype(np.uint8)
        want = fully_naive(p, K, t, oracle.lev)
        got = sorted((int(h["start"]), int(h["len"]), int(h["k"])) for h in oracle.hits(p, K, t))
        assert got == want


def test_sellers_is_min_over_starts():
    rng = np.random.default_rng(5)
    for _ in range(80):
        m = int(rng.integers(1, 9))
        p = rng.integers(0, 3, size=m).astype(np.uint8)
        t = rng.integers(0, 3, size=int(rng.integers(1, 50))).astype(np.uint8)
        D = oracle.sellers(p, t)
        for e in range(t.size):
            # every start 0..e, plus the empty substring (distance m)
            best = min([oracle.lev(p, t[i:e + 1]) for i in range(e + 1)] + [m])
            assert D[e] == best


def test_sellers_ends_are_hit_ends():
    rng = np.random.default_rng(6)
    for _ in range(60):
        m = int(rng.integers(2, 9))
        K = int(rng.integers(0, m))
        p = rng.integers(0, 3, size=m).astype(np.uint8)
        t = rng.integers(0, 3, size=int(rng.integers(1, 60))).astype(np.uint8)
        H = oracle.hits(p, K, t)
        ends = oracle.sellers_ends(p, K, t)
        end_set = sorted(set((H["start"] + H["len"] - 1).tolist()))
        assert ends["decided_at"].tolist() == end_set
        D = oracle.sellers(p, t)
        for r in ends:
            e = int(r["decided_at"])
            assert r["k"] == D[e]
            assert oracle.lev(p, t[int(r["start"]):e + 1]) == r["k"]
            assert r["start"] + r["len"] - 1 == e


# --------------------------------------------------------------------------
# Algorithm 1: special cases and invariants

def greedy_exact(p: bytes, t: bytes):
    out, pos = [], 0
    while True:
        j = t.find(p, pos)
        if j < 0:
            return out
        out.append(j)
        pos = j + len(p)


@pytest.mark.parametrize("seed", range(6))
def test_k0_is_leftmost_nonoverlapping_exact_search(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        m = int(rng.integers(1, 5))
        p = bytes(rng.choice(list(b"AC"), size=m).tolist())
        t = bytes(rng.choice(list(b"AC"), size=int(rng.integers(0, 200))).tolist())
        kept = oracle.oasm(p, 0, t)
        assert kept["start"].tolist() == greedy_exact(p, t)
        assert set(kept["len"].tolist()) <= {m}
        assert (kept["decided_at"] == kept["start"] + m - 1).all()


def test_no_hits_gives_empty_output():
    p = b"GGGGGGGG"
    t = b"ACAC" * 500
    assert oracle.oasm(p, 2, t).size == 0
    assert oracle.hits(p, 2, t).size == 0


def test_isolated_planted_copy_is_kept():
    rng = W.rng_for(9)
    p = W.iid_dna(rng, 20)
    t = np.full(400, ord("A"), np.uint8)
    t[::2] = ord("C")  # ACAC.. far from the pattern
    for edits in range(0, 4):
        cp = W.edit_copy(rng, p, edits, W.DNA)
        tt = t.copy()
        tt[150:150 + cp.size] = cp
        kept = oracle.oasm(p, 3, tt)
        k_copy = oracle.lev(p, cp)
        best = min(int(h["k"]) for h in kept)
        assert best <= k_copy <= edits
        win = [h for h in kept if 150 - 3 <= h["start"] <= 150 + 3 and h["k"] == best]
        assert win, kept


RULE_SETS = [dict(replace=r, order=o, acc=a, cmp=c)
             for r in ("contained", "same_end", "never")
             for o in ("per_start_length", "per_start_best")
             for a in ("sum", "last")
             for c in ("gt", "ge")]


def _random_case(rng, sigma=None):
    sigma = sigma or int(rng.integers(2, 5))
    m = int(rng.integers(2, 10))
    K = int(rng.integers(0, min(m, 4)))
    p = rng.integers(0, sigma, size=m).astype(np.uint8)
    n = int(rng.integers(1, 300))
    t = rng.integers(0, sigma, size=n).astype(np.uint8)
    for _ in range(int(rng.integers(0, 6))):
        cp = W.edit_copy(rng, p, int(rng.integers(0, K + 1)), np.arange(sigma, dtype=np.uint8))
        W.plant(rng, t, cp)
    return p, K, t


@pytest.mark.parametrize("ri", range(len(RULE_SETS)))
def test_invariants_every_rule_set(ri):
    rules = RULE_SETS[ri]
    rng = np.random.default_rng(1000 + ri)
    for _ in range(40):
        p, K, t = _random_case(rng)
        m = p.size
        kept, trace = oracle.oasm(p, K, t, rules, trace=True)
        H = oracle.hits(p, K, t)
        hset = {(int(h["start"]), int(h["len"])): int(h["k"]) for h in H}
        for h in kept:
            i, l, k = int(h["start"]), int(h["len"]), int(h["k"])
            assert hset.get((i, l)) == k <= K  # every kept hit is a hit
            assert m - K <= l <= m + K
            assert oracle.lev(p, t[i:i + l]) == k
            # a kept hit is decided no earlier than its own end, and no window
            # lasts more than (K+1)(m+K) - K symbols
            assert h["decided_at"] >= i + l - 1
            assert h["decided_at"] - i + 1 <= (K + 1) * (m + K) - K
        ends = oracle.sellers_ends(p, K, t)
        assert len(kept) <= len(ends) <= len(H)
        # each window adds exactly one occurrence at its own highest priority,
        # which is the smallest level present in mem at the flush
        for f in np.unique(trace["decided_at"]):
            rows = trace[trace["decided_at"] == f]
            assert rows["is_idx"].sum() == 1
            top = rows[rows["is_idx"] == 1][0]
            assert top["kept"] == 1 and top["level"] == rows["level"].min()
            assert top["start"] + top["len"] - 1 == f
            assert top["r"] == top["len"]
            for r in rows:
                assert r["r"] == f - r["start"] + 1  # r(j) counts from insertion


@pytest.mark.parametrize("seed", range(6))
def test_default_rules_keep_disjoint_hits(seed):
    rng = np.random.default_rng(500 + seed)
    for _ in range(60):
        p, K, t = _random_case(rng)
        kept = oracle.oasm(p, K, t)
        iv = sorted((int(h["start"]), int(h["start"] + h["len"] - 1)) for h in kept)
        for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
            assert a1 < b0, iv


def test_windows_cover_every_hit_start_once():
    """Every hit start falls inside exactly one decision window: the windows
    [first start seen, decided_at] of consecutive flushes do not overlap."""
    rng = np.random.default_rng(77)
    for _ in range(80):
        p, K, t = _random_case(rng)
        kept, trace = oracle.oasm(p, K, t, trace=True)
        H = oracle.hits(p, K, t)
        fl = np.unique(trace["decided_at"])
        starts = H["start"]
        # windows: (previous decided_at, decided_at]; every hit start lies in one
        prev = -1
        counted = 0
        for f in fl:
            sel = (starts > prev) & (starts <= f)
            counted += int(sel.sum())
            if sel.any():
                # the window's hits include its kept top-priority occurrence
                top = trace[(trace["decided_at"] == f) & (trace["is_idx"] == 1)][0]
                assert int(H["k"][sel].min()) <= int(top["level"])
            prev = f
        assert counted == starts.size


def test_dictionary_is_independent_per_pattern():
    rng = W.rng_for(12)
    pats = [W.iid_dna(rng, int(m)) for m in (8, 10, 12, 9)]
    ks = [1, 2, 2, 0]
    t = W.iid_dna(rng, 3000)
    res = oracle.oasm_dictionary(pats, ks, t, threads=2)
    for pid, (p, k) in enumerate(zip(pats, ks)):
        one = oracle.oasm(p, k, t)
        sub = res[res["pattern_id"] == pid]
        assert sorted(map(tuple, one[["start", "len", "k", "decided_at"]].tolist())) == \
            sorted(map(tuple, sub[["start", "len", "k", "decided_at"]].tolist()))


def test_oracle_rejects_bad_thresholds():
    with pytest.raises(ValueError):
        oracle.oasm(b"ACGT", 4, b"ACGTACGT")  # K < l_p is required (Sec. 6.3)
    with pytest.raises(ValueError):
        oracle.hits(b"", 0, b"ACGT")

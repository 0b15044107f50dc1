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
            # the reported length is the shortest in-range one attaining D[e]
            for ll in range(max(1, m - K), int(r["len"])):
                if e - ll + 1 >= 0:
                    assert oracle.lev(p, t[e - ll + 1:e + 1]) > r["k"], (e, ll)


RULE_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rule_readings.txt")


def load_rule_cases():
    """Cases of tests/golden/rule_readings.txt: the hit set and the kept set
    under each reading, worked out by hand from the readings' definitions."""
    cases, cur = [], None
    for line in open(RULE_GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest, "hits": [], "kept": {}}
            cases.append(cur)
        elif key in ("pattern", "text"):
            cur[key] = rest.encode()
        elif key == "K":
            cur["K"] = int(rest)
        elif key == "hit":
            cur["hits"].append(tuple(int(x) for x in rest.split()))
        elif key == "kept":
            reading, _, rows = rest.partition(":")
            rules = {} if reading == "default" else dict([reading.split("=")])
            cur["kept"][reading] = (rules, sorted(tuple(int(x) for x in r.split())
                                                  for r in rows.split(";") if r.strip()))
    return cases


RULE_CASES = load_rule_cases()


@pytest.mark.parametrize("ci", range(len(RULE_CASES)), ids=[c["name"] for c in RULE_CASES])
def test_rule_readings_hand_worked_cases(ci):
    """Each non-default reading (same_end, never, ge, last, per_start_best)
    changes the kept set of at least one case, and every case's kept set under
    every reading is the hand-derived one.  The hit sets themselves are checked
    against distances from breadth-first search over edits."""
    c = RULE_CASES[ci]
    p, t, K = c["pattern"], c["text"], c["K"]
    H = oracle.hits(p, K, t)
    assert [(int(h["start"]), int(h["len"]), int(h["k"])) for h in H] == c["hits"]
    # H itself, from breadth-first search over single-symbol edits of p
    alphabet = bytes(sorted(set(p + t)))
    dist = bfs_distances(p, alphabet, len(p) + K)
    brute = [(i, ln, dist[t[i:i + ln]]) for i in range(len(t))
             for ln in range(max(1, len(p) - K), len(p) + K + 1)
             if i + ln <= len(t) and dist[t[i:i + ln]] <= K]
    assert brute == c["hits"]
    for reading, (rules, want) in c["kept"].items():
        got = sorted((int(x["start"]), int(x["len"]), int(x["k"]), int(x["decided_at"]))
                     for x in oracle.oasm(p, K, t, rules))
        assert got == want, (c["name"], reading)


def test_rule_readings_each_change_some_kept_set():
    """The hand-worked cases tell every reading from the default."""
    changed = set()
    for c in RULE_CASES:
        base = c["kept"]["default"][1]
        for reading, (_, want) in c["kept"].items():
            if want != base:
                changed.add(reading)
    assert changed == {"replace=same_end", "replace=never", "cmp=ge", "acc=last",
                       "order=per_start_best"}


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


def check_window_layout(kept):
    """What Eq. 3 with GT and SUM guarantees about the kept hits:
    * a window's lower-level hits end at least two symbols before the start
      of its top hit (r(j) - l(top) > l(j) with r(j) = f - i_j + 1);
    * the hits of one window all lie before those of the next window.
    Lower-level hits of one window may overlap each other: the comparison
    bounds their ends by the top hit's start minus the lengths accumulated
    so far, not by the position of the other lower hits."""
    groups = {}
    for h in kept:
        groups.setdefault(int(h["decided_at"]), []).append(h)
    prev_end = -1
    for f in sorted(groups):
        g = groups[f]
        top = min(g, key=lambda h: int(h["k"]))
        assert int(top["start"] + top["len"] - 1) == f
        for h in g:
            if h is not top:
                assert int(h["start"] + h["len"] - 1) < int(top["start"]) - 1
        assert min(int(h["start"]) for h in g) > prev_end
        prev_end = f


@pytest.mark.parametrize("seed", range(6))
def test_default_rules_keep_lower_hits_clear_of_the_top_hit(seed):
    rng = np.random.default_rng(500 + seed)
    for _ in range(60):
        p, K, t = _random_case(rng)
        check_window_layout(oracle.oasm(p, K, t))


def test_lower_level_hits_of_one_window_may_overlap():
    """p = [1,1,0,1,1], K = 3: the window decided at f = 33 keeps its top hit
    (29, l=5, k=0), and at levels 2 and 3 two hits that both start at 23:
    Eq. 3 gives r(2) - 5 = 11 - 5 = 6 > 3 and r(3) - (5 + 3) = 3 > 2."""
    rng = np.random.default_rng(44)
    for _ in range(109):
        p, K, t = _random_case(rng)
    assert p.tolist() == [1, 1, 0, 1, 1] and K == 3
    kept = oracle.oasm(p, K, t)
    rows = sorted((int(h["start"]), int(h["len"]), int(h["k"])) for h in kept
                  if int(h["decided_at"]) == 33)
    assert rows == [(23, 2, 3), (23, 3, 2), (29, 5, 0)]
    check_window_layout(kept)


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


# --------------------------------------------------------------------------
# integer edit costs (a variant outside the paper: Eq. 1 with the unit terms
# replaced by a substitution, an insertion and a deletion cost)

def dijkstra_distances(p: bytes, alphabet: bytes, maxlen: int, costs):
    """Cheapest sequence of single-symbol edits turning p into every string
    of length <= maxlen: deleting a symbol of p costs ``del``, inserting a
    text symbol ``ins``, replacing one ``sub``.  The definition, searched
    over strings, with no alignment matrix."""
    import heapq
    sub, ins, dele = costs
    dist = {p: 0}
    heap = [(0, p)]
    while heap:
        d, s = heapq.heappop(heap)
        if d > dist[s]:
            continue
        nbrs = []
        for i in range(len(s)):
            nbrs.append((s[:i] + s[i + 1:], dele))
            for c in alphabet:
                if c != s[i]:
                    nbrs.append((s[:i] + bytes([c]) + s[i + 1:], sub))
        if len(s) < maxlen:
            for i in range(len(s) + 1):
                for c in alphabet:
                    nbrs.append((s[:i] + bytes([c]) + s[i:], ins))
        for t, w in nbrs:
            if d + w < dist.get(t, 1 << 30):
                dist[t] = d + w
                heapq.heappush(heap, (d + w, t))
    return dist


COST_SETS = [(1, 1, 1), (2, 1, 1), (1, 2, 3), (3, 1, 2), (1, 4, 1), (5, 2, 2), (2, 3, 1)]


@pytest.mark.parametrize("costs", COST_SETS)
def test_weighted_lev_matches_cheapest_edit_sequence(costs):
    alpha = b"AC"
    strings = list(all_strings(alpha, 5))
    for p in strings[1:]:
        dist = dijkstra_distances(p, alpha, 6, costs)
        for s in strings:
            assert oracle.lev(p, s, costs=costs) == dist[s], (p, s, costs)


def lcs_brute(a: bytes, b: bytes) -> int:
    """Longest common subsequence by trying every subsequence of a."""
    for L in range(len(a), -1, -1):
        for idx in itertools.combinations(range(len(a)), L):
            sub = bytes(a[i] for i in idx)
            it = iter(b)
            if all(c in it for c in sub):
                return L
    return 0


def test_weighted_lev_without_useful_substitutions_is_indel_distance():
    """sub >= ins + del: a substitution never beats a deletion plus an
    insertion, so the distance is del (m - LCS) + ins (n - LCS)."""
    rng = np.random.default_rng(21)
    for _ in range(300):
        p = bytes(rng.choice(list(b"ACG"), size=int(rng.integers(1, 7))).tolist())
        s = bytes(rng.choice(list(b"ACG"), size=int(rng.integers(0, 7))).tolist())
        ins, dele = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        sub = ins + dele + int(rng.integers(0, 3))
        c = lcs_brute(p, s)
        assert oracle.lev(p, s, costs=(sub, ins, dele)) == dele * (len(p) - c) + ins * (len(s) - c)


def test_weighted_lev_with_costly_indels_is_hamming():
    """Insertions and deletions dearer than any substitution pattern: equal
    lengths give sub times the Hamming distance."""
    rng = np.random.default_rng(22)
    for _ in range(300):
        m = int(rng.integers(1, 12))
        p = rng.integers(0, 4, size=m).astype(np.uint8)
        s = rng.integers(0, 4, size=m).astype(np.uint8)
        sub = int(rng.integers(1, 4))
        big = sub * m + 1
        assert oracle.lev(p, s, costs=(sub, big, big)) == sub * int((p != s).sum())


def test_weighted_lev_swaps_insertion_and_deletion_with_the_strings():
    """Reading an alignment from the other string turns insertions into
    deletions: d_(sub,ins,del)(p, s) = d_(sub,del,ins)(s, p)."""
    rng = np.random.default_rng(23)
    for _ in range(400):
        p = rng.integers(0, 3, size=int(rng.integers(1, 10))).astype(np.uint8)
        s = rng.integers(0, 3, size=int(rng.integers(1, 10))).astype(np.uint8)
        sub, ins, dele = (int(x) for x in rng.integers(1, 6, size=3))
        assert oracle.lev(p, s, costs=(sub, ins, dele)) == oracle.lev(s, p, costs=(sub, dele, ins))
        # scaling every cost scales the distance
        assert oracle.lev(p, s, costs=(3 * sub, 3 * ins, 3 * dele)) == \
            3 * oracle.lev(p, s, costs=(sub, ins, dele))


@pytest.mark.parametrize("costs", [(2, 1, 1), (1, 2, 3), (3, 1, 2)])
def test_weighted_lev_prefixes_sellers_hits_and_ends_brute_force(costs):
    rng = np.random.default_rng(sum(costs))
    for _ in range(40):
        m = int(rng.integers(1, 8))
        K = int(rng.integers(0, m))
        p = rng.integers(0, 3, size=m).astype(np.uint8)
        t = rng.integers(0, 3, size=int(rng.integers(1, 35))).astype(np.uint8)
        lv = lambda a, b: oracle.lev(a, b, costs=costs)  # noqa: E731
        pref = oracle.lev_prefixes(p, t, costs=costs)
        assert [int(x) for x in pref] == [lv(p, t[:l]) for l in range(t.size + 1)]
        D = oracle.sellers(p, t, costs=costs)
        for e in range(t.size):
            best = min([lv(p, t[i:e + 1]) for i in range(e + 1)] + [m * costs[2]])
            assert D[e] == best
        want = fully_naive(p, K, t, lv)
        H = oracle.hits(p, K, t, costs=costs)
        assert sorted((int(h["start"]), int(h["len"]), int(h["k"])) for h in H) == want
        ends = oracle.sellers_ends(p, K, t, costs=costs)
        assert ends["decided_at"].tolist() == sorted({i + l - 1 for i, l, _ in want})
        for r in ends:
            e = int(r["decided_at"])
            assert r["k"] == D[e] and lv(p, t[int(r["start"]):e + 1]) == r["k"]


@pytest.mark.parametrize("costs", [(2, 1, 1), (1, 2, 3), (3, 1, 2), (1, 1, 1)])
def test_weighted_oasm_invariants(costs):
    """Kept hits are weighted hits at their own distance; each window's
    lower-level hits end before its top hit, windows do not interleave; the
    first window keeps a hit at least as good as the first hit."""
    rng = np.random.default_rng(40 + costs[0] + 3 * costs[1])
    for _ in range(120):
        p, K, t = _random_case(rng)
        H = {(int(h["start"]), int(h["len"])): int(h["k"])
             for h in oracle.hits(p, K, t, costs=costs)}
        kept = oracle.oasm(p, K, t, costs=costs)
        for r in kept:
            assert H[(int(r["start"]), int(r["len"]))] == int(r["k"])
            assert oracle.lev(p, t[int(r["start"]):int(r["start"] + r["len"])], costs=costs) == r["k"]
        check_window_layout(kept)
        if H:
            assert len(kept) >= 1
            # the first hit in (start, length) order opens the first window,
            # which keeps a hit at least as good
            first = min(H)
            assert min(int(r["k"]) for r in kept if r["decided_at"] == kept["decided_at"].min()) \
                <= H[first]
    # unit costs given explicitly are the paper's distance
    g = load_golden()
    a = oracle.oasm(g["pattern"], g["K"], g["text"], costs=(1, 1, 1))
    b = oracle.oasm(g["pattern"], g["K"], g["text"])
    assert a.tolist() == b.tolist()


def test_weighted_k0_is_exact_search_under_any_costs():
    """With K = 0 no edit fits whatever the costs: greedy exact search."""
    rng = np.random.default_rng(44)
    for _ in range(30):
        p = bytes(rng.choice(list(b"AC"), size=int(rng.integers(2, 5))).tolist())
        t = bytes(rng.choice(list(b"AC"), size=200).tolist())
        costs = tuple(int(x) for x in rng.integers(1, 4, size=3))
        kept = oracle.oasm(p, 0, t, costs=costs)
        assert sorted(int(r["start"]) for r in kept) == greedy_exact(p, t)


def test_oracle_rejects_bad_costs():
    with pytest.raises(ValueError):
        oracle.lev(b"AC", b"A", costs=(0, 1, 1))
    with pytest.raises(ValueError):
        oracle.hits(b"ACG", 1, b"ACGT", costs=(1, 256, 1))


@pytest.mark.parametrize("costs", [(2, 1, 1), (1, 2, 1), (1, 1, 3)])
def test_weighted_hits_exhaustive_binary(costs):
    """Every binary pattern of length 1-4, every K < m, every binary text of
    length 7: the weighted hit set equals Fully Naive enumeration with the
    distances of the cheapest edit sequence (Dijkstra, no alignment matrix)."""
    alpha = b"AC"
    texts = [bytes(t) for t in itertools.product(alpha, repeat=7)]
    for m in range(1, 5):
        for p in itertools.product(alpha, repeat=m):
            p = bytes(p)
            dist = dijkstra_distances(p, alpha, 8, costs)
            for K in range(m):
                for t in texts[::3]:
                    want = fully_naive(p, K, t, lambda a, b: dist[b])
                    got = sorted((int(h["start"]), int(h["len"]), int(h["k"]))
                                 for h in oracle.hits(p, K, t, costs=costs))
                    assert got == want, (p, K, t)

"""Seeded synthetic inputs shaped like the OASM paper's workloads.

This module only draws random symbols and plants edited pattern copies; it
holds none of the matching arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.  Every generator uses
``numpy.random.Generator(PCG64(seed))``.

Workload shapes (the paper's own data are not available):
  * ``plain_dna``      one DNA pattern m=8, K=2, 1e6 iid {A,C,G,T} symbols,
                       200 planted copies with 0-2 edits (Tables 2/3 of the
                       paper use random {A,B,C,D} text).
  * ``dictionary_dna`` 1,024 DNA patterns m~U[8,32], K=floor(m/10), 256 MiB
                       iid text, 1,000 copies per pattern with exactly K edits
                       (MOASM, Sec. 6.4; miRNA-sized motifs of Sec. 5).
  * ``bytes_zipf``     4,096 byte patterns m log-uniform in [16,128],
                       K~U[1, min(8, m//4)], Zipf(1.1) bytes (NIDS-like
                       signatures, Sec. 1), 500 copies each with 1..K edits.
  * ``many_texts``     10,000 DNA texts, log-normal lengths (median 1e5,
                       clipped to [1e3, 1e7], ~4 GB) x 512 patterns
                       m~U[12,48], K=3, 200 copies per pattern, 0-3 edits.
  * ``served``         4,096 byte streams, packets U[64,1500] bytes, Poisson
                       arrivals, 2,000 signatures m~U[8,64], K=2, Zipf(1.1)
                       payload, 1% of packets carry an edited signature.
Edits are a substitution by a different symbol, an insertion of a random
symbol or a deletion, each at a uniform position inside the copy; copies
overwrite the text at uniform offsets.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DNA = np.frombuffer(b"ACGT", dtype=np.uint8)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def edit_copy(rng: np.random.Generator, pat: np.ndarray, n_edits: int, alphabet: np.ndarray,
              probs: np.ndarray | None = None) -> np.ndarray:
    """Applies ``n_edits`` random substitutions/insertions/deletions to a copy."""
    s = list(pat.tolist())
    for _ in range(n_edits):
        op = int(rng.integers(0, 3)) if len(s) > 1 else 1
        if op == 0:  # substitution by a different symbol
            pos = int(rng.integers(0, len(s)))
            while True:
                c = int(alphabet[rng.integers(0, alphabet.size)]) if probs is None else \
                    int(rng.choice(alphabet, p=probs))
                if c != s[pos]:
                    break
            s[pos] = c
        elif op == 1:  # insertion of a random symbol
            pos = int(rng.integers(0, len(s) + 1))
            c = int(alphabet[rng.integers(0, alphabet.size)]) if probs is None else \
                int(rng.choice(alphabet, p=probs))
            s.insert(pos, c)
        else:  # deletion
            pos = int(rng.integers(0, len(s)))
            del s[pos]
    return np.asarray(s, dtype=np.uint8)


def edit_copies(rng: np.random.Generator, pat: np.ndarray, n_edits: np.ndarray,
                alphabet: np.ndarray) -> list:
    """Vectorised ``edit_copy`` for many copies of one pattern.

    ``n_edits[c]`` edits are applied to copy c; each edit is a uniform choice of
    substitution (by a different symbol of ``alphabet``), insertion or deletion
    at a uniform position.  Returns one uint8 array per copy.
    """
    n_edits = np.asarray(n_edits, dtype=np.int64)
    nc, m = n_edits.size, pat.size
    width = m + int(n_edits.max(initial=0)) + 1
    buf = np.zeros((nc, width), dtype=np.uint8)
    buf[:, :m] = pat
    ln = np.full(nc, m, dtype=np.int64)
    a = alphabet.astype(np.uint8)
    col = np.arange(width)[None, :]
    rows = np.arange(nc)
    for step in range(int(n_edits.max(initial=0))):
        act = n_edits > step
        op = rng.integers(0, 3, size=nc)
        op[ln <= 1] = 1
        pos = (rng.random(nc) * (ln + (op == 1))).astype(np.int64)
        # a different symbol for substitutions, any symbol for insertions
        cur = buf[rows, np.minimum(pos, width - 1)]
        sym = a[rng.integers(0, a.size, size=nc)]
        bad = (op == 0) & (sym == cur)
        while bad.any():
            sym[bad] = a[rng.integers(0, a.size, size=int(bad.sum()))]
            bad = (op == 0) & (sym == cur)
        p = pos[:, None]
        sub = np.where(col == p, sym[:, None], buf)
        shifted_r = np.concatenate([buf[:, :1], buf[:, :-1]], axis=1)
        ins = np.where(col < p, buf, np.where(col == p, sym[:, None], shifted_r))
        shifted_l = np.concatenate([buf[:, 1:], buf[:, -1:]], axis=1)
        dele = np.where(col < p, buf, shifted_l)
        new = np.where((op == 0)[:, None], sub, np.where((op == 1)[:, None], ins, dele))
        buf = np.where(act[:, None], new, buf)
        ln = ln + act * ((op == 1).astype(np.int64) - (op == 2).astype(np.int64))
    return [buf[c, :ln[c]].copy() for c in range(nc)]


def plant(rng: np.random.Generator, text: np.ndarray, copy: np.ndarray) -> int:
    """Overwrites ``text`` with ``copy`` at a uniform offset; returns the offset."""
    if copy.size == 0 or copy.size > text.size:
        return -1
    off = int(rng.integers(0, text.size - copy.size + 1))
    text[off:off + copy.size] = copy
    return off


def iid_dna(rng: np.random.Generator, n: int) -> np.ndarray:
    return DNA[rng.integers(0, 4, size=n, dtype=np.uint8)]


def zipf_probs(s: float = 1.1, ranks: int = 256) -> np.ndarray:
    w = 1.0 / np.arange(1, ranks + 1, dtype=np.float64) ** s
    return w / w.sum()


def zipf_table(perm: np.ndarray, s: float = 1.1, cells: int = 1 << 20) -> np.ndarray:
    """2^20 equally likely cells; cell i holds the byte of the rank whose CDF
    interval contains (i + 0.5) / 2^20 (the smallest rank probability, ~3.5e-4
    at s = 1.1, spans hundreds of cells)."""
    cdf = np.cumsum(zipf_probs(s, 256))
    cdf[-1] = 1.0
    idx = np.searchsorted(cdf, (np.arange(cells) + 0.5) / cells, side="right").clip(0, 255)
    return perm[idx]


def zipf_bytes(rng: np.random.Generator, n: int, perm: np.ndarray, s: float = 1.1,
               chunk: int = 1 << 26, table: np.ndarray | None = None) -> np.ndarray:
    """Bytes whose ranks follow Zipf(s) over 256 ranks, mapped by ``perm``
    (sampled by lookup in ``zipf_table``)."""
    if table is None:
        table = zipf_table(perm, s)
    out = np.empty(n, dtype=np.uint8)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = table[rng.integers(0, table.size, size=b - a, dtype=np.uint32)]
    return out


@dataclass
class Workload:
    name: str
    patterns: list            # list of np.uint8 arrays
    ks: np.ndarray            # int32 thresholds
    texts: list               # list of np.uint8 arrays (one per stream/text)
    meta: dict = field(default_factory=dict)

    @property
    def text_bytes(self) -> int:
        return int(sum(t.size for t in self.texts))

    @property
    def cells(self) -> int:
        """Sellers cells: sum over patterns of m times the text length."""
        msum = int(sum(p.size for p in self.patterns))
        return msum * self.text_bytes


def plain_dna(seed: int = 1, n: int = 1_000_000, m: int = 8, K: int = 2,
              copies: int = 200) -> Workload:
    rng = rng_for(seed)
    pat = iid_dna(rng, m)
    text = iid_dna(rng, n)
    for cp in edit_copies(rng, pat, rng.integers(0, K + 1, size=copies), DNA):
        plant(rng, text, cp)
    return Workload("plain_dna", [pat], np.array([K], np.int32), [text],
                    {"m": m, "K": K, "n": n, "copies": copies})


def dictionary_dna(seed: int = 2, n: int = 256 << 20, n_pat: int = 1024, mlo: int = 8,
                   mhi: int = 32, copies: int = 1000) -> Workload:
    rng = rng_for(seed)
    ms = rng.integers(mlo, mhi + 1, size=n_pat)
    pats = [iid_dna(rng, int(m)) for m in ms]
    ks = (ms // 10).astype(np.int32)
    text = iid_dna(rng, n)
    for pid, p in enumerate(pats):
        for cp in edit_copies(rng, p, np.full(copies, ks[pid]), DNA):
            plant(rng, text, cp)
    return Workload("dictionary_dna", pats, ks, [text],
                    {"n": n, "n_pat": n_pat, "copies": copies, "m_range": [mlo, mhi]})


def bytes_zipf(seed: int = 3, n: int = 1 << 30, n_pat: int = 4096, mlo: int = 16,
               mhi: int = 128, copies: int = 500, s: float = 1.1) -> Workload:
    rng = rng_for(seed)
    perm = rng.permutation(256).astype(np.uint8)
    ms = np.exp(rng.uniform(np.log(mlo), np.log(mhi + 1), size=n_pat)).astype(np.int64)
    ms = ms.clip(mlo, mhi)
    kmax = np.minimum(8, ms // 4)
    ks = np.array([int(rng.integers(1, int(k) + 1)) for k in kmax], np.int32)
    tab = zipf_table(perm, s)
    pats = [zipf_bytes(rng, int(m), perm, s, table=tab) for m in ms]
    text = zipf_bytes(rng, n, perm, s, table=tab)
    alpha = perm  # all 256 byte values
    for pid, p in enumerate(pats):
        for cp in edit_copies(rng, p, rng.integers(1, int(ks[pid]) + 1, size=copies), alpha):
            plant(rng, text, cp)
    return Workload("bytes_zipf", pats, ks, [text],
                    {"n": n, "n_pat": n_pat, "copies": copies, "zipf_s": s})


def many_texts(seed: int = 4, n_texts: int = 10_000, total: float = 4e9, n_pat: int = 512,
               mlo: int = 12, mhi: int = 48, K: int = 3, copies: int = 200,
               sigma: float = 1.75, lo: int = 1000, hi: int = 10_000_000) -> Workload:
    rng = rng_for(seed)
    lens = np.exp(rng.normal(np.log(1e5), sigma, size=n_texts)).astype(np.int64).clip(lo, hi)
    if total:
        lens = (lens * (total / lens.sum())).astype(np.int64).clip(lo, hi)
    ms = rng.integers(mlo, mhi + 1, size=n_pat)
    pats = [iid_dna(rng, int(m)) for m in ms]
    ks = np.full(n_pat, K, np.int32)
    texts = [iid_dna(rng, int(L)) for L in lens]
    for p in pats:
        tids = rng.integers(0, n_texts, size=copies)
        for tid, cp in zip(tids.tolist(), edit_copies(rng, p, rng.integers(0, K + 1, size=copies), DNA)):
            plant(rng, texts[tid], cp)
    return Workload("many_texts", pats, ks, texts,
                    {"n_texts": n_texts, "n_pat": n_pat, "copies": copies, "sigma": sigma})


@dataclass
class ServedTrace:
    """Packet arrivals for online matching, sorted by time.

    Packet j arrives at ``times[j]`` seconds for stream ``streams[j]`` with
    payload ``payload[offs[j]:offs[j] + lens[j]]``; ``last[j]`` marks the last
    packet of its stream (the connection closes after it)."""
    patterns: list
    ks: np.ndarray
    times: np.ndarray
    streams: np.ndarray
    payload: np.ndarray
    offs: np.ndarray
    lens: np.ndarray
    last: np.ndarray
    n_streams: int
    meta: dict = field(default_factory=dict)

    @property
    def n_packets(self) -> int:
        return int(self.times.size)

    def packet(self, j: int) -> np.ndarray:
        return self.payload[self.offs[j]:self.offs[j] + self.lens[j]]

    def stream_texts(self) -> list:
        """Each stream's packets concatenated in arrival order."""
        parts = [[] for _ in range(self.n_streams)]
        for j, sid in enumerate(self.streams.tolist()):
            parts[sid].append(self.packet(j))
        return [np.concatenate(p) if p else np.zeros(0, np.uint8) for p in parts]


def served(seed: int = 5, n_streams: int = 4096, n_sig: int = 2000, mlo: int = 8, mhi: int = 64,
           K: int = 2, gbps: float = 10.0, duration: float = 0.01, plo: int = 64,
           phi: int = 1500, planted_frac: float = 0.01, s: float = 1.1,
           life: float = 1.0, n_packets: int | None = None) -> ServedTrace:
    """Poisson packet arrivals at ``gbps`` (aggregate) over ``duration`` s.

    Each stream is active during a window of ``life * duration`` placed at a
    uniform start; with ``life = 1`` every stream is active throughout and the
    arrivals are a Poisson process.  ``n_packets`` fixes the packet count
    instead (the duration then follows from the rate)."""
    rng = rng_for(seed)
    perm = rng.permutation(256).astype(np.uint8)
    ms = rng.integers(mlo, mhi + 1, size=n_sig)
    tab = zipf_table(perm, s)
    pats = [zipf_bytes(rng, int(m), perm, s, table=tab) for m in ms]
    ks = np.full(n_sig, K, np.int32)
    mean_pkt = (plo + phi) / 2.0
    rate = gbps * 1e9 / 8.0 / mean_pkt  # packets per second
    if n_packets is not None:
        n_pkt = int(n_packets)
        duration = n_pkt / rate
    else:
        n_pkt = max(1, int(rng.poisson(rate * duration)))
    streams = rng.integers(0, n_streams, size=n_pkt).astype(np.int32)
    win = duration * life
    starts = rng.uniform(0.0, max(duration - win, 0.0), size=n_streams)
    times = starts[streams] + rng.uniform(0.0, win, size=n_pkt)
    order = np.argsort(times, kind="stable")
    times, streams = times[order], streams[order]
    lens = rng.integers(plo, phi + 1, size=n_pkt).astype(np.uint32)
    offs = np.concatenate([[0], np.cumsum(lens.astype(np.uint64))[:-1]]).astype(np.uint64)
    payload = zipf_bytes(rng, int(lens.astype(np.int64).sum()), perm, s, table=tab)
    # next packet of the same stream, for copies that straddle a packet boundary
    nxt = np.full(n_pkt, -1, np.int64)
    seen = {}
    for j in range(n_pkt - 1, -1, -1):
        sid = int(streams[j])
        nxt[j] = seen.get(sid, -1)
        seen[sid] = j
    last = nxt < 0
    for j in np.nonzero(rng.random(n_pkt) < planted_frac)[0]:
        pid = int(rng.integers(0, n_sig))
        cp = edit_copy(rng, pats[pid], int(rng.integers(0, K + 1)), perm)
        o, ln = int(offs[j]), int(lens[j])
        if cp.size > ln:
            continue
        if rng.random() < 0.5 and nxt[j] >= 0:
            # the copy starts near the end of this packet and continues in the
            # stream's next packet
            head = int(rng.integers(1, cp.size + 1))
            payload[o + ln - head:o + ln] = cp[:head]
            rest = cp[head:]
            k2 = int(nxt[j])
            take = min(rest.size, int(lens[k2]))
            payload[int(offs[k2]):int(offs[k2]) + take] = rest[:take]
        else:
            at = int(rng.integers(0, ln - cp.size + 1))
            payload[o + at:o + at + cp.size] = cp
    return ServedTrace(pats, ks, times, streams, payload, offs, lens, last, n_streams,
                       {"gbps": gbps, "duration": duration, "n_pkt": n_pkt, "life": life})

"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same inputs and compare element by element."""
import numpy as np

import oracle
from paper_1712_03560_gb300 import binding as B

RULE_NAMES = ("replace", "order", "acc", "cmp")


def gpu_rows(res: np.ndarray):
    return [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
             int(r["len"])) for r in res]


def oracle_rows(patterns, ks, text, rules=None, mode="oasm", threads=None, costs=None):
    """Canonical (pattern_id, decided_at, k, start, len) rows from the oracle."""
    res = oracle.oasm_dictionary(patterns, ks, text, rules, threads=threads, mode=mode,
                                 costs=costs)
    if mode == "hits":  # decided_at is the end for raw hits; order like the library
        pass
    rows = [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]), int(r["start"]),
             int(r["len"])) for r in res]
    return sorted(rows, key=lambda x: (x[0], x[1], x[2], x[3], x[4]))


def canon(rows):
    return sorted(rows, key=lambda x: (x[0], x[1], x[2], x[3], x[4]))


def run_gpu(patterns, ks, text, rules=None, splits=None, device_feed=False, cfg=None,
            costs=None):
    """Feeds `text` as one stream (in pieces when `splits` is given) and ends it."""
    r = dict(rules or {})
    ctx = B.oasm_create(patterns, ks, r or None, cfg, costs=costs)
    try:
        sid = B.oasm_open_stream(ctx)
        text = np.asarray(text, dtype=np.uint8)
        pieces = [text] if splits is None or len(splits) == 0 else np.split(text, splits)
        out = []
        keep = []
        for pc in pieces:
            if device_feed:
                import torch
                t = torch.from_numpy(pc.copy()).cuda()
                keep.append(t)
                B.oasm_feed_device(ctx, sid, t)
            else:
                B.oasm_feed(ctx, sid, pc)
            if splits is not None and len(splits):
                out.append(B.oasm_flush(ctx, sid))  # decisions available so far
        out.append(B.oasm_flush(ctx, sid, end_of_stream=True))
        res = np.concatenate(out)
        return gpu_rows(res), B.oasm_get_stats(ctx)
    finally:
        B.oasm_destroy(ctx)


def random_case(rng, sigma, n_pat, mlo, mhi, n, kmax=None, plant=True):
    alphabet = np.arange(sigma, dtype=np.uint8) if sigma < 256 else np.arange(256, dtype=np.uint8)
    if sigma == 4:
        alphabet = np.frombuffer(b"ACGT", dtype=np.uint8)
    pats, ks = [], []
    for _ in range(n_pat):
        m = int(rng.integers(mlo, mhi + 1))
        pats.append(alphabet[rng.integers(0, alphabet.size, size=m)])
        hi = min(m - 1, kmax if kmax is not None else 3, 15)
        ks.append(int(rng.integers(0, hi + 1)))
    text = alphabet[rng.integers(0, alphabet.size, size=n)]
    if plant and n:
        from paper_1712_03560_gb300 import workloads as Wl
        for p, k in zip(pats, ks):
            for _ in range(int(rng.integers(0, 4))):
                cp = Wl.edit_copy(rng, p, int(rng.integers(0, k + 1)), alphabet)
                Wl.plant(rng, text, cp)
    return pats, ks, text

"""A JSON cache of autotuned launch settings, keyed by the GPU and the pattern
set, so that a context over the same patterns on the same kind of GPU skips
the timing runs of ``oasm_autotune``.

The key covers what decides a context's scan classes and their best settings:
the GPU's name, the histogram of (pattern length, threshold) pairs, the edit
costs and the configuration fields that change the classes.  The value is
the class list of ``oasm_get_tuning``; ``oasm_set_tuning`` checks it against
the new context's classes and rejects a mismatch.
"""
from __future__ import annotations

import hashlib
import json
import os
from collections import Counter


def cache_key(gpu_name: str, patterns, ks, costs=None, cfg: dict | None = None) -> str:
    hist = Counter((len(bytes(p)) if isinstance(p, (bytes, bytearray)) else int(len(p)), int(k))
                   for p, k in zip(patterns, ks))
    cfg = cfg or {}
    doc = {"gpu": gpu_name,
           "hist": sorted([m, k, c] for (m, k), c in hist.items()),
           "costs": list(costs) if costs is not None else None,
           "myers_only": int(cfg.get("myers_only", 0)),
           "prefilter_piece": int(cfg.get("prefilter_piece", 0)),
           "groups_per_warp": int(cfg.get("groups_per_warp", 0))}
    return hashlib.sha1(json.dumps(doc, sort_keys=True).encode()).hexdigest()


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def autotune_cached(lib, ctx, dsample, key: str, path: str | None):
    """Settings from the cache when ``key`` is there (returns "cached"), else
    ``oasm_autotune`` on ``dsample`` and a cache entry (returns "tuned").  With
    no path it only tunes."""
    if path:
        hit = _read(path).get(key)
        if hit is not None:
            try:
                lib.oasm_set_tuning(ctx, hit)
                return "cached"
            except Exception:
                pass  # a stale or foreign entry: tune again and overwrite it
    lib.oasm_autotune(ctx, dsample)
    if path:
        entries = lib.oasm_get_tuning(ctx)
        d = _read(path)
        d[key] = entries
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return "tuned"

"""CPU oracle for OASM (Cinti et al., arXiv:1712.03560) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The product
path (``paper_1712_03560_gb300``) never imports it and shares no code with it:
the C source ``oasm_oracle.c`` is compiled on its own with gcc.

Functions (each follows the passage cited in ``oasm_oracle.c``):
  lev            Eq. 1, full matrix
  lev_prefixes   Eq. 1 column by column from one start (Fig. 1(a))
  sellers        Less Naive column DP (Sec. 5.1)
  hits           the hit set of Eq. 2
  sellers_ends   Less Naive end positions with their distance
  oasm           Algorithm 1 (Sec. 4) with the readings A-G of the C file
  oasm_dictionary  MOASM (Sec. 6.4): one independent Algorithm 1 per pattern

Every function takes ``costs=(sub, ins, del)``: integer edit costs >= 1 in
place of Eq. 1's unit terms (a variant outside the paper; ``ins`` is a text
symbol matched by no pattern symbol, ``del`` a pattern symbol missing from
the text).  ``None`` is the paper's unit-cost distance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oasm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboasm_oracle.so")
_lock = threading.Lock()
_lib = None

REPLACE = {"contained": 0, "same_end": 1, "never": 2}
ORDER = {"per_start_length": 0, "per_start_best": 1}
ACC = {"sum": 0, "last": 1}
CMP = {"gt": 0, "ge": 1}

HIT_DTYPE = np.dtype([("start", "<i8"), ("decided_at", "<i8"), ("len", "<i4"), ("k", "<i4")])
FLUSH_DTYPE = np.dtype([("decided_at", "<i8"), ("start", "<i8"), ("r", "<i8"), ("acc", "<i8"),
                        ("level", "<i4"), ("len", "<i4"), ("kept", "<i4"), ("is_idx", "<i4")])


class _Rules(ctypes.Structure):
    _fields_ = [("replace", ctypes.c_int32), ("order", ctypes.c_int32),
                ("acc", ctypes.c_int32), ("cmp", ctypes.c_int32)]


class _Costs(ctypes.Structure):
    _fields_ = [("sub", ctypes.c_int32), ("ins", ctypes.c_int32), ("del_", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain C11, no architecture flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.orc_lev.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int]
            lib.orc_lev.restype = ctypes.c_int
            lib.orc_lev_prefixes.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, i32p]
            lib.orc_lev_prefixes.restype = None
            lib.orc_sellers.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int64, i32p]
            lib.orc_sellers.restype = None
            for fn in (lib.orc_hits, lib.orc_sellers_ends):
                fn.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int64,
                               ctypes.c_void_p, ctypes.c_int64]
                fn.restype = ctypes.c_int64
            lib.orc_oasm.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int64,
                                     ctypes.POINTER(_Rules), ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int64, i64p]
            lib.orc_oasm.restype = ctypes.c_int64
            cp = ctypes.POINTER(_Costs)
            lib.orc_wlev.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, cp]
            lib.orc_wlev.restype = ctypes.c_int
            lib.orc_wlev_prefixes.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, cp, i32p]
            lib.orc_wlev_prefixes.restype = None
            lib.orc_wsellers.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int64, cp, i32p]
            lib.orc_wsellers.restype = ctypes.c_int
            for fn in (lib.orc_whits, lib.orc_wsellers_ends):
                fn.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int64, cp,
                               ctypes.c_void_p, ctypes.c_int64]
                fn.restype = ctypes.c_int64
            lib.orc_woasm.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int64,
                                      ctypes.POINTER(_Rules), cp, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, i64p]
            lib.orc_woasm.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    elif isinstance(a, str):
        a = np.frombuffer(a.encode("latin-1"), dtype=np.uint8)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8))
    if a.size == 0:  # keep a valid pointer for empty inputs
        a = np.zeros(1, dtype=np.uint8)[:0]
    return a


def _ptr(a: np.ndarray, ctype=ctypes.c_uint8):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _costs(costs):
    """None (unit costs) or a ctypes struct of (sub, ins, del), each an int >= 1."""
    if costs is None:
        return None
    sub, ins, dele = (int(c) for c in costs)
    if min(sub, ins, dele) < 1 or max(sub, ins, dele) > 255:
        raise ValueError("edit costs must be integers in 1..255")
    return _Costs(sub, ins, dele)


def lev(p, s, costs=None) -> int:
    p, s = _u8(p), _u8(s)
    w = _costs(costs)
    if w is None:
        return int(_load().orc_lev(_ptr(p), p.size, _ptr(s), s.size))
    return int(_load().orc_wlev(_ptr(p), p.size, _ptr(s), s.size, ctypes.byref(w)))


def lev_prefixes(p, s, costs=None) -> np.ndarray:
    """out[l] = lev(p, s[:l]) for l = 0..len(s)."""
    p, s = _u8(p), _u8(s)
    out = np.zeros(s.size + 1, dtype=np.int32)
    w = _costs(costs)
    if w is None:
        _load().orc_lev_prefixes(_ptr(p), p.size, _ptr(s), s.size, _ptr(out, ctypes.c_int32))
    else:
        _load().orc_wlev_prefixes(_ptr(p), p.size, _ptr(s), s.size, ctypes.byref(w),
                                  _ptr(out, ctypes.c_int32))
    return out


def sellers(p, t, costs=None) -> np.ndarray:
    p, t = _u8(p), _u8(t)
    out = np.zeros(t.size, dtype=np.int32)
    w = _costs(costs)
    if w is None:
        _load().orc_sellers(_ptr(p), p.size, _ptr(t), t.size, _ptr(out, ctypes.c_int32))
    else:
        _load().orc_wsellers(_ptr(p), p.size, _ptr(t), t.size, ctypes.byref(w),
                             _ptr(out, ctypes.c_int32))
    return out


def _check(p, K):
    if not (1 <= p.size and 0 <= K < p.size):
        raise ValueError("need 1 <= len(p) and 0 <= K < len(p)")


def _collect(fn, p, K, t, cap0=1024, w=None):
    cap = cap0
    while True:
        out = np.zeros(cap, dtype=HIT_DTYPE)
        if w is None:
            n = fn(_ptr(p), p.size, K, _ptr(t), t.size, out.ctypes.data, cap)
        else:
            n = fn(_ptr(p), p.size, K, _ptr(t), t.size, ctypes.byref(w), out.ctypes.data, cap)
        if n < 0:
            raise ValueError("oracle rejected the arguments")
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def hits(p, K: int, t, costs=None) -> np.ndarray:
    """Eq. 2 hit set in (start, len) order; ``decided_at`` holds the end."""
    p, t = _u8(p), _u8(t)
    _check(p, K)
    w = _costs(costs)
    lib = _load()
    return _collect(lib.orc_hits if w is None else lib.orc_whits, p, K, t, w=w)


def sellers_ends(p, K: int, t, costs=None) -> np.ndarray:
    p, t = _u8(p), _u8(t)
    _check(p, K)
    w = _costs(costs)
    lib = _load()
    return _collect(lib.orc_sellers_ends if w is None else lib.orc_wsellers_ends, p, K, t, w=w)


def _rules(replace="contained", order="per_start_length", acc="sum", cmp="gt") -> _Rules:
    return _Rules(REPLACE[replace], ORDER[order], ACC[acc], CMP[cmp])


def oasm(p, K: int, t, rules: dict | None = None, trace: bool = False, costs=None):
    """Algorithm 1 over one finite text.  Returns kept hits (and flush rows)."""
    p, t = _u8(p), _u8(t)
    _check(p, K)
    ru = _rules(**(rules or {}))
    w = _costs(costs)
    lib = _load()
    cap, tcap = 256, 256 if trace else 0
    while True:
        out = np.zeros(cap, dtype=HIT_DTYPE)
        tr = np.zeros(max(tcap, 1), dtype=FLUSH_DTYPE)
        tn = ctypes.c_int64(0)
        if w is None:
            n = lib.orc_oasm(_ptr(p), p.size, K, _ptr(t), t.size, ctypes.byref(ru),
                             out.ctypes.data, cap, tr.ctypes.data if trace else None, tcap,
                             ctypes.byref(tn))
        else:
            n = lib.orc_woasm(_ptr(p), p.size, K, _ptr(t), t.size, ctypes.byref(ru),
                              ctypes.byref(w), out.ctypes.data, cap,
                              tr.ctypes.data if trace else None, tcap, ctypes.byref(tn))
        if n < 0:
            raise ValueError("oracle rejected the arguments")
        if n <= cap and (not trace or tn.value <= tcap):
            res = out[:n].copy()
            return (res, tr[: tn.value].copy()) if trace else res
        cap = max(cap, int(n))
        tcap = max(tcap, int(tn.value)) if trace else 0


def oasm_dictionary(patterns, ks, t, rules: dict | None = None, threads: int | None = None,
                    mode: str = "oasm", costs=None):
    """MOASM: independent Algorithm 1 instances, one per pattern, same text.

    Returns a structured array with a ``pattern_id`` column, sorted by
    (pattern_id, decided_at, k).  ctypes releases the GIL during each call,
    so a thread pool runs the patterns on several host cores.
    """
    t = _u8(t)
    fn = {"oasm": lambda p, k: oasm(p, k, t, rules, costs=costs),
          "hits": lambda p, k: hits(p, k, t, costs=costs),
          "ends": lambda p, k: sellers_ends(p, k, t, costs=costs)}[mode]
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda a: fn(_u8(a[0]), int(a[1])), zip(patterns, ks)))
    dt = np.dtype([("pattern_id", "<i4")] + [(n, HIT_DTYPE[n]) for n in HIT_DTYPE.names])
    total = sum(len(x) for x in parts)
    res = np.zeros(total, dtype=dt)
    o = 0
    for pid, x in enumerate(parts):
        res[o:o + len(x)]["pattern_id"] = pid
        for n in HIT_DTYPE.names:
            res[o:o + len(x)][n] = x[n]
        o += len(x)
    order = np.lexsort((res["k"], res["decided_at"], res["pattern_id"]))
    return res[order]

"""Thin Python binding of the OASM C ABI (``include/oasm.h``).

Argument marshalling only: every step of the matching path runs in the CUDA
library ``_build/liboasm.so``.  The functions keep the C names.  There is no
fallback: if the library cannot be loaded, or no CUDA device is present,
the calls raise ``OasmError``.

Device memory for ``oasm_feed_device`` may be given as a torch CUDA tensor
(uint8) or as a raw integer device pointer.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OASM_OK = 0
OASM_EINVAL = -1
OASM_ENOMEM = -2
OASM_EBUSY = -3
OASM_ETRUNC = -4
OASM_ETIMEOUT = -5
OASM_ECUDA = -6
OASM_ESTATE = -7
OASM_ALL_STREAMS = 0xFFFFFFFF  # oasm_ready: total over every open stream

REPLACE = {"contained": 0, "same_end": 1, "never": 2}
ORDER = {"per_start_length": 0, "per_start_best": 1}
ACC = {"sum": 0, "last": 1}
CMP = {"gt": 0, "ge": 1}
OUTPUT = {"filtered": 0, "ends": 1, "all_hits": 2}

HIT_DTYPE = np.dtype([("pattern_id", "<u4"), ("k", "<u4"), ("start", "<u8"), ("len", "<u4"),
                      ("stream_id", "<u4"), ("decided_at", "<u8")])
END_DTYPE = np.dtype([("pattern_id", "<u4"), ("k", "<u4"), ("end", "<u8")])


class OasmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class oasm_rules(ctypes.Structure):
    _fields_ = [("replace", ctypes.c_int32), ("order", ctypes.c_int32), ("acc", ctypes.c_int32),
                ("cmp", ctypes.c_int32), ("output", ctypes.c_int32)]


class oasm_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_streams", ctypes.c_uint32),
                ("mem_budget", ctypes.c_uint64), ("region_bytes", ctypes.c_uint32),
                ("tile_warps", ctypes.c_uint32), ("timing", ctypes.c_int32),
                ("flush_timeout_ms", ctypes.c_uint32), ("cuda_stream", ctypes.c_void_p),
                ("myers_only", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("groups_per_warp", ctypes.c_uint32), ("prefilter_piece", ctypes.c_uint32),
                ("full_words", ctypes.c_int32), ("record_order", ctypes.c_int32)]


class oasm_hit(ctypes.Structure):
    _fields_ = [("pattern_id", ctypes.c_uint32), ("k", ctypes.c_uint32), ("start", ctypes.c_uint64),
                ("len", ctypes.c_uint32), ("stream_id", ctypes.c_uint32),
                ("decided_at", ctypes.c_uint64)]


assert ctypes.sizeof(oasm_hit) == HIT_DTYPE.itemsize == 32


class oasm_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("steps", "launches", "text_bytes", "cells",
                                                "word_steps", "candidates", "hits", "kept",
                                                "reruns")] + \
               [(n, ctypes.c_double) for n in ("scan_ms", "verify_ms", "order_ms", "filter_ms",
                                               "copy_ms", "step_ms")] + \
               [("scan_launches", ctypes.c_uint64), ("graph_builds", ctypes.c_uint64),
                ("prefilter_ms", ctypes.c_double), ("prefilter_candidates", ctypes.c_uint64),
                ("host_plan_ms", ctypes.c_double), ("host_launch_ms", ctypes.c_double),
                ("host_wait_ms", ctypes.c_double), ("host_post_ms", ctypes.c_double),
                ("buffer_grows", ctypes.c_uint64), ("host_copy_ms", ctypes.c_double),
                ("record_bytes", ctypes.c_uint64)]


class oasm_costs(ctypes.Structure):
    _fields_ = [("sub", ctypes.c_uint32), ("ins", ctypes.c_uint32), ("del_", ctypes.c_uint32)]


class oasm_tuning(ctypes.Structure):
    _fields_ = [("words", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("groups_per_warp", ctypes.c_int32), ("warps", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("region_scale", ctypes.c_float)]


class oasm_trace(ctypes.Structure):
    _fields_ = [("t", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("off", ctypes.c_void_p),
                ("len", ctypes.c_void_p), ("last", ctypes.c_void_p), ("payload", ctypes.c_void_p),
                ("n_packets", ctypes.c_uint64), ("n_streams", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_szp = ctypes.POINTER(ctypes.c_size_t)
SERVE_OP_TYPES = {
    "open_streams": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32, _u32p, _u32p),
    "feed_many": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32, _u32p,
                                  ctypes.POINTER(ctypes.c_uint8), _u64p, _u32p),
    "end_streams": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32, _u32p),
    "close_streams": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32, _u32p),
    "step_begin": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p),
    "step_end": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p),
    "ready": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32, _szp),
    "drain": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                              _szp),
    "get_stats": ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p),
}


class oasm_serve_ops(ctypes.Structure):
    _fields_ = [("handle", ctypes.c_void_p)] + [(k, t) for k, t in SERVE_OP_TYPES.items()]


class oasm_replay_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("steps", "packets", "bytes", "kept", "n_out",
                                                "streams_admitted", "max_waiting_streams")] + \
               [(n, ctypes.c_double) for n in ("wall_s", "step_s_sum", "step_s_max")] + \
               [(n, ctypes.c_uint64) for n in ("reruns", "graph_builds", "buffer_grows",
                                                "slowest_step", "slowest_bytes", "slowest_reruns",
                                                "slowest_graph_builds", "slowest_buffer_grows")]


EXPORTS = ["oasm_config_default", "oasm_rules_default", "oasm_create", "oasm_create_weighted",
           "oasm_destroy",
           "oasm_open_stream", "oasm_close_stream", "oasm_open_streams", "oasm_end_streams",
           "oasm_close_streams", "oasm_feed", "oasm_feed_many", "oasm_feed_device",
           "oasm_end_stream", "oasm_step", "oasm_flush", "oasm_drain", "oasm_ready", "oasm_get_stats", "oasm_reset_stats",
           "oasm_cuda_stream", "oasm_last_error", "oasm_strerror", "oasm_autotune",
           "oasm_measure_int_peak", "oasm_measure_int_peak_mix", "oasm_scan_ends_noalloc",
           "oasm_stream_state_size",
           "oasm_save_stream", "oasm_restore_stream", "oasm_replay", "oasm_register_host",
           "oasm_unregister_host", "oasm_step_begin", "oasm_step_end", "oasm_replay_ops",
           "oasm_piece_filter_choice", "oasm_selftest_wait", "oasm_get_tuning",
           "oasm_set_tuning"]

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Loads liboasm.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.build()
        if not os.path.exists(path):
            raise OasmError(OASM_ECUDA, f"CUDA library {path} is missing")
        lib = ctypes.CDLL(path)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        u8pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "oasm_config_default": ([ctypes.POINTER(oasm_config)], i32),
            "oasm_rules_default": ([ctypes.POINTER(oasm_rules)], i32),
            "oasm_create": ([u8pp, ctypes.POINTER(u32), ctypes.POINTER(u32), u32,
                             ctypes.POINTER(oasm_rules), ctypes.POINTER(oasm_config),
                             ctypes.POINTER(vp)], i32),
            "oasm_create_weighted": ([u8pp, ctypes.POINTER(u32), ctypes.POINTER(u32), u32,
                                      ctypes.POINTER(oasm_rules), ctypes.POINTER(oasm_costs),
                                      ctypes.POINTER(oasm_config), ctypes.POINTER(vp)], i32),
            "oasm_destroy": ([vp], i32),
            "oasm_open_stream": ([vp, ctypes.POINTER(u32)], i32),
            "oasm_close_stream": ([vp, u32], i32),
            "oasm_feed": ([vp, u32, vp, ctypes.c_size_t], i32),
            "oasm_open_streams": ([vp, u32, vp, ctypes.POINTER(u32)], i32),
            "oasm_end_streams": ([vp, u32, vp], i32),
            "oasm_close_streams": ([vp, u32, vp], i32),
            "oasm_feed_device": ([vp, u32, vp, ctypes.c_size_t], i32),
            "oasm_feed_many": ([vp, u32, vp, vp, vp, vp], i32),
            "oasm_drain": ([vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], i32),
            "oasm_end_stream": ([vp, u32], i32),
            "oasm_step": ([vp], i32),
            "oasm_step_begin": ([vp], i32),
            "oasm_step_end": ([vp], i32),
            "oasm_flush": ([vp, u32, i32, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], i32),
            "oasm_ready": ([vp, u32, ctypes.POINTER(ctypes.c_size_t)], i32),
            "oasm_get_stats": ([vp, ctypes.POINTER(oasm_stats)], i32),
            "oasm_reset_stats": ([vp], i32),
            "oasm_cuda_stream": ([vp], vp),
            "oasm_last_error": ([vp], ctypes.c_char_p),
            "oasm_strerror": ([i32], ctypes.c_char_p),
            "oasm_autotune": ([vp, vp, ctypes.c_size_t, ctypes.c_char_p, ctypes.c_size_t], i32),
            "oasm_selftest_wait": ([i32, u32, i32], i32),
            "oasm_get_tuning": ([vp, ctypes.POINTER(oasm_tuning), u32, ctypes.POINTER(u32)], i32),
            "oasm_set_tuning": ([vp, ctypes.POINTER(oasm_tuning), u32], i32),
            "oasm_measure_int_peak": ([i32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)], i32),
            "oasm_measure_int_peak_mix": ([i32, i32, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)], i32),
            "oasm_stream_state_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], i32),
            "oasm_save_stream": ([vp, u32, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], i32),
            "oasm_restore_stream": ([vp, u32, vp, ctypes.c_size_t], i32),
            "oasm_scan_ends_noalloc": ([u8pp, ctypes.POINTER(u32), ctypes.POINTER(u32), u32, vp,
                                        u64, vp, u64, ctypes.POINTER(u64), vp], i32),
            "oasm_replay": ([vp, ctypes.POINTER(oasm_trace), i32, u64, vp, vp, ctypes.c_size_t,
                             ctypes.POINTER(oasm_replay_stats)], i32),
            "oasm_replay_ops": ([ctypes.POINTER(oasm_serve_ops), ctypes.POINTER(oasm_trace), i32,
                                 u64, vp, vp, ctypes.c_size_t,
                                 ctypes.POINTER(oasm_replay_stats)], i32),
            "oasm_register_host": ([vp, vp, ctypes.c_size_t], i32),
            "oasm_piece_filter_choice": ([u8pp, ctypes.POINTER(u32), ctypes.POINTER(u32), u32, u32,
                                          vp], i32),
            "oasm_unregister_host": ([vp, vp], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, ctx=None, allow=()):
    if rc < 0 and rc not in allow:
        lib = load()
        msg = lib.oasm_last_error(ctx).decode() if lib else ""
        raise OasmError(rc, msg or lib.oasm_strerror(rc).decode())
    return rc


def oasm_rules_make(replace="contained", order="per_start_length", acc="sum", cmp="gt",
                    output="filtered") -> oasm_rules:
    return oasm_rules(REPLACE[replace], ORDER[order], ACC[acc], CMP[cmp], OUTPUT[output])


def oasm_config_make(**kw) -> oasm_config:
    cfg = oasm_config()
    load().oasm_config_default(ctypes.byref(cfg))
    names = {f[0] for f in oasm_config._fields_}
    for k, v in kw.items():
        if k not in names:
            raise KeyError(f"oasm_config has no field {k!r}")
        setattr(cfg, k, v)
    return cfg


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    if isinstance(a, str):
        return np.frombuffer(a.encode("latin-1"), dtype=np.uint8)
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def oasm_create(patterns, ks, rules: oasm_rules | dict | None = None,
                cfg: oasm_config | dict | None = None, costs=None):
    """costs: None (unit costs, oasm_create) or (sub, ins, del), which calls
    oasm_create_weighted."""
    lib = load()
    pats = [_u8(p) for p in patterns]
    n = len(pats)
    ptrs = (ctypes.c_void_p * n)(*[p.ctypes.data for p in pats])
    lens = (ctypes.c_uint32 * n)(*[p.size for p in pats])
    kk = (ctypes.c_uint32 * n)(*[int(k) for k in ks])
    if isinstance(rules, dict):
        rules = oasm_rules_make(**rules)
    if isinstance(cfg, dict):
        cfg = oasm_config_make(**cfg)
    ctx = ctypes.c_void_p()
    if costs is None:
        rc = lib.oasm_create(ptrs, lens, kk, n, ctypes.byref(rules) if rules else None,
                             ctypes.byref(cfg) if cfg else None, ctypes.byref(ctx))
    else:
        w = oasm_costs(*(int(c) for c in costs))
        rc = lib.oasm_create_weighted(ptrs, lens, kk, n, ctypes.byref(rules) if rules else None,
                                      ctypes.byref(w), ctypes.byref(cfg) if cfg else None,
                                      ctypes.byref(ctx))
    _check(rc, None)
    return ctx


def oasm_destroy(ctx):
    return _check(load().oasm_destroy(ctx), None)


def oasm_open_stream(ctx) -> int:
    sid = ctypes.c_uint32()
    _check(load().oasm_open_stream(ctx, ctypes.byref(sid)), ctx)
    return sid.value


def oasm_close_stream(ctx, sid: int):
    return _check(load().oasm_close_stream(ctx, sid), ctx)


def oasm_open_streams(ctx, n: int) -> np.ndarray:
    """Up to n new stream ids (fewer when slots or memory run out)."""
    sids = np.zeros(max(n, 1), dtype=np.uint32)
    got = ctypes.c_uint32(0)
    _check(load().oasm_open_streams(ctx, n, sids.ctypes.data, ctypes.byref(got)), ctx)
    return sids[: got.value]


def oasm_end_streams(ctx, sids):
    sids = np.ascontiguousarray(sids, dtype=np.uint32)
    return _check(load().oasm_end_streams(ctx, sids.size, sids.ctypes.data), ctx)


def oasm_close_streams(ctx, sids):
    sids = np.ascontiguousarray(sids, dtype=np.uint32)
    return _check(load().oasm_close_streams(ctx, sids.size, sids.ctypes.data), ctx)


def oasm_feed(ctx, sid: int, chunk):
    a = _u8(chunk)
    return _check(load().oasm_feed(ctx, sid, a.ctypes.data if a.size else None, a.size), ctx)


def oasm_feed_many(ctx, sids, buf, offs, lens):
    """Packets j = buf[offs[j] : offs[j] + lens[j]] for streams sids[j]."""
    sids = np.ascontiguousarray(sids, dtype=np.uint32)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    lens = np.ascontiguousarray(lens, dtype=np.uint32)
    buf = _u8(buf)
    n = sids.size
    if n == 0:
        return 0
    return _check(load().oasm_feed_many(ctx, n, sids.ctypes.data, buf.ctypes.data,
                                        offs.ctypes.data, lens.ctypes.data), ctx)


def _dev_ptr(d):
    if isinstance(d, int):
        return d
    if hasattr(d, "data_ptr"):
        if not d.is_cuda or not d.is_contiguous():
            raise OasmError(OASM_EINVAL, "need a contiguous CUDA tensor")
        return d.data_ptr()
    raise OasmError(OASM_EINVAL, "device chunk must be a CUDA tensor or a device pointer")


def oasm_feed_device(ctx, sid: int, dchunk, n: int | None = None):
    if n is None:
        n = dchunk.numel() * dchunk.element_size()
    return _check(load().oasm_feed_device(ctx, sid, _dev_ptr(dchunk), n), ctx)


def oasm_end_stream(ctx, sid: int):
    return _check(load().oasm_end_stream(ctx, sid), ctx)


def oasm_step(ctx):
    return _check(load().oasm_step(ctx), ctx)


def oasm_step_begin(ctx):
    return _check(load().oasm_step_begin(ctx), ctx)


def oasm_step_end(ctx):
    return _check(load().oasm_step_end(ctx), ctx)


def oasm_drain(ctx, out: np.ndarray | None = None) -> np.ndarray:
    """All queued hits of all streams (streams in id order, canonical order
    within a stream).  With ``out`` (a HIT_DTYPE array), the hits are written
    into it when it is large enough and a view of it is returned."""
    lib = load()
    total = oasm_ready(ctx, OASM_ALL_STREAMS)
    if out is not None and out.dtype == HIT_DTYPE and out.size >= total and out.flags.c_contiguous:
        buf = out[:total]
    else:
        buf = np.empty(total, dtype=HIT_DTYPE)
    n = ctypes.c_size_t(0)
    rc = lib.oasm_drain(ctx, buf.ctypes.data if total else None, total, ctypes.byref(n))
    _check(rc, ctx)
    return buf[: n.value]


def oasm_ready(ctx, sid: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().oasm_ready(ctx, sid, ctypes.byref(n)), ctx)
    return n.value


def oasm_flush(ctx, sid: int, end_of_stream: bool = False) -> np.ndarray:
    """Every hit of the stream decided so far, in canonical order.

    The first call runs any pending step with no output buffer; the second
    copies the whole queue into one array sized by ``oasm_ready``."""
    lib = load()
    n = ctypes.c_size_t(0)
    rc = lib.oasm_flush(ctx, sid, 1 if end_of_stream else 0, None, 0, ctypes.byref(n))
    _check(rc, ctx, allow=(OASM_ETRUNC,))
    if rc != OASM_ETRUNC:
        return np.zeros(0, dtype=HIT_DTYPE)
    cnt = oasm_ready(ctx, sid)
    buf = np.zeros(cnt, dtype=HIT_DTYPE)
    rc = lib.oasm_flush(ctx, sid, 0, buf.ctypes.data, cnt, ctypes.byref(n))
    _check(rc, ctx)
    return buf[: n.value]


def oasm_get_stats(ctx) -> dict:
    st = oasm_stats()
    _check(load().oasm_get_stats(ctx, ctypes.byref(st)), ctx)
    return {n: getattr(st, n) for n, _ in oasm_stats._fields_}


def oasm_reset_stats(ctx):
    return _check(load().oasm_reset_stats(ctx), ctx)


def oasm_cuda_stream(ctx) -> int:
    return load().oasm_cuda_stream(ctx) or 0


def oasm_autotune(ctx, dsample, n: int | None = None) -> str:
    if n is None:
        n = dsample.numel()
    buf = ctypes.create_string_buffer(65536)
    _check(load().oasm_autotune(ctx, _dev_ptr(dsample), n, buf, 65536), ctx)
    return buf.value.decode()


def oasm_measure_int_peak(device: int = 0):
    """(integer ops per second, ms of the best launch) of the scan's op mix."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().oasm_measure_int_peak(device, ctypes.byref(ops), ctypes.byref(ms)))
    return ops.value, ms.value


INT_MIXES = {"alu": 0, "multiply_add": 1, "scan_step": 2, "weighted_step": 3}


def oasm_measure_int_peak_mix(device: int = 0, mix: str = "scan_step"):
    """(integer ops per second, ms of the best launch) of one mix of
    INT_MIXES: the ALU pipe alone, integer multiply-adds alone, the scan's
    column step, or the weighted wave-front's cell pairs."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().oasm_measure_int_peak_mix(device, INT_MIXES[mix], ctypes.byref(ops),
                                            ctypes.byref(ms)))
    return ops.value, ms.value


TUNING_FIELDS = ("words", "algo", "groups_per_warp", "warps", "chunk", "region_scale")


def oasm_get_tuning(ctx) -> list:
    """Launch settings of every scan class, as dicts of TUNING_FIELDS."""
    lib = load()
    n = ctypes.c_uint32(0)
    rc = lib.oasm_get_tuning(ctx, None, 0, ctypes.byref(n))
    if rc not in (OASM_OK, OASM_ETRUNC):
        _check(rc, ctx)
    arr = (oasm_tuning * max(1, n.value))()
    _check(lib.oasm_get_tuning(ctx, arr, n.value, ctypes.byref(n)), ctx)
    return [{f: getattr(arr[i], f) for f in TUNING_FIELDS} for i in range(n.value)]


def oasm_set_tuning(ctx, entries):
    arr = (oasm_tuning * max(1, len(entries)))()
    for i, e in enumerate(entries):
        for f in TUNING_FIELDS:
            setattr(arr[i], f, e[f])
    return _check(load().oasm_set_tuning(ctx, arr, len(entries)), ctx)


def oasm_selftest_wait(device: int = 0, spin_limit: int = 1 << 16, arrive: bool = False) -> int:
    """Bounded-wait self-test: the library's status code (OASM_ETIMEOUT when
    nothing completes the barrier, OASM_OK when it completes)."""
    return int(load().oasm_selftest_wait(device, spin_limit, 1 if arrive else 0))


def _check_device_buffer(d, need_bytes: int, what: str):
    """A contiguous CUDA tensor on the current device holding need_bytes."""
    import torch
    if not hasattr(d, "data_ptr") or not d.is_cuda or not d.is_contiguous():
        raise OasmError(OASM_EINVAL, f"{what} must be a contiguous CUDA tensor")
    if d.device.index != torch.cuda.current_device():
        raise OasmError(OASM_EINVAL, f"{what} is on cuda:{d.device.index}, the current "
                                     f"device is cuda:{torch.cuda.current_device()}")
    have = d.numel() * d.element_size()
    if need_bytes > have:
        raise OasmError(OASM_EINVAL, f"{what} holds {have} bytes, the call needs {need_bytes}")


def oasm_scan_ends_noalloc(patterns, ks, d_text, d_out, cap: int, n: int | None = None,
                           stream: int | None = None) -> int:
    """Less Naive ends of up to 64 patterns over a device text, allocating no
    device memory (for callers that cannot allocate: see include/oasm.h).

    ``d_text`` is a CUDA tensor of at least ``n`` bytes (default: all of it)
    and ``d_out`` one of at least ``cap`` records of ``END_DTYPE`` (16 bytes
    each), both on the current device; anything smaller is rejected here, so
    the kernel never reads or writes past them.  ``stream`` is a
    cudaStream_t handle; by default torch's current stream, the one the
    caller's tensors were filled on.  Returns the number of ends found, which
    may exceed ``cap`` (then only ``cap`` were written)."""
    import torch
    lib = load()
    pats = [_u8(p) for p in patterns]
    m = len(pats)
    ptrs = (ctypes.c_void_p * m)(*[p.ctypes.data for p in pats])
    lens = (ctypes.c_uint32 * m)(*[p.size for p in pats])
    kk = (ctypes.c_uint32 * m)(*[int(k) for k in ks])
    if n is None:
        n = d_text.numel() * d_text.element_size()
    if n < 0 or cap < 0:
        raise OasmError(OASM_EINVAL, "n and cap must be >= 0")
    _check_device_buffer(d_text, n, "d_text")
    _check_device_buffer(d_out, cap * END_DTYPE.itemsize, "d_out")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    found = ctypes.c_uint64(0)
    rc = lib.oasm_scan_ends_noalloc(ptrs, lens, kk, m, _dev_ptr(d_text) if n else None, n,
                                    _dev_ptr(d_out) if cap else None, cap, ctypes.byref(found),
                                    stream or None)
    if rc < 0 and rc != OASM_ETRUNC:
        raise OasmError(rc, lib.oasm_strerror(rc).decode())
    return found.value


def oasm_save_stream(ctx, sid: int) -> bytes:
    """The stream's matching state (position, stored tail, pending windows)."""
    lib = load()
    n = ctypes.c_size_t(0)
    _check(lib.oasm_stream_state_size(ctx, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.oasm_save_stream(ctx, sid, buf, n.value, ctypes.byref(n)), ctx)
    return buf.raw[: n.value]


def oasm_restore_stream(ctx, sid: int, state: bytes):
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    return _check(load().oasm_restore_stream(ctx, sid, buf, len(state)), ctx)


def oasm_strerror(code: int) -> str:
    return load().oasm_strerror(code).decode()


def oasm_last_error(ctx=None) -> str:
    return load().oasm_last_error(ctx).decode()


def oasm_piece_filter_choice(patterns, ks, prefilter_piece: int) -> np.ndarray:
    """Boolean per pattern: searched by the piece filter (True) or the scan
    under cfg.prefilter_piece = prefilter_piece (host-only, no device)."""
    arrs = [_u8(p) for p in patterns]
    n = len(arrs)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in arrs])
    lens = (ctypes.c_uint32 * max(n, 1))(*[a.size for a in arrs])
    kk = (ctypes.c_uint32 * max(n, 1))(*[int(k) for k in ks])
    out = np.zeros(max(n, 1), dtype=np.uint8)
    _check(load().oasm_piece_filter_choice(ptrs, lens, kk, n, int(prefilter_piece),
                                           out.ctypes.data))
    return out[:n].astype(bool)


def oasm_register_host(ctx, buf: np.ndarray):
    """Pins and maps a host array for zero-copy feeds; keep ``buf`` alive and
    unchanged until oasm_unregister_host."""
    if not (isinstance(buf, np.ndarray) and buf.flags.c_contiguous and buf.nbytes):
        raise ValueError("need a non-empty C-contiguous numpy array")
    return _check(load().oasm_register_host(ctx, buf.ctypes.data, buf.nbytes), ctx)


def oasm_unregister_host(ctx, buf: np.ndarray):
    return _check(load().oasm_unregister_host(ctx, buf.ctypes.data), ctx)


def oasm_replay(ctx, times, streams, offs, lens, last, payload, n_streams: int,
                realtime: bool = True, max_batch_bytes: int = 32 << 20, collect: bool = False,
                out_cap: int | None = None):
    """Runs the native serving loop over a packet trace.  Returns (done_at,
    hits, stats): done_at[q] = seconds from the start to the end of the step
    that matched packet q (NaN if never fed), hits = the drained records
    (external stream ids) when ``collect``, stats = the loop's counters."""
    t = np.ascontiguousarray(times, dtype=np.float64)
    st_ = np.ascontiguousarray(streams, dtype=np.uint32)
    of = np.ascontiguousarray(offs, dtype=np.uint64)
    ln = np.ascontiguousarray(lens, dtype=np.uint32)
    la = np.ascontiguousarray(last, dtype=np.uint8)
    pay = _u8(payload)
    n = t.size
    tr = oasm_trace(t.ctypes.data, st_.ctypes.data, of.ctypes.data, ln.ctypes.data,
                    la.ctypes.data, pay.ctypes.data, n, int(n_streams), 0)
    done = np.full(n, np.nan)
    cap = 0
    out = None
    if collect:
        cap = int(out_cap) if out_cap is not None else max(1 << 16, n * 4)
        out = np.empty(cap, dtype=HIT_DTYPE)
    rs = oasm_replay_stats()
    rc = load().oasm_replay(ctx, ctypes.byref(tr), 1 if realtime else 0, int(max_batch_bytes),
                            done.ctypes.data, out.ctypes.data if out is not None else None, cap,
                            ctypes.byref(rs))
    _check(rc, ctx, allow=(OASM_ETRUNC,))
    stats = {f[0]: getattr(rs, f[0]) for f in oasm_replay_stats._fields_}
    if rc == OASM_ETRUNC:
        raise OasmError(rc, f"replay kept {stats['kept']} hits, more than out_cap={cap}")
    hits = out[: rs.n_out] if out is not None else None
    return done, hits, stats


def oasm_replay_ops(ops: dict, times, streams, offs, lens, last, payload, n_streams: int,
                    realtime: bool = False, max_batch_bytes: int = 32 << 20):
    """The native serving loop driven through a table of Python callables
    (keys of SERVE_OP_TYPES, each taking the C arguments after the handle;
    get_stats may be left out) instead of a context.  Returns (rc, done_at,
    stats); the loop's own error code is returned, not raised."""
    cb = {k: SERVE_OP_TYPES[k](lambda *a, f=f: int(f(*a[1:]))) for k, f in ops.items()}
    table = oasm_serve_ops(None, *[cb.get(k, SERVE_OP_TYPES[k]()) for k in SERVE_OP_TYPES])
    t = np.ascontiguousarray(times, dtype=np.float64)
    st_ = np.ascontiguousarray(streams, dtype=np.uint32)
    of = np.ascontiguousarray(offs, dtype=np.uint64)
    ln = np.ascontiguousarray(lens, dtype=np.uint32)
    la = np.ascontiguousarray(last, dtype=np.uint8)
    pay = _u8(payload)
    n = t.size
    tr = oasm_trace(t.ctypes.data, st_.ctypes.data, of.ctypes.data, ln.ctypes.data,
                    la.ctypes.data, pay.ctypes.data, n, int(n_streams), 0)
    done = np.full(n, np.nan)
    rs = oasm_replay_stats()
    rc = load().oasm_replay_ops(ctypes.byref(table), ctypes.byref(tr), 1 if realtime else 0,
                                int(max_batch_bytes), done.ctypes.data, None, 0,
                                ctypes.byref(rs))
    stats = {f[0]: getattr(rs, f[0]) for f in oasm_replay_stats._fields_}
    return int(rc), done, stats


class Matcher:
    """Convenience owner of one context (still marshalling only)."""

    def __init__(self, patterns, ks, rules=None, costs=None, **cfg):
        self.ctx = oasm_create(patterns, ks, rules, cfg or None, costs=costs)

    def close(self):
        if self.ctx is not None:
            oasm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def search(self, text, device=False) -> np.ndarray:
        """One whole text as one stream: feed, end, flush."""
        sid = oasm_open_stream(self.ctx)
        try:
            if device:
                oasm_feed_device(self.ctx, sid, text)
            else:
                oasm_feed(self.ctx, sid, text)
            return oasm_flush(self.ctx, sid, end_of_stream=True)
        finally:
            oasm_close_stream(self.ctx, sid)

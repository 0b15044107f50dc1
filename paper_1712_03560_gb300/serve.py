"""Online matching of many concurrent byte streams (the serving loop).

Packets of many streams arrive over time.  The server runs the device path in
batched steps with continuous batching:

* every step takes all packets that have arrived so far (up to a byte
  budget), hands them to the library in one ``oasm_feed_many`` call, runs one
  ``oasm_step`` (the whole device path over every stream that has new bytes)
  and drains the decided hits of all streams with one ``oasm_drain``;
* packets that arrive while a step is on the GPU go into the next step;
* each stream's bit-vector state (as its stored tail) and pending filter
  windows stay resident on the device between steps;
* a stream is admitted when its first packet arrives if a stream slot and
  the device memory budget allow it; otherwise it waits (its packets are
  kept in arrival order) and is admitted when a closing stream frees a slot;
* a stream closes after its last packet: the step that ingests that packet
  also ends the stream, decides its pending windows and frees the slot.

Latency of a packet = time from its arrival to the end of the step that
matched it (all hits it makes decidable are on the host by then).

The scheduler is plain host logic; all matching runs in the CUDA library.
"""
from __future__ import annotations

import collections
import time

import numpy as np


class Server:
    def __init__(self, patterns, ks, max_streams: int = 4096, mem_budget: int = 0, rules=None,
                 device: int = 0, max_batch_bytes: int = 8 << 20, graphs: bool = True,
                 timing: bool = False, prefilter_piece: int = 0, lib=None, costs=None):
        if lib is None:
            from . import binding as lib
        self.B = lib
        # costs: integer edit costs (sub, ins, del) select the weighted path
        kw = {} if costs is None else {"costs": tuple(costs)}
        self.ctx = lib.oasm_create(patterns, ks, rules,
                                   {"device": device, "max_streams": max_streams,
                                    "mem_budget": mem_budget, "graphs": 1 if graphs else 0,
                                    "timing": 1 if timing else 0,
                                    "prefilter_piece": int(prefilter_piece)}, **kw)
        self.max_batch_bytes = int(max_batch_bytes)

    def stats(self) -> dict:
        """The library's counters (steps, launches, scan time with timing on)."""
        return self.B.oasm_get_stats(self.ctx)

    def reset_stats(self):
        self.B.oasm_reset_stats(self.ctx)

    def close(self):
        if self.ctx is not None:
            self.B.oasm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _admit_many(self, n: int):
        """Up to n new library stream ids (fewer when slots or memory run out)."""
        return self.B.oasm_open_streams(self.ctx, n).tolist() if n else []

    def replay(self, tr, realtime: bool = True, collect: bool = False,
               engine: str = "python", zero_copy: bool = False) -> dict:
        """Replays a ``workloads.ServedTrace``; returns latency/throughput stats.

        With ``realtime`` the packets become visible at their arrival times;
        otherwise all of them are present at the start (pure throughput).
        With ``collect`` the hits of each stream are returned under ``hits``
        (one structured array per external stream id).  ``engine="native"``
        runs the same scheduler inside the library (``oasm_replay``).  With
        ``zero_copy`` the trace's payload is registered with the library for
        the replay, and the device reads packets straight from it."""
        if zero_copy:
            payload = np.ascontiguousarray(tr.payload, dtype=np.uint8)
            self.B.oasm_register_host(self.ctx, payload)
            try:
                if payload is not tr.payload:
                    import dataclasses
                    tr = dataclasses.replace(tr, payload=payload)
                return self.replay(tr, realtime, collect, engine, zero_copy=False)
            finally:
                self.B.oasm_unregister_host(self.ctx, payload)
        if engine == "native":
            return self._replay_native(tr, realtime, collect)
        B = self.B
        n = tr.n_packets
        times = np.asarray(tr.times, dtype=np.float64)
        streams = np.asarray(tr.streams, dtype=np.int64)
        lens = np.asarray(tr.lens, dtype=np.int64)
        offs = np.asarray(tr.offs, dtype=np.uint64)
        last = np.asarray(tr.last, dtype=bool)
        sid_of = np.full(tr.n_streams, -1, np.int64)   # -1 new, >=0 library sid, -2 closed
        ext_of = {}                                      # library sid -> external id
        waiting = collections.deque()                    # external ids waiting for a slot
        held = collections.defaultdict(list)             # packets of waiting streams
        done_at = np.full(n, np.nan)
        csum = np.cumsum(lens)                          # bytes of packets [0, q]
        hits = collections.defaultdict(list) if collect else None
        steps = 0
        kept = 0
        fed_bytes = 0
        max_wait = 0
        admitted = 0
        step_ms = []
        phase = {"schedule": 0.0, "feed": 0.0, "step_drain": 0.0, "close": 0.0}
        t0 = time.perf_counter()
        i = 0
        while i < n or waiting or held:
            t_it = time.perf_counter()
            now = t_it - t0
            if realtime:
                j = int(np.searchsorted(times, now, side="right"))
            else:
                j = n
            # admit waiting streams first (slots freed by the last step)
            parts = []
            if waiting:
                for sid in self._admit_many(len(waiting)):
                    ext = waiting.popleft()
                    sid_of[ext] = sid
                    ext_of[sid] = ext
                    admitted += 1
                    got = held.pop(ext, None)
                    if got:
                        parts.append(np.asarray(got, dtype=np.int64))
            # newly arrived packets, within the byte budget
            used = int(sum(int(lens[p].sum()) for p in parts))
            budget = self.max_batch_bytes - used
            k = i
            if j > i:
                before = int(csum[i - 1]) if i else 0
                k = int(np.searchsorted(csum, before + budget, side="right"))
                k = min(j, max(i + 1, k))
            if k > i:
                exts = streams[i:k]
                # streams seen for the first time: admit now or queue (in arrival order)
                fresh = exts[sid_of[exts] == -1]
                if fresh.size:
                    _, first = np.unique(fresh, return_index=True)
                    order = fresh[np.sort(first)].tolist()
                    got = self._admit_many(0 if waiting else len(order))  # FIFO behind waiters
                    for ext, sid in zip(order, got):
                        sid_of[ext] = sid
                        ext_of[sid] = ext
                        admitted += 1
                    for ext in order[len(got):]:
                        waiting.append(ext)
                        sid_of[ext] = -3  # waiting
                qs = np.arange(i, k)
                live = sid_of[exts] >= 0
                parts.append(qs[live])
                for q in qs[~live].tolist():
                    held[int(streams[q])].append(q)
            i = k
            max_wait = max(max_wait, len(waiting))
            batch = np.concatenate(parts) if parts else np.zeros(0, np.int64)
            if batch.size == 0:
                if i < n and realtime:
                    gap = times[i] - (time.perf_counter() - t0)
                    if gap > 2e-3:
                        time.sleep(gap - 1e-3)
                elif waiting and not ext_of:
                    raise RuntimeError("no stream can be admitted under the memory budget")
                continue
            sids = sid_of[streams[batch]].astype(np.uint32)
            tf = time.perf_counter()
            B.oasm_feed_many(self.ctx, sids, tr.payload, offs[batch], lens[batch].astype(np.uint32))
            ending = sids[last[batch]].astype(np.int64).tolist()
            if ending:
                B.oasm_end_streams(self.ctx, ending)
            ts = time.perf_counter()
            B.oasm_step(self.ctx)
            out = B.oasm_drain(self.ctx)
            te = time.perf_counter()
            phase["schedule"] += tf - t_it
            phase["feed"] += ts - tf
            phase["step_drain"] += te - ts
            step_ms.append((te - ts) * 1e3)
            done_at[batch] = te - t0
            steps += 1
            kept += int(out.size)
            fed_bytes += int(lens[batch].sum())
            if collect and out.size:
                for s in np.unique(out["stream_id"]):
                    hits[ext_of[int(s)]].append(out[out["stream_id"] == s])
            if ending:  # their last decisions are drained: free the slots
                B.oasm_close_streams(self.ctx, ending)
                for s in ending:
                    sid_of[ext_of.pop(s)] = -2
            phase["close"] += time.perf_counter() - te
        wall = time.perf_counter() - t0
        lat = (done_at - times) * 1e3
        ok = ~np.isnan(lat)
        res = {
            "packets": int(n), "bytes": int(lens.sum()), "fed_bytes": fed_bytes,
            "offered_gbps": float(tr.meta.get("gbps", 0.0)),
            "achieved_gbps": lens.sum() * 8 / wall / 1e9,
            "wall_s": wall, "steps": steps, "kept": kept,
            "p50_ms": float(np.percentile(lat[ok], 50)) if ok.any() else None,
            "p99_ms": float(np.percentile(lat[ok], 99)) if ok.any() else None,
            "max_ms": float(lat[ok].max()) if ok.any() else None,
            "step_ms_p50": float(np.percentile(step_ms, 50)) if step_ms else None,
            "step_ms_p99": float(np.percentile(step_ms, 99)) if step_ms else None,
            "step_ms_max": float(max(step_ms)) if step_ms else None,
            "mean_batch_bytes": fed_bytes / max(1, steps),
            "phase_ms_per_step": {k: v * 1e3 / max(1, steps) for k, v in phase.items()},
            "streams_admitted": admitted, "max_waiting_streams": max_wait,
        }
        if collect:
            res["hits"] = {e: np.concatenate(v) for e, v in hits.items()}
        return res

    def _replay_native(self, tr, realtime: bool, collect: bool) -> dict:
        times = np.asarray(tr.times, dtype=np.float64)
        lens = np.asarray(tr.lens, dtype=np.int64)
        done, hits, st = self.B.oasm_replay(self.ctx, times, tr.streams, tr.offs, tr.lens,
                                            tr.last, tr.payload, tr.n_streams,
                                            realtime=realtime,
                                            max_batch_bytes=self.max_batch_bytes,
                                            collect=collect)
        lat = (done - times) * 1e3
        ok = ~np.isnan(lat)
        steps = int(st["steps"])
        res = {
            "packets": int(times.size), "bytes": int(lens.sum()), "fed_bytes": int(st["bytes"]),
            "offered_gbps": float(tr.meta.get("gbps", 0.0)),
            "achieved_gbps": lens.sum() * 8 / max(st["wall_s"], 1e-12) / 1e9,
            "wall_s": float(st["wall_s"]), "steps": steps, "kept": int(st["kept"]),
            "p50_ms": float(np.percentile(lat[ok], 50)) if ok.any() else None,
            "p99_ms": float(np.percentile(lat[ok], 99)) if ok.any() else None,
            "max_ms": float(lat[ok].max()) if ok.any() else None,
            "step_ms_mean": st["step_s_sum"] * 1e3 / max(1, steps),
            "step_ms_max": st["step_s_max"] * 1e3,
            "mean_batch_bytes": st["bytes"] / max(1, steps),
            "streams_admitted": int(st["streams_admitted"]),
            "max_waiting_streams": int(st["max_waiting_streams"]),
            "engine": "native",
            # what the library did during the replay, and during its slowest step
            "reruns": int(st["reruns"]), "graph_builds": int(st["graph_builds"]),
            "buffer_grows": int(st["buffer_grows"]),
            "slowest_step": {"index": int(st["slowest_step"]), "ms": st["step_s_max"] * 1e3,
                             "bytes": int(st["slowest_bytes"]),
                             "reruns": int(st["slowest_reruns"]),
                             "graph_builds": int(st["slowest_graph_builds"]),
                             "buffer_grows": int(st["slowest_buffer_grows"])},
        }
        if collect:
            out = {}
            if hits is not None and hits.size:
                order = np.argsort(hits["stream_id"], kind="stable")
                h = hits[order]
                ids, starts = np.unique(h["stream_id"], return_index=True)
                bounds = list(starts[1:]) + [h.size]
                for e, a, b in zip(ids.tolist(), starts.tolist(), bounds):
                    out[int(e)] = h[a:b]
            res["hits"] = out
        return res

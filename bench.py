#!/usr/bin/env python
"""Benchmark of the OASM device path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload bytes_zipf|dictionary_dna|dictionary_dna_64m|plain_dna|
                     plain_dna_1g|bytes_zipf_256m|many_texts|many_texts_256m|served|
                     dictionary_dna_weighted] [--costs SUB,INS,DEL] [--no-extras]

One step = one pass of the whole path over the workload: open a stream, feed
the text, end it and flush (stage, bit-parallel scan, anchored verification,
ordering, filter, emit), all through the C ABI.  The default workload is the
largest single-GPU configuration, the batched dictionary of uneven byte
patterns: 4,096 patterns (m log-uniform in [16, 128], K uniform in
[1, min(8, m/4)]) over a 1 GiB Zipf(1.1) byte text with 500 planted copies
per pattern.

Printed: one JSON line with the metric (GCUPS: sum over patterns of m times
text symbols, per second), device-resident throughput (`value`), end-to-end
throughput through host buffers (`e2e`), the scan kernel's roofline against
the integer issue peak, the CPU oracle on a bounded sample, and the SM
clocks seen during the timed region.  The default run adds, as extra keys,
the same measurements (fewer steps) for the DNA dictionary (1,024 patterns,
256 MiB), the plain one-pattern kernel (m = 8, K = 2 over 1 GiB of DNA) and a
compact served block (the native serving loop at three offered loads, p50 and
p99 latency).  With integer edit costs (--costs, or the
dictionary_dna_weighted workload: the DNA dictionary with substitution 1,
insertion 2, deletion 2) the path is the weighted one: the wave-front dynamic
program replaces the bit-parallel scan.  Under torchrun every rank runs its own
replica (a different seed) on its own GPU (weak scaling); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OPS_PER_WORD_STEP = 16  # integer ops of one 32-bit column step of the scan
# integer ops of one cell of the weighted dynamic program: two cells (one per
# 16-bit half) share 5 operations -- the symbol test, its 0/1 by a 16x2
# minimum, the substitution cost by a multiply-add, two 16x2 add-minimums
OPS_PER_DP_CELL = 2.5
WEIGHTED_DEFAULT_COSTS = (1, 2, 2)
# DRAM bytes per scan launch and text byte, from an ncu capture of the current
# scan kernels (traffic scales with the text: each launch reads it once); a
# workload without a capture of the current kernels reports traffic null
SCAN_DRAM_BYTES_PER_TEXT_BYTE = {
    # the Zipf byte dictionary's six scan launches on a 256 MiB text: 292.8 MB
    # per launch (mean of the 12 launches of two steps)
    "bytes_zipf": 292.84e6 / (256 << 20),
    "bytes_zipf_256m": 292.84e6 / (256 << 20)}
# integer lanes per SM that can issue one integer instruction per clock (four
# sub-partitions of 32 lanes): the derived peak is SMs x 128 x SM clock
INT_LANES_PER_SM = 128
DEFAULT_WORKLOAD = "bytes_zipf"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-alt", action="store_true",
                    help="skip the extra measurement with the automatic piece filter")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra workloads of the default run (DNA dictionary, plain "
                         "one-pattern kernel, served block)")
    ap.add_argument("--served-packets", type=int, default=200000)
    ap.add_argument("--served-engine", default="native", choices=["native", "python"],
                    help="serving loop: inside the library (oasm_replay) or in Python")
    ap.add_argument("--served-zero-copy", action="store_true",
                    help="register each trace's payload for zero-copy feeds instead of "
                         "copying packets through pinned staging")
    ap.add_argument("--served-batch-mb", type=float, default=32.0,
                    help="byte budget of one serving step (MiB)")
    ap.add_argument("--prefilter", type=int, default=None,
                    help="cfg.prefilter_piece: patterns whose K+1 pieces are at least this "
                         "long use the exact piece filter instead of the scan (0 = off, "
                         "1 = automatic per pattern; default 1 for the served signatures, "
                         "0 elsewhere)")
    ap.add_argument("--output", default="filtered", choices=["filtered", "ends", "all_hits"],
                    help="rules.output: the filtered occurrence set (OASM, default), every "
                         "Less Naive end, or every hit of Eq. 2 unfiltered (the raw counts of "
                         "the paper's Table 1 comparison)")
    ap.add_argument("--record-order", type=int, default=0, choices=[0, 1, 2],
                    help="cfg.record_order (filtered output): 0 automatic, 1 records written "
                         "in canonical order by the filter, 2 appended then sorted")
    ap.add_argument("--tuning-cache", default=None,
                    help="JSON file of autotuned launch settings keyed by GPU and pattern "
                         "set: reused when the key is there, written after tuning otherwise")
    ap.add_argument("--graphs", type=int, default=1,
                    help="cfg.graphs: launch each step as a captured CUDA graph, updated in "
                         "place while its shape repeats (1, default) or directly (0)")
    ap.add_argument("--text-mib", type=int, default=None,
                    help="text size of the dictionary_dna workloads in MiB (planted copies "
                         "scale with it); for small profiling captures")
    ap.add_argument("--costs", default=None,
                    help="integer edit costs SUB,INS,DEL (each 1..255): the weighted path "
                         "(oasm_create_weighted); default 1,2,2 for dictionary_dna_weighted, "
                         "unit costs (the bit-parallel path) elsewhere")
    a = ap.parse_args()
    if a.prefilter is None:
        a.prefilter = 1 if a.workload == "served" else 0
    if a.costs is not None:
        a.costs = tuple(int(x) for x in a.costs.split(","))
        if len(a.costs) != 3:
            raise SystemExit("--costs takes SUB,INS,DEL")
    elif a.workload.endswith("_weighted"):
        a.costs = WEIGHTED_DEFAULT_COSTS
    if a.costs is not None:
        a.prefilter = 0  # the weighted path has no piece filter
    return a


def make_workload(name: str, seed_offset: int, text_mib: int | None = None):
    from paper_1712_03560_gb300 import workloads as W
    if text_mib is not None and name.startswith("dictionary_dna"):
        n = int(text_mib) << 20
        return W.dictionary_dna(seed=2 + 1000 * seed_offset, n=n, copies=max(1, 1000 * n >> 28)), \
            (f"{name} at {text_mib} MiB: 1024 DNA patterns m~U[8,32] K=floor(m/10), "
             f"{text_mib} MiB iid DNA text, {max(1, 1000 * n >> 28)} planted copies/pattern")
    if name == "dictionary_dna":
        return W.dictionary_dna(seed=2 + 1000 * seed_offset), \
            "dictionary_dna: 1024 DNA patterns m~U[8,32] K=floor(m/10), 256 MiB iid DNA text, 1000 planted copies/pattern"
    if name == "dictionary_dna_weighted":
        return W.dictionary_dna(seed=2 + 1000 * seed_offset), \
            "dictionary_dna_weighted: 1024 DNA patterns m~U[8,32] K=floor(m/10), 256 MiB iid DNA text, 1000 planted copies/pattern, integer edit costs"
    if name == "dictionary_dna_64m":
        return W.dictionary_dna(seed=2 + 1000 * seed_offset, n=64 << 20, copies=250), \
            "dictionary_dna_64m: 1024 DNA patterns m~U[8,32] K=floor(m/10), 64 MiB iid DNA text, 250 planted copies/pattern"
    if name == "bytes_zipf_256m":
        return W.bytes_zipf(seed=3 + 1000 * seed_offset, n=256 << 20, copies=125), \
            "bytes_zipf_256m: 4096 byte patterns m log-uniform [16,128], K~U[1,min(8,m/4)], 256 MiB Zipf(1.1) text, 125 copies/pattern"
    if name == "plain_dna":
        return W.plain_dna(seed=1 + 1000 * seed_offset), \
            "plain_dna: 1 DNA pattern m=8 K=2, 1e6 iid DNA symbols, 200 planted copies"
    if name == "plain_dna_1g":
        return W.plain_dna(seed=1 + 1000 * seed_offset, n=1 << 30, copies=200_000), \
            "plain_dna_1g: 1 DNA pattern m=8 K=2, 1 GiB iid DNA symbols, 200000 planted copies"
    if name == "bytes_zipf":
        return W.bytes_zipf(seed=3 + 1000 * seed_offset), \
            "bytes_zipf: 4096 byte patterns m log-uniform [16,128], K~U[1,min(8,m/4)], 1 GiB Zipf(1.1) text, 500 copies/pattern"
    if name == "many_texts":
        return W.many_texts(seed=4 + 1000 * seed_offset), \
            "many_texts: 10000 DNA texts lognormal(median 1e5) ~4 GB x 512 DNA patterns m~U[12,48] K=3"
    if name == "served":
        tr = W.served(seed=5 + 1000 * seed_offset, n_packets=20000, gbps=1.0)
        texts = [t for t in tr.stream_texts() if t.size]
        return W.Workload("served", tr.patterns, tr.ks, texts, dict(tr.meta)), \
            "served: 2000 signatures m~U[8,64] K=2 over the concatenated streams of a 20,000-packet trace"
    if name == "many_texts_256m":
        return W.many_texts(seed=4 + 1000 * seed_offset, n_texts=640, total=2.56e8, copies=13), \
            "many_texts_256m: 640 DNA texts lognormal(median 1e5) ~256 MB x 512 DNA patterns m~U[12,48] K=3"
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


ORACLE_MODE = {"filtered": "oasm", "ends": "ends", "all_hits": "hits"}


def cpu_baseline(wl, budget_s: float, costs=None, output: str = "filtered"):
    """The oracle as it stands on a bounded sample: whole text, a subset of patterns."""
    import oracle
    cores = os.cpu_count() or 1
    text = wl.texts[0] if len(wl.texts) == 1 else np.concatenate(wl.texts[:50])
    # estimate the per-pattern cost on a prefix, then size the sample
    probe = text[: min(text.size, 1 << 22)]
    t0 = time.perf_counter()
    oracle.oasm(wl.patterns[0], int(wl.ks[0]), probe, costs=costs)
    per_sym = (time.perf_counter() - t0) / max(1, probe.size)
    per_pat = per_sym * text.size
    n_pat = int(max(1, min(len(wl.patterns), cores * max(1, int(budget_s / max(per_pat, 1e-9))))))
    if per_pat > budget_s:  # one pattern over the whole text is already too slow
        n_sym = int(budget_s / per_sym)
        text = text[:max(1024, n_sym)]
        n_pat = min(len(wl.patterns), cores)
    idx = np.linspace(0, len(wl.patterns) - 1, n_pat).astype(int)
    pats = [wl.patterns[i] for i in idx]
    ks = [int(wl.ks[i]) for i in idx]
    t0 = time.perf_counter()
    res = oracle.oasm_dictionary(pats, ks, text, threads=cores, costs=costs,
                                 mode=ORACLE_MODE[output])
    dt = time.perf_counter() - t0
    cells = sum(p.size for p in pats) * text.size
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": min(cores, n_pat), "kind": "oracle",
            "sample": f"{n_pat} of {len(wl.patterns)} patterns x {text.size} text symbols, "
                      f"{dt:.1f} s, {len(res)} occurrences"}, (idx, text, res)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, desc = make_workload(args.workload, 0, args.text_mib)
    import oracle
    cores = os.cpu_count() or 1
    text = wl.texts[0] if len(wl.texts) == 1 else np.concatenate(wl.texts[:50])
    probe = text[: min(text.size, 1 << 21)]
    t0 = time.perf_counter()
    oracle.oasm(wl.patterns[0], int(wl.ks[0]), probe, costs=args.costs)
    per_sym = (time.perf_counter() - t0) / max(1, probe.size)
    # each step: `cores` patterns over a prefix sized for ~6 s of work
    n_sym = int(min(text.size, max(1 << 16, 6.0 / max(per_sym, 1e-12))))
    n_pat = min(len(wl.patterns), cores)
    idx = np.linspace(0, len(wl.patterns) - 1, n_pat).astype(int)
    pats = [wl.patterns[i] for i in idx]
    ks = [int(wl.ks[i]) for i in idx]
    sample = text[:n_sym]
    for _ in range(args.warmup):
        oracle.oasm_dictionary(pats, ks, sample[: min(n_sym, 1 << 16)], threads=cores,
                               costs=args.costs, mode=ORACLE_MODE[args.output])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.oasm_dictionary(pats, ks, sample, threads=cores, costs=args.costs,
                               mode=ORACLE_MODE[args.output])
    dt = time.perf_counter() - t0
    cells = sum(p.size for p in pats) * n_sym * args.steps
    val = cells / dt / 1e9
    line = {"metric": "GCUPS", "value": val, "unit": "GCUPS", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": run_config(args, wl, desc, int(os.environ.get("WORLD_SIZE", "1"))),
            "runs_on": "the oracle on the host cores",
            "cpu_baseline": {"value": val, "unit": "GCUPS", "cores": n_pat, "kind": "oracle",
                             "sample": f"{n_pat} of {len(wl.patterns)} patterns x {n_sym} text symbols per step"},
            "e2e": {"value": val, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVED_LOADS_GBPS = (0.5, 1.0, 2.0, 3.0, 4.0, 6.0, 10.0, 25.0, 100.0, 400.0)


def filter_mask(patterns, ks, piece: int) -> list:
    """Which patterns cfg.prefilter_piece = piece routes to the piece filter
    (asked of the library, which applies the same rule at oasm_create)."""
    from paper_1712_03560_gb300 import binding as B
    return B.oasm_piece_filter_choice(patterns, ks, piece).tolist()


def measured_hbm_gbs():
    """HBM copy bandwidth from MEASURED_PEAKS.json (a copy kernel measured on
    this GPU model), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_served(args):
    """Load sweep of the serving loop: 4,096 byte streams, 2,000 signatures.
    One server on one GPU: under torchrun, rank 0 runs it and the other
    ranks exit without work."""
    import torch
    from paper_1712_03560_gb300 import serve
    from paper_1712_03560_gb300 import workloads as W
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n_pkt = args.served_packets
    base = W.served(seed=5, n_packets=200, gbps=1.0)
    msum = sum(p.size for p in base.patterns)
    desc = ("served: 4096 byte streams, packets U[64,1500] B with Poisson arrivals, 2000 signatures "
            "m~U[8,64] K=2, Zipf(1.1) payload, 1% planted; latency = arrival to end of the step "
            "that matched the packet")
    sweep = []
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    clocks = Clocks(dev)
    with serve.Server(base.patterns, base.ks, max_streams=4096, timing=True, device=dev,
                      prefilter_piece=args.prefilter,
                      max_batch_bytes=int(args.served_batch_mb * (1 << 20))) as srv:
        # warm-up: grow every step buffer to the sweep's sizes, then a paced pass
        for _ in range(max(1, args.warmup)):
            srv.replay(W.served(seed=99, n_packets=20000, gbps=10.0), realtime=False,
                       engine=args.served_engine)
        srv.replay(W.served(seed=98, n_packets=20000, gbps=1.0), realtime=True,
                   engine=args.served_engine)
        clocks.start()
        srv.reset_stats()
        st_best, kept_best = None, 0
        for g in SERVED_LOADS_GBPS:
            # overload points get a longer trace: a saturated replay of 200,000
            # packets lasts only a few steps
            tr = W.served(seed=int(5 + 10 * g), n_packets=n_pkt if g < 50 else 4 * n_pkt, gbps=g)
            st0 = srv.stats()
            r = srv.replay(tr, realtime=True, engine=args.served_engine,
                           zero_copy=args.served_zero_copy)
            st1 = srv.stats()
            r["gcups"] = msum * r["bytes"] / r["wall_s"] / 1e9
            if not sweep or r["achieved_gbps"] > max(x["achieved_gbps"] for x in sweep):
                st_best = {k: st1[k] - st0[k] for k in st1}
                kept_best = r["kept"]
            sweep.append({k: r.get(k) for k in ("offered_gbps", "achieved_gbps", "p50_ms",
                                                 "p99_ms", "max_ms", "steps", "mean_batch_bytes",
                                                 "step_ms_p50", "step_ms_p99", "step_ms_mean",
                                                 "step_ms_max", "gcups", "packets",
                                                 "phase_ms_per_step", "reruns", "graph_builds",
                                                 "buffer_grows", "slowest_step")})
        clk = clocks.stop()
        st_all = srv.stats()
    best = max(sweep, key=lambda x: x["achieved_gbps"])
    # roofline of the scan over the steps of the best load point (library events)
    peaks = int_peaks(dev)
    derived = derived_peak_tops(dev, clk)
    fm = filter_mask(base.patterns, base.ks, args.prefilter)
    words = sum((p.size + 31) // 32 for p, on in zip(base.patterns, fm) if not on) \
        * st_best["text_bytes"]
    scan_ms = st_best["scan_ms"]
    achieved_alg = words * OPS_PER_WORD_STEP / max(scan_ms * 1e-3, 1e-12) / 1e12
    achieved = st_best["word_steps"] * OPS_PER_WORD_STEP / max(scan_ms * 1e-3, 1e-12) / 1e12
    derived_peak = derived["tops"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": derived_peak, "unit": "Tops/s",
                "frac": achieved / derived_peak, "traffic": None,
                "peak_source": (f"derived: {derived['sms']} SMs x {INT_LANES_PER_SM} integer "
                                f"lanes x {derived['sm_mhz']:.0f} MHz"),
                "units": "executed lane word-steps x 16 ops (a packed lane counts once)",
                "achieved_algorithmic": achieved_alg, "frac_algorithmic": achieved_alg / derived_peak,
                "measured_peaks_tops": peaks, "peak_measured_mix": peaks["scan_step"],
                "frac_of_measured_mix": achieved / peaks["scan_step"],
                "kernel": "scan_kernel (all classes of a step)",
                "kernel_ms_per_launch": scan_ms / max(1, st_best["scan_launches"]),
                "ops_per_word_step": OPS_PER_WORD_STEP,
                "scan_share_of_device_step": scan_ms / max(st_best["step_ms"], 1e-12),
                "prefilter_share_of_device_step": st_best["prefilter_ms"] / max(st_best["step_ms"], 1e-12)}
    cpu = None
    if not args.no_cpu:
        wl, _ = make_workload("served", 0)
        cpu, _ = cpu_baseline(wl, args.cpu_seconds)
    knee = max((x for x in sweep if x["achieved_gbps"] >= 0.9 * x["offered_gbps"]),
               key=lambda x: x["offered_gbps"], default=None)
    line = {"metric": "GCUPS", "value": best["gcups"], "unit": "GCUPS", "n_gpus": 1,
            "steps": sum(x["steps"] for x in sweep), "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc, "streams": 4096, "signatures": len(base.patterns),
                       "prefilter_piece": args.prefilter,
                       "step_budget_bytes": int(args.served_batch_mb * (1 << 20)),
                       "engine": args.served_engine,
                       "zero_copy": args.served_zero_copy,
                       "packets_per_load": n_pkt, "packets_per_overload_point": 4 * n_pkt, "l2": "per-step text is small; L2-resident"},
            "served": {"sweep": sweep, "sustained_gbps": best["achieved_gbps"],
                       "knee_offered_gbps": knee["offered_gbps"] if knee else None,
                       "p50_ms_at_knee": knee["p50_ms"] if knee else None,
                       "p99_ms_at_knee": knee["p99_ms"] if knee else None},
            # the served value is already end to end: packets from host memory
            # through oasm_feed_many, results drained to host memory, wall clock
            "e2e": {"value": best["gcups"], "unit": "GCUPS",
                    "h2d_bytes_per_step": int(best["mean_batch_bytes"]),
                    "d2h_bytes_per_step": int(kept_best * 32 / max(1, best["steps"])),
                    "note": "the served value is measured end to end (wall clock, host packets in, "
                            "host hits out)"},
            "gpu_launches": int(st_all["launches"]),
            "library_ms_per_step_at_best": {
                k: st_best[k] / max(1, st_best["steps"])
                for k in ("step_ms", "scan_ms", "prefilter_ms", "host_plan_ms", "host_launch_ms",
                          "host_wait_ms", "host_post_ms")},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk}
    print(json.dumps(line), flush=True)


def sm_count(dev: int) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def sm_max_mhz(dev: int, clk: dict | None = None) -> tuple:
    """The GPU's maximum SM clock: from the samples of the timed region, else
    one nvidia-smi query; (MHz, source)."""
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"]), "nvidia-smi during the timed region"
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits", "-i", str(dev)],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        return float(out.splitlines()[0]), "nvidia-smi"
    except Exception:
        return 2070.0, "the GB300's nominal maximum (no nvidia-smi)"


def derived_peak_tops(dev: int, clk: dict | None = None) -> dict:
    """Integer issue peak from unit counts and the clock: every SM issues one
    32-lane integer instruction per clock in each of its four sub-partitions."""
    sms = sm_count(dev)
    mhz, src = sm_max_mhz(dev, clk)
    return {"tops": sms * INT_LANES_PER_SM * mhz * 1e6 / 1e12, "sms": sms, "sm_mhz": mhz,
            "clock_source": src}


def int_peaks(dev: int) -> dict:
    """Measured integer issue rates (T ops/s) of the three microbenchmark mixes."""
    from paper_1712_03560_gb300 import binding as B
    return {mix: B.oasm_measure_int_peak_mix(dev, mix)[0] / 1e12 for mix in B.INT_MIXES}


def run_config(args, wl, desc, world: int) -> dict:
    """The workload keys of the JSON line (the same for both arms)."""
    return {"workload": desc, "text_bytes": int(wl.text_bytes),
            "patterns": len(wl.patterns), "l2": "inputs larger than L2 (text > 129 MB)"
            if wl.text_bytes > (129 << 20) else "input smaller than L2",
            "parallelism": f"replicas x{world}",
            "prefilter_piece": args.prefilter, "graphs": args.graphs,
            "output": args.output, "record_order": args.record_order,
            "costs": None if args.costs is None else dict(zip(("sub", "ins", "del"), args.costs))}


def measure_workload(args, name, dev, steps, warmup, *, rank=0, world=1, dist=None,
                     with_e2e=True, with_cpu=True, with_alt=True):
    """One workload through the C ABI: `steps` timed steps on device-resident
    input (CUDA events on the library's stream), the scan's roofline, and
    optionally the end-to-end run through host buffers, the oracle on a
    bounded sample with a parity check, and the automatic piece filter."""
    import torch
    from paper_1712_03560_gb300 import binding as B

    wl, desc = make_workload(name, rank, args.text_mib if name == args.workload else None)
    rules = None if args.output == "filtered" else {"output": args.output}
    # two sets of streams are open at once in the pipelined steps below
    ctx = B.oasm_create(wl.patterns, wl.ks, rules,
                        {"device": dev, "timing": 1, "max_streams": max(64, 2 * len(wl.texts)),
                         "prefilter_piece": args.prefilter, "graphs": args.graphs,
                         "record_order": args.record_order},
                        costs=args.costs)
    stream = torch.cuda.ExternalStream(B.oasm_cuda_stream(ctx), device=dev)
    dtexts = [torch.from_numpy(t).to(f"cuda:{dev}") for t in wl.texts]
    torch.cuda.synchronize()
    tuned = None
    if not args.no_autotune:
        # tile shapes for this GPU and pattern set, timed on a slice of the text
        big = max(dtexts, key=lambda t: t.numel())
        sample = big[: min(big.numel(), 32 << 20)]
        if args.tuning_cache:
            from paper_1712_03560_gb300 import tuning as TU
            key = TU.cache_key(torch.cuda.get_device_name(dev), wl.patterns, wl.ks, args.costs,
                               {"prefilter_piece": args.prefilter})
            how = TU.autotune_cached(B, ctx, sample, key, args.tuning_cache)
            tuned = {"buckets": B.oasm_get_tuning(ctx), "source": how}
        else:
            tuned = json.loads(B.oasm_autotune(ctx, sample))
        print(json.dumps({"autotune": name, **tuned}), file=sys.stderr, flush=True)
        for bk in tuned["buckets"]:
            bk.pop("trials", None)

    # host time per phase of a step (submit, device step, drain, close)
    host_ms = {"submit": 0.0, "step": 0.0, "drain": 0.0, "close": 0.0}
    drain_buf = [None]

    def timed(phase, fn, *a):
        t0 = time.perf_counter()
        r = fn(*a)
        host_ms[phase] += (time.perf_counter() - t0) * 1e3
        return r

    def open_feed(c, submit):
        sids = B.oasm_open_streams(c, len(wl.texts))
        submit(c, sids.tolist())
        B.oasm_end_streams(c, sids)
        return sids

    def drain(c):
        out = B.oasm_drain(c, drain_buf[0])
        n = len(out)
        if drain_buf[0] is None or drain_buf[0].size < n:  # reused from the next step on
            drain_buf[0] = np.empty(max(1024, n * 5 // 4), dtype=B.HIT_DTYPE)
        return out

    def pipeline(c, submit, nsteps):
        """nsteps steps, each over the whole workload, software-pipelined through
        the split step (oasm_step_begin / oasm_step_end): while step i runs on
        the device, the host drains and closes step i - 1's streams (their
        records' copy to the host overlaps step i) and opens and feeds step i +
        1's.  Returns the last step's records."""
        cur = timed("submit", open_feed, c, submit)
        prev, out = None, None
        for i in range(nsteps):
            timed("step", B.oasm_step_begin, c)
            if prev is not None:
                out = timed("drain", drain, c)
                timed("close", B.oasm_close_streams, c, prev)
            nxt = timed("submit", open_feed, c, submit) if i + 1 < nsteps else None
            timed("step", B.oasm_step_end, c)
            prev, cur = cur, nxt
        out = timed("drain", drain, c)
        timed("close", B.oasm_close_streams, c, prev)
        return out

    def feed_device(c, sids):
        for sd, t in zip(sids, dtexts):
            B.oasm_feed_device(c, sd, t)

    def steps_device(nsteps):
        return len(pipeline(ctx, feed_device, nsteps))

    def steps_host(host_texts, nsteps):
        def feed_host(c, sids):
            for sd, t in zip(sids, host_texts):
                B.oasm_feed(c, sd, t)
        return len(pipeline(ctx, feed_host, nsteps))

    kept = steps_device(warmup)

    # ---- timed region: device-resident inputs
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    builds_warmup = int(B.oasm_get_stats(ctx)["graph_builds"])
    B.oasm_reset_stats(ctx)
    for k in host_ms:
        host_ms[k] = 0.0
    clocks = Clocks(dev)
    clocks.start()
    time.sleep(0.25)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    kept = steps_device(steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    st = B.oasm_get_stats(ctx)
    host_step_ms = {k: v / steps for k, v in host_ms.items()}
    if dist:
        t = torch.tensor([ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    cells_step = wl.cells
    value = cells_step * steps * world / (ms * 1e-3) / 1e9
    text_gbps = wl.text_bytes * steps * world / (ms * 1e-3) / 1e9

    # ---- roofline of the dominant kernel (the forward scan), measured live
    peaks = int_peaks(dev)
    derived = derived_peak_tops(dev, clk)
    scan_ms_launch = st["scan_ms"] / max(1, st["scan_launches"])
    fm = filter_mask(wl.patterns, wl.ks, args.prefilter)
    launches_step = max(1, st["scan_launches"] // max(1, steps))
    # algorithmic words: what the scan's algorithm must run per text symbol --
    # every word of a one-pass pattern, word 0 of a cut-off class pattern
    # (the words it runs beyond that near matches are in the executed count)
    cut_classes = {b["words"] for b in B.oasm_get_tuning(ctx) if b["algo"] == 9}
    words = sum((1 if (p.size + 31) // 32 in cut_classes else (p.size + 31) // 32)
                for p, on in zip(wl.patterns, fm) if not on) * wl.text_bytes
    alg_ops_launch = words * OPS_PER_WORD_STEP / launches_step
    achieved_alg = alg_ops_launch / (scan_ms_launch * 1e-3) / 1e12
    # executed work: lane word-steps the scan ran (oasm_stats.word_steps)
    exec_ops_launch = st["word_steps"] / max(1, steps) * OPS_PER_WORD_STEP / launches_step
    achieved = exec_ops_launch / (scan_ms_launch * 1e-3) / 1e12
    units = ("executed lane word-steps x 16 ops (a packed lane counts once; a cut-off "
             "class counts word 0 of every step plus the words its full form ran)")
    kname, opu = "scan_kernel (all classes of a step)", OPS_PER_WORD_STEP
    mix = "scan_step"
    if args.costs is not None:
        # weighted path: a unit is one cell of the dynamic program; executed
        # cells count every row of a pattern's 32 W-row column
        cells_alg = sum(p.size for p in wl.patterns) * wl.text_bytes
        achieved_alg = cells_alg * OPS_PER_DP_CELL / launches_step / (scan_ms_launch * 1e-3) / 1e12
        achieved = st["word_steps"] / max(1, steps) * OPS_PER_DP_CELL / launches_step \
            / (scan_ms_launch * 1e-3) / 1e12
        units = ("executed dynamic-program cells (32 W rows per pattern) x 2.5 ops (5 per "
                 "pair of cells in 16-bit halves)")
        kname, opu = "wscan_kernel (weighted wave-front, all classes of a step)", OPS_PER_DP_CELL
        mix = "weighted_step"
    tpb = None if args.costs is not None else SCAN_DRAM_BYTES_PER_TEXT_BYTE.get(name)
    traffic = tpb * wl.text_bytes if tpb else None  # bytes per scan launch
    hbm_peak = measured_hbm_gbs()
    peak = derived["tops"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak,
                "peak_source": (f"derived: {derived['sms']} SMs x {INT_LANES_PER_SM} integer "
                                f"lanes x {derived['sm_mhz']:.0f} MHz ({derived['clock_source']})"),
                "units": units,
                "achieved_algorithmic": achieved_alg, "frac_algorithmic": achieved_alg / peak,
                "traffic": traffic,
                "hbm": None if traffic is None else {
                    "achieved_gbs": traffic / (scan_ms_launch * 1e-3) / 1e9, "peak_gbs": hbm_peak[0],
                    "frac": traffic / (scan_ms_launch * 1e-3) / 1e9 / hbm_peak[0],
                    "peak_source": hbm_peak[1]},
                "measured_peaks_tops": peaks,
                "peak_measured_mix": peaks[mix], "measured_mix": mix,
                "frac_of_measured_mix": achieved / peaks[mix],
                "kernel": kname, "kernel_ms_per_launch": scan_ms_launch,
                "launches_per_step": launches_step,
                "ops_per_word_step": opu}

    # ---- end to end through host buffers (pinned-free: oasm_feed copies the
    # caller's pageable bytes into the library's pinned staging)
    e2e = None
    if with_e2e and not args.no_e2e:
        # the texts in one pinned host buffer, registered once (as a caller
        # that keeps its input in pinned memory would): each step's gather
        # reads them over the CPU-GPU link, with no staging copy
        host_all = np.ascontiguousarray(np.concatenate(wl.texts) if len(wl.texts) > 1
                                        else wl.texts[0])
        offs = np.concatenate([[0], np.cumsum([t.size for t in wl.texts])])
        host = [host_all[offs[i]:offs[i + 1]] for i in range(len(wl.texts))]
        B.oasm_register_host(ctx, host_all)
        steps_host(host, 1)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        kept_h = steps_host(host, steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], device=f"cuda:{dev}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        B.oasm_unregister_host(ctx, host_all)
        e2e = {"value": cells_step * steps * world / dt / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": int(wl.text_bytes), "d2h_bytes_per_step": int(kept_h * 32 + 48),
               "ms_per_step": dt / steps * 1e3, "steps": steps,
               "input": "host texts in pinned memory (oasm_register_host), read by each step"}

    res = {"wl": wl, "desc": desc, "value": value, "ms_per_step": ms / steps,
           "text_gbps": text_gbps, "occurrences_per_step": int(kept), "clocks": clk,
           "kernel_ms": {k: st[k] / steps for k in ("copy_ms", "scan_ms", "prefilter_ms",
                                                     "verify_ms", "order_ms", "filter_ms",
                                                     "step_ms")},
           "prefilter": None if not args.prefilter else {
               "piece": args.prefilter if args.prefilter >= 4 else "auto",
               "patterns": int(sum(fm)),
               "candidates_per_step": st["prefilter_candidates"] / steps,
               "text_gbs": None if st["prefilter_ms"] <= 0 else
               wl.text_bytes * steps / (st["prefilter_ms"] * 1e-3) / 1e9},
           "host_ms_per_step": host_step_ms,
           "library_host_ms_per_step": {k: st[k] / steps for k in
                                        ("host_plan_ms", "host_launch_ms", "host_wait_ms",
                                         "host_post_ms", "host_copy_ms")},
           "record_bytes_per_step": st["record_bytes"] / steps,
           "candidates_per_step": st["candidates"] / steps,
           "hits_per_step": st["hits"] / steps,
           "gpu_launches": int(st["launches"]),
           "graph_builds": {"warmup": builds_warmup, "timed": int(st["graph_builds"])},
           "reruns": int(st["reruns"]), "buffer_grows_timed": int(st["buffer_grows"]),
           "roofline": roofline, "e2e": e2e, "autotune": tuned,
           "cpu_baseline": None, "parity_sample": None, "with_piece_filter": None}
    if rank != 0:
        B.oasm_destroy(ctx)
        return res

    want = idx = text = None
    if with_cpu and not args.no_cpu and world == 1:
        cpu, (idx, text, ores) = cpu_baseline(wl, args.cpu_seconds, args.costs, args.output)
        res["cpu_baseline"] = cpu
        # the sampled patterns' GPU output must equal the oracle's on that sample
        sub_pats = [wl.patterns[i] for i in idx]
        sub_ks = [int(wl.ks[i]) for i in idx]
        with B.Matcher(sub_pats, sub_ks, rules=rules, costs=args.costs,
                       prefilter_piece=args.prefilter) as mt:
            g = mt.search(torch.from_numpy(np.ascontiguousarray(text)).to(f"cuda:{dev}"),
                          device=True)
        got = sorted((int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]),
                      int(r["start"]), int(r["len"])) for r in g)
        want = sorted((int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]),
                       int(r["start"]), int(r["len"])) for r in ores)
        res["parity_sample"] = {"patterns": len(idx), "text_symbols": int(text.size),
                                "occurrences": len(want), "equal": got == want}
    B.oasm_destroy(ctx)

    # ---- the same workload with the automatic piece filter (prefilter_piece = 1):
    # patterns whose pieces rarely match go to the exact filter, the rest stay
    # on the scan; device-resident inputs, timed like the main value
    if with_alt and args.prefilter == 0 and not args.no_alt and world == 1 and \
            args.costs is None and args.output == "filtered":
        ctx2 = B.oasm_create(wl.patterns, wl.ks, None,
                             {"device": dev, "timing": 1,
                              "max_streams": max(64, 2 * len(wl.texts)),
                              "prefilter_piece": 1, "graphs": args.graphs,
                              "record_order": args.record_order})
        try:
            stream2 = torch.cuda.ExternalStream(B.oasm_cuda_stream(ctx2), device=dev)
            if not args.no_autotune:
                big = max(dtexts, key=lambda t: t.numel())
                B.oasm_autotune(ctx2, big[: min(big.numel(), 32 << 20)])
            last = [None]

            pipeline(ctx2, feed_device, warmup)
            torch.cuda.synchronize()
            B.oasm_reset_stats(ctx2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream2)
            last[0] = pipeline(ctx2, feed_device, steps).copy()
            e1.record(stream2)
            e1.synchronize()
            ms2 = e0.elapsed_time(e1)
            st2 = B.oasm_get_stats(ctx2)
            fm2 = filter_mask(wl.patterns, wl.ks, 1)
            par2 = None
            if want is not None and len(wl.texts) == 1:
                # the sampled patterns' rows of the full output against the oracle
                sel = set(int(i) for i in idx)
                full = text.size == wl.texts[0].size
                lim = {i: text.size - wl.patterns[i].size - int(wl.ks[i]) for i in sel}
                pos = {int(i): j for j, i in enumerate(idx)}
                got2 = sorted((pos[int(r["pattern_id"])], int(r["decided_at"]), int(r["k"]),
                               int(r["start"]), int(r["len"])) for r in last[0]
                              if int(r["pattern_id"]) in sel and
                              (full or int(r["decided_at"]) <= lim[int(r["pattern_id"])]))
                want2 = sorted(w for w in want if full or w[1] <= lim[int(idx[w[0]])])
                par2 = {"patterns": len(idx), "occurrences": len(want2), "equal": got2 == want2}
            res["with_piece_filter"] = {
                "path": "automatic piece filter + scan (prefilter_piece = 1)",
                "value": cells_step * steps / (ms2 * 1e-3) / 1e9, "unit": "GCUPS",
                "ms_per_step": ms2 / steps,
                "patterns_on_filter": int(sum(fm2)),
                "kernel_ms": {k: st2[k] / steps for k in ("scan_ms", "prefilter_ms", "verify_ms",
                                                         "order_ms", "filter_ms", "step_ms")},
                "parity_sample": par2}
        finally:
            B.oasm_destroy(ctx2)
    del dtexts
    torch.cuda.empty_cache()
    return res


def served_block(args, dev: int) -> dict:
    """Compact served measurement: the native serving loop (continuous
    batching, split steps, automatic piece filter, steps of at most 32 MiB)
    over 4,096 byte streams and 2,000 signatures, at an offered load below the
    knee, near it and beyond saturation; latency = packet arrival to the end
    of the step that matched it."""
    from paper_1712_03560_gb300 import serve
    from paper_1712_03560_gb300 import workloads as W
    base = W.served(seed=5, n_packets=200, gbps=1.0)
    loads = ((1.0, 50_000), (25.0, 100_000), (400.0, 400_000))
    out = []
    with serve.Server(base.patterns, base.ks, max_streams=4096, timing=True, device=dev,
                      prefilter_piece=1, max_batch_bytes=32 << 20) as srv:
        # warm-up: full 32 MiB steps grow every step buffer to its final size,
        # then a paced pass at a low load
        srv.replay(W.served(seed=99, n_packets=100_000, gbps=10.0), realtime=False,
                   engine="native")
        srv.replay(W.served(seed=98, n_packets=20000, gbps=1.0), realtime=True, engine="native")
        for g, n_pkt in loads:
            tr = W.served(seed=int(5 + 10 * g), n_packets=n_pkt, gbps=g)
            r = srv.replay(tr, realtime=True, engine="native")
            out.append({k: r.get(k) for k in ("offered_gbps", "achieved_gbps", "p50_ms", "p99_ms",
                                               "max_ms", "steps", "packets", "step_ms_mean",
                                               "reruns", "graph_builds", "buffer_grows",
                                               "slowest_step")})
    return {"workload": "4096 byte streams, packets U[64,1500] B, Poisson arrivals, 2000 "
                        "signatures m~U[8,64] K=2; native loop, split steps, automatic piece "
                        "filter, steps <= 32 MiB",
            "loads": out, "sustained_gbps": max(x["achieved_gbps"] for x in out)}


def extra_entry(m: dict) -> dict:
    """The short form of a measurement for an extra key of the line."""
    rf = m["roofline"]
    return {"workload": m["desc"], "value": m["value"], "unit": "GCUPS",
            "ms_per_step": m["ms_per_step"], "text_gbps": m["text_gbps"],
            "e2e": None if m["e2e"] is None else {k: m["e2e"][k] for k in ("value", "ms_per_step",
                                                                         "steps")},
            "frac": rf["frac"], "frac_of_measured_mix": rf["frac_of_measured_mix"],
            "occurrences_per_step": m["occurrences_per_step"],
            "kernel_ms": m["kernel_ms"],
            "scan_share_of_step": m["kernel_ms"]["scan_ms"] / max(m["ms_per_step"], 1e-9),
            "host_ms_per_step": m["host_ms_per_step"],
            "library_host_ms_per_step": m["library_host_ms_per_step"],
            "record_bytes_per_step": m["record_bytes_per_step"]}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "served":
        return run_served(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    m = measure_workload(args, args.workload, dev, args.steps, args.warmup, rank=rank,
                         world=world, dist=dist)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "GCUPS", "value": m["value"], "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": run_config(args, m["wl"], m["desc"], world),
        "text_gbps": m["text_gbps"],
        "occurrences_per_step": m["occurrences_per_step"],
        "kernel_ms": m["kernel_ms"],
        "prefilter": m["prefilter"],
        "host_ms_per_step": m["host_ms_per_step"],
        "library_host_ms_per_step": m["library_host_ms_per_step"],
        "record_bytes_per_step": m["record_bytes_per_step"],
        "candidates_per_step": m["candidates_per_step"],
        "hits_per_step": m["hits_per_step"],
        "gpu_launches": m["gpu_launches"],
        # executable graphs instantiated: during warm-up, and during the timed
        # steps (0 there: each timed step updated the cached graph in place)
        "graph_builds": m["graph_builds"],
        "reruns": m["reruns"],
        "roofline": m["roofline"],
        "e2e": m["e2e"],
        "cpu_baseline": m["cpu_baseline"],
        "parity_sample": m["parity_sample"],
        "with_piece_filter": m["with_piece_filter"],
        "autotune": m["autotune"],
        "clocks": m["clocks"],
    }
    del m
    if world == 1 and not args.no_extras and args.workload == DEFAULT_WORKLOAD and \
            args.costs is None and args.output == "filtered" and args.prefilter == 0:
        # the other dictionary and the plain one-pattern kernel, fewer steps;
        # the served loop at three loads
        ks = min(args.steps, 10)
        for key, name in (("dictionary_dna", "dictionary_dna"), ("plain_kernel", "plain_dna_1g")):
            x = measure_workload(args, name, dev, ks, 3, with_cpu=False, with_alt=False)
            line[key] = extra_entry(x)
            line[key]["steps"], line[key]["warmup"] = ks, 3
            del x
        line["served"] = served_block(args, dev)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

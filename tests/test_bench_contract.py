"""The benchmark's reference arm runs on the host cores (the CPU oracle), so
its JSON line can be checked without a GPU: one line, the contract's keys,
a positive throughput."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("extra", [[], ["--costs", "1,2,2"], ["--output", "ends"]])
def test_reference_arm_prints_one_contract_line(extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "plain_dna", "--steps", "1", "--warmup", "0"] + extra
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "GCUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["costs"] == ({"sub": 1, "ins": 2, "del": 2} if "--costs" in extra
                                    else None)
    # the workload keys are the ones the GPU arm prints for the same arguments
    for k in ("workload", "text_bytes", "patterns", "l2", "parallelism", "prefilter_piece",
              "graphs", "output", "record_order", "costs"):
        assert k in d["config"], k
    assert d["config"]["output"] == (extra[1] if "--output" in extra else "filtered")


def test_bench_help_lists_the_options():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0
    for opt in ("--gpus", "--steps", "--warmup", "--impl", "--workload", "--costs",
                "--graphs", "--tuning-cache", "--record-order"):
        assert opt in r.stdout

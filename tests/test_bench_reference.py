"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the contract's keys, on a workload whose oracle steps take
milliseconds: untimed warm-up steps first, then the timed ones."""
import argparse
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                          "--warmup", "3", "--workload", "ensemble48"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "run-steps/s" and d["n_gpus"] == 1
    assert d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 / d["value"]) < 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"] == "ensemble48" and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "after 3 untimed" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the same config block as the GPU arm prints for the same command
    sys.path.insert(0, ROOT)
    import bench
    w = dict(bench.WORKLOADS["ensemble48"])
    assert d["config"] == bench.config_of(argparse.Namespace(workload="ensemble48"), w, 1)


def test_default_workload_is_the_precision_form_at_512():
    sys.path.insert(0, ROOT)
    import bench
    w = bench.WORKLOADS["forced512"]
    assert w["n"] == 512 and w["prec"] == "fp64" and w["companion"] == "fp32"
    assert w["nu"] == 2e-3 and w["dt"] == 1e-3 and w["force_k"] == 3 and w["force_amp"] == 0.5
    assert w["large"] == ("forced1024", "plain768")

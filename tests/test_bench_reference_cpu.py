"""The benchmark's reference arm (the CPU oracle timed on the host's cores) on a
tiny sample: it runs without a GPU and prints one JSON line with the contract's
keys -- impl, the headline metric and unit, the step count, a cpu_baseline that
says what was timed, and an e2e object with no host/device copies.  Its config
is the GPU arm's (same keys and values), and ms_per_step is the time a step
actually took (the extrapolation to the full workload has its own key)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(300)
def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--ref-rings", "2", "--cpu-samples", "100000"], cwd=ROOT, capture_output=True, text=True,
                       timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("TOD samples/s") and d["unit"] == "samples/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "rings" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert abs(d["ms_per_step"] * d["steps"] / 1e3 - d["measured_seconds"]) < 1e-6 * max(1.0, d["measured_seconds"])
    assert d["extrapolated_ms_per_full_step"] >= d["ms_per_step"]
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    assert d["config"] == bench.workload_config(W.config_lfi(with_pointings=False), int(1e8), "fp64", False)

"""bench.py's output line on a small case: one JSON line with the keys and value types the measurement
contract needs (metric, value, unit, timing, roofline with its peak and fraction, the CPU oracle baseline,
the end-to-end number through the C ABI with its copied bytes, the launch count and the sampled clocks),
and the reference arm's line.  Small sizes keep it to seconds; the numbers themselves are not checked."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_bench_line_has_the_contract_keys():
    d = run_bench("--n", "16", "--depth", "3", "--steps", "2", "--warmup", "3", "--no-f64", "--no-autotune",
                  "--cpu-seconds", "0.5")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert "workload" in d["config"]
    r = d["roofline"]
    assert r["bound"] in ("alu", "hbm", "tensor") and r["peak"] > 0 and 0 < r["frac"] < 2
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1 and c["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"] and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    acc = d["accuracy"]
    assert acc["n"] == 16 and acc["c128_df32"]["max_abs_err"] < 1e-12 and acc["c128_f64"]["max_abs_err"] < 1e-12
    assert acc["c64"]["one_minus_fidelity"] < 1e-8
    q = d["qft"]["qft20"]
    assert q["n"] == 20 and q["value"] > 0 and q["steps"] == 5 and q["warmup"] == 3


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--n", "14", "--depth", "2", "--steps", "1", "--warmup", "1")
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

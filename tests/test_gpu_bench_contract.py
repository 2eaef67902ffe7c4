"""bench.py's JSON line on a GPU: a small run of the batched workload and of
the 3-D workload print one line each with the fields the benchmark contract
asks for (throughput, roofline of the dominant kernel, end-to-end rate with
its copied bytes, clocks during the timed region, kernel launches)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _check_common(d, steps, warmup):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == warmup
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert "workload" in d["config"]
    rf = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert 0 < rf["frac"] < 1.5 and rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["traffic"] is None or rf["traffic"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["gpu_launches"] > 0


def test_batched_line():
    d = _run(["--instances", "8", "--steps", "3", "--warmup", "3", "--no-cpu-baseline", "--no-tune",
              "--no-big"])
    _check_common(d, 3, 3)
    assert d["dtype"] == "f32"
    acc = d["accuracy"]
    assert acc["instances"] == 8 and acc["oracle_sample"]["instances"] == 8
    # FP64 on the GPU after 200 steps: rounding-order differences from the
    # oracle grow with the scheme's own sensitivity, so only a loose bound
    assert acc["oracle_sample"]["fp64_gpu_max_rel_linf"] < 1e-2
    assert acc["rel_linf_vs_fp64"]["max"] >= acc["rel_linf_vs_fp64"]["median"] > 0
    assert acc["rel_linf_vs_fp64_oracle"] < 1e-2
    assert d["fp64_batch"]["value"] > 0 and d["fp64_batch"]["fp32_speedup"] > 1
    assert d["fp64_single"]["rel_linf_vs_fp64_oracle"] < 100 * 1e-12
    # 2 sweeps per step, every sweep at least one launch
    assert d["gpu_launches"] >= 3 * 200 * 2
    assert d["fp64_plain"]["rel_linf_vs_oracle"] < 250 * 1e-12
    assert d["fp32_single"]["rel_linf_vs_fp64_oracle"] < 1e-4
    assert d["nonlinear_chi"]["rel_linf_vs_fp64_oracle"] < 1e-4
    assert d["speedup_vs_explicit"]["speedup"] > 100
    assert d["three_d"]["value"] > 0


def test_three_d_line():
    d = _run(["--workload", "random3d", "--steps", "3", "--warmup", "3", "--no-cpu-baseline"])
    _check_common(d, 3, 3)
    assert d["gpu_launches"] == 3 * 3 * 200
    assert d["accuracy"]["rel_linf_vs_fp64_oracle"] < 1e-4

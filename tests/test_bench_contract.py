"""CPU checks of bench.py's output contract: the reference arm (the FP64
oracle on a small sample of the workload) prints one JSON line with the
required keys, and the roofline block is the dominant leaf region's
algorithmic bytes per launch over its event time against the peak."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-sample-side", "12"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_roofline_of_the_dominant_leaf_region():
    sys.path.insert(0, ROOT)
    import bench
    kernels = {
        "broad_phase": {"launches": 2, "total_ms": 9.0, "algo_bytes": 0.0},     # a parent region: skipped
        "cheb_sweep": {"launches": 100, "total_ms": 0.8, "algo_bytes": 100 * 30e6},
        "local_residual": {"launches": 10, "total_ms": 0.6, "algo_bytes": 10 * 80e6},
    }
    # without an L2 measurement: against the HBM copy peak
    rl = bench.roofline(kernels, {"hbm_gbs": 6000.0}, 15.0)
    assert rl["kernel"] == "cheb_sweep" and rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert rl["ms_per_launch"] == pytest.approx(0.008)
    assert rl["achieved"] == pytest.approx(30e6 / 8e-6 / 1e9, rel=1e-3)
    assert rl["frac"] == pytest.approx(rl["achieved"] / 6000.0, rel=1e-3)
    assert rl["traffic"] == bench.TRAFFIC["cheb_sweep"] and rl["peak_source"].startswith("HBM")
    assert bench.roofline(kernels, {"hbm_gbs": 6800.0, "_fallback": True}, 15.0)["peak_source"] == "fallback"
    # the Chebyshev step's working set fits in L2: against the L2 copy peak
    rl = bench.roofline(kernels, {"hbm_gbs": 6000.0}, 15.0, l2_gbs=12000.0)
    assert rl["bound"] == "l2" and rl["peak"] == 12000.0
    assert rl["frac"] == pytest.approx(rl["achieved"] / 12000.0, rel=1e-3)
    assert rl["hbm_frac"] == pytest.approx(rl["achieved"] / 6000.0, rel=1e-3)
    # a kernel with no working-set model stays on the HBM roof
    k2 = dict(kernels, local_residual={"launches": 10, "total_ms": 9.6, "algo_bytes": 10 * 80e6})
    rl = bench.roofline(k2, {"hbm_gbs": 6000.0}, 15.0, l2_gbs=12000.0)
    assert rl["kernel"] == "local_residual" and rl["bound"] == "hbm" and rl["peak"] == 6000.0

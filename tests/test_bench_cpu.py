"""Host-side parts of bench.py, without a GPU: the reference arm's JSON line,
the roofline arithmetic and the clock-sample filtering."""
import argparse
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    """`--impl reference` times the oracle on a bounded sample and prints the
    contract's line, with the GPU arm's config for the same workload."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--gaussians", "3000", "--views", "4", "--cpu-sample-views", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    w = bench._workload(argparse.Namespace(gaussians=3000, views=4), 0)
    assert d["config"] == bench._config(w, 1)


ALU = {"sm_count": 152, "probe_sm_mhz": 1900.0, "fp32_fma_per_sm_clk": 120.0, "fp32x2_fma_per_sm_clk": 121.0,
       "ex2_per_sm_clk": 30.0, "fp32_fma_per_s": 0.0, "fp32x2_fma_per_s": 0.0, "ex2_per_s": 0.0,
       "fp64_fma_per_sm_clk": 2.0, "fp64_fma_per_s": 0.0, "red_f32_per_s": 4e10, "red_f32x4_per_s": 2e10}


def test_roofline_arithmetic():
    # blend_bwd: (16 eval + 33 contributing) lane-ops per pair over the launch
    # time, against the measured FFMA rate x SM count x the run's SM clock
    c = [0, 0, 1_000_000, 500_000, 0, 2_000, 0, 0, 0, 40_000, 0]
    r = bench.roofline_for("blend_bwd", 1.0, 1, c, 10, 2, 100, 3, {"hbm_gbs": 5000.0}, ALU, 2000.0)
    ops = 16 * 1_000_000 + 33 * 500_000
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(ops / 1e-3 / 1e12)
    assert r["peak"] == pytest.approx(120.0 * 152 * 2000e6 / 1e12)
    assert r["mufu_frac"] == pytest.approx((1_000_000 + 500_000) / 1e-3 / (30.0 * 152 * 2000e6))
    tr = bench.TRAFFIC_PER_UNIT.get("blend_bwd")
    # traffic: DRAM bytes per unit from a capture of the kernel as it stands, else null
    assert r["traffic"] == (pytest.approx(tr[0] * c[tr[1]]) if tr else None)
    assert "2000 MHz" in r["peak_source"] and "of measured" in r["peak_source"]
    # gradient atomics: two float4 adds and one float add per used warp entry
    assert r["atomics_per_s"] == pytest.approx(3 * 40_000 / 1e-3)
    assert r["atomic_frac"] == pytest.approx(2 * 40_000 / 1e-3 / 2e10 + 40_000 / 1e-3 / 4e10)
    # HBM kernels: algorithmic bytes (visible pairs counted apart) over time
    n, V, n_vis = 1000, 4, 1500
    c[10] = n_vis
    r = bench.roofline_for("scatter_keys", 2.0, 2, c, n, V, 5000, 3, {"hbm_gbs": 5000.0}, ALU, 2000.0)
    by = (n * V * 8 + n_vis * 4 + 5000 * 8) / 2
    assert r["achieved"] == pytest.approx(by / 2e-3 / 1e9) and r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert "of measured" in r["peak_source"]
    r = bench.roofline_for("preprocess_fwd", 1.0, 1, c, n, V, 0, 3, {"hbm_gbs": 6800.0, "_fallback": True}, ALU,
                           2070.0)
    by = n * 236 + n_vis * 60 + (n * V - n_vis) * 16
    assert r["achieved"] == pytest.approx(by / 1e-3 / 1e9)
    assert "of fallback" in r["peak_source"]


def test_clock_rows_before_the_timed_region_are_dropped(tmp_path):
    """stop() keeps the rows written after start() returned; throttle reasons
    are collected from those rows only."""
    path = tmp_path / "clk.csv"
    pre = "0, 1000, 2070, 300.0, 0x4, Active, Not Active, Not Active, Not Active\n"   # hw_slowdown, before
    row = "0, 2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
    path.write_text(pre + row + row)

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc, cs.path, cs.skip = _Proc(), str(path), 1
    cs.fh = open(os.devnull, "w")
    out = cs.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    assert not path.exists()


def test_tuning_cache_key_classes():
    """The autotuner caches per GPU, view-count/resolution class and
    Gaussian-count class (powers of two), under a version prefix."""
    from paper_2410_08743_gb300 import tune
    v = [dict(width=1008, height=756), dict(width=256, height=192)]
    k = tune.workload_key("GPU X", v, 1_000_000)
    assert k.startswith("t4|GPU X|views2-px2^20|") and k.endswith("|n2^20")
    assert tune.workload_key("GPU X", v, 1_100_000) == k            # same class
    assert tune.workload_key("GPU X", v, 3_000_000) != k            # another Gaussian-count class
    assert tune.workload_key("GPU X", v[:1], 1_000_000) != k        # another view count

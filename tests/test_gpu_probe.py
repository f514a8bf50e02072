"""The measured arithmetic peaks (the "alu" roofline's denominators): the
probe runs on the device and returns rates within the hardware's plausible
range, consistent between its per-cycle and per-second forms."""
import pytest
import torch

from paper_2410_08743_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def test_alu_peak_probe():
    from paper_2410_08743_gb300 import build
    build.build()
    a = L.gs_measure_alu_peaks(0)
    assert a["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    # 128 FP32 lanes per SM; the paired form issues half the instructions for
    # the same lane work; MUFU ex2 runs at a fraction of the FP32 rate
    assert 64.0 <= a["fp32_fma_per_sm_clk"] <= 136.0, a
    assert 64.0 <= a["fp32x2_fma_per_sm_clk"] <= 272.0, a
    assert 4.0 <= a["ex2_per_sm_clk"] <= 68.0, a
    assert 500.0 <= a["probe_sm_mhz"] <= 3000.0, a
    per_s = a["fp32_fma_per_sm_clk"] * a["sm_count"] * a["probe_sm_mhz"] * 1e6
    assert 0.7 * per_s <= a["fp32_fma_per_s"] <= 1.3 * per_s, a
    # FP64: at most the FP32 rate (GB300's FP64 is far below it)
    assert 0.0 < a["fp64_fma_per_sm_clk"] <= a["fp32_fma_per_sm_clk"], a
    per_s64 = a["fp64_fma_per_sm_clk"] * a["sm_count"] * a["probe_sm_mhz"] * 1e6
    assert 0.7 * per_s64 <= a["fp64_fma_per_s"] <= 1.3 * per_s64, a
    # global atomic adds to distinct L2-resident addresses: between 1e9/s and
    # one per SM-lane per cycle
    lanes_per_s = 128.0 * a["sm_count"] * a["probe_sm_mhz"] * 1e6
    for k in ("red_f32_per_s", "red_f32x4_per_s"):
        assert 1e9 <= a[k] <= lanes_per_s, (k, a)

"""simr_unit_rates: the measured throughput of the execution units the path
kernels use (the roofline's denominators).  The numbers must be positive and
within the GPU's unit counts at its highest clock: 152 SMs x 128 FP32 lanes x 2
flops, 16 special-function results per SM per clock (GB300; generous bounds so
that a clock below the maximum passes)."""
import math

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_unit_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    r = simr.unit_rates()
    assert set(r) == set(simr.api.UNIT_RATES)
    assert all(math.isfinite(v) and v > 0 for v in r.values()), r
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_cap = sms * 128 * 2 * 2.2e9 * 1e-12  # TFLOP/s at 2.2 GHz
    mufu_cap = sms * 16 * 2.2e9 * 1e-12
    assert 0.3 * fp32_cap < r["fp32_fma_tflops"] < 1.05 * fp32_cap, r
    assert 0.3 * fp32_cap < r["fp32_fma2_tflops"] < 1.05 * fp32_cap, r
    assert 0.3 * mufu_cap < r["mufu_rsqrt_tops"] < 1.05 * mufu_cap, r
    # a 64-bit product takes the FMA-heavy pipe longer than an FMA: fewer per second than FMAs (flops / 2)
    assert r["mul_wide_tops"] < 0.5 * r["fp32_fma_tflops"], r
    assert r["fp64_fma_tflops"] < 0.1 * r["fp32_fma_tflops"], r
    assert r["ms"] < 2000.0, r

"""The SIMT FMA-rate probe that gives the arithmetic roofline its denominator."""
import pytest
import torch

pytestmark = pytest.mark.gpu

# GB300: 152 SMs x 128 FP32 lanes x 2 flops per FMA at the 2070 MHz maximum SM clock
NOMINAL_FP32 = 152 * 128 * 2 * 2070e6


def test_fp32_rate_is_near_the_nominal_simt_peak():
    from paper_2508_09568_gb300.bunch import fma_rate
    r = fma_rate(torch.float32)
    assert 0.25 * NOMINAL_FP32 < r < 1.1 * NOMINAL_FP32, r


def test_fp64_rate_is_positive_and_below_fp32():
    from paper_2508_09568_gb300.bunch import fma_rate
    r64 = fma_rate(torch.float64)
    assert 0 < r64 < fma_rate(torch.float32)

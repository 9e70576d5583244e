"""The FP32 multiply-add microbenchmark behind the fused solver's roofline denominator: the
measured rate agrees with SMs x 128 lanes x 2 flop x clock (the figure the bench divides by),
and the paired f32x2 form the butterflies use does not exceed it (it halves issue slots, not
the lanes' throughput), so the derived figure stays the right peak for paired code too."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_fma_rate_matches_the_derived_fp32_peak(lib):
    import torch

    props = torch.cuda.get_device_properties(0)
    derived_max = props.multi_processor_count * 128 * 2 * 2070e6 / 1e12  # at the GB300's top SM clock
    scalar = lib.bccb_fp32_fma_rate(False)
    paired = lib.bccb_fp32_fma_rate(True)
    print(f"FP32 multiply-add rate: scalar {scalar:.1f}, paired {paired:.1f} TFLOP/s; derived {derived_max:.1f}")
    assert 0.7 * derived_max <= scalar <= 1.05 * derived_max
    assert paired <= 1.05 * derived_max


def test_fma_rate_rejects_bad_arguments(lib):
    out = ctypes.c_double(0.0)
    assert lib._lib.bccb_fp32_fma_rate(0, 0, None, ctypes.byref(out)) == lib.ERR_INVALID_ARG
    assert lib._lib.bccb_fp32_fma_rate(0, 10, None, None) == lib.ERR_INVALID_ARG

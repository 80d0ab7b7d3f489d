"""The throughput microbenchmarks that give the FP64 and tensor-core roofline denominators:
they run, return plausible rates for a GB300-class part, and order as the arithmetic says
(one 32-byte K-step holds twice as many bf16 as tf32 elements)."""
import ctypes

import pytest

import paper_1407_0904_gb300 as coffee


def test_peak_entry_points_reject_bad_arguments_on_the_host():
    L = coffee.lib()
    L.coffee_peak_mma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.coffee_peak_fp64.argtypes = [ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double()
    assert L.coffee_peak_fp64(None) == -1
    assert L.coffee_peak_mma(coffee.TF32, 256, None) == -1
    assert L.coffee_peak_mma(coffee.FP64, 256, ctypes.byref(v)) == -1
    assert L.coffee_peak_mma(coffee.TF32X3, 256, ctypes.byref(v)) == -1
    assert L.coffee_peak_mma(coffee.TF32, 64, ctypes.byref(v)) == -1


@pytest.mark.gpu
def test_measured_peaks_are_plausible():
    fp64 = coffee.peak_fp64()
    tf32 = coffee.peak_mma(coffee.TF32, 256)
    bf16 = coffee.peak_mma(coffee.BF16, 256)
    tf32_128 = coffee.peak_mma(coffee.TF32, 128)
    print("fp64 %.2f  tf32 N=256 %.1f  N=128 %.1f  bf16 N=256 %.1f TFLOP/s" % (fp64, tf32, tf32_128, bf16))
    assert 0.3 < fp64 < 10.0
    assert 100.0 < tf32 < 2000.0 and 100.0 < tf32_128 <= tf32 * 1.05
    assert bf16 > 1.5 * tf32 and bf16 < 3000.0

"""CUDA's erff / erfcf stay within the ulp bounds the FP32-sound path uses
(K_ERF = 2 and K_ERFC = 5 ulps), checked over every finite float argument."""

import ctypes
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_erf_erfc_ulp_bounds_exhaustive(tmp_path):
    src = os.path.join(HERE, "cuda", "erf_ulp.cu")
    lib = str(tmp_path / "liberfulp.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                    "-Xcompiler", "-fPIC", src, "-o", lib], check=True)
    f = ctypes.CDLL(lib).erf_ulp_scan
    f.restype = ctypes.c_int
    out = (ctypes.c_float * 2)()
    assert f(out) == 0
    max_erf, max_erfc = out[0], out[1]
    print(f"max ulp error: erff {max_erf:.3f}, erfcf {max_erfc:.3f}")
    assert max_erf <= 2.0
    assert max_erfc <= 5.0


def test_fp64_fma_rate_probe(tmp_path):
    """Measures the FP64 and FP32 FMA rates (the FP64 one bounds the FP64-plain
    build and explains where the synthesis kernel spent its time)."""
    src = os.path.join(HERE, "cuda", "fp64_rate.cu")
    lib = str(tmp_path / "libfprate.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                    "-Xcompiler", "-fPIC", src, "-o", lib], check=True)
    f = ctypes.CDLL(lib).fp_rate
    f.restype = ctypes.c_int
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    assert f(ctypes.byref(f64), ctypes.byref(f32)) == 0
    print(f"FMA rate: FP64 {f64.value / 1e12:.3f} TFLOP/s, FP32 {f32.value / 1e12:.1f} TFLOP/s, "
          f"ratio {f32.value / f64.value:.0f}")
    assert f64.value > 0 and f32.value > f64.value

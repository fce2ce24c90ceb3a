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

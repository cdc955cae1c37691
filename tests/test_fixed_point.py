"""The kernels' FP32 -> int64 fixed-point conversion (the 2^-32 scale of the
children's exact sums) equals CUDA's float -> int64 conversion of x * 2^32,
round to nearest even, for every one of the 2^32 FP32 bit patterns."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_to_fixed_matches_cuda_conversion_exhaustively(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import build
    lib = str(tmp_path / "fixed_point_check.so")
    subprocess.check_call(["nvcc"] + build.NVFLAGS + ["-shared", "-o", lib,
                                                       os.path.join(HERE, "cuda", "fixed_point_check.cu")])
    f = ctypes.CDLL(lib).fixed_point_check
    f.restype = ctypes.c_int
    n_bad, first = ctypes.c_ulonglong(0), ctypes.c_uint(0)
    assert f(ctypes.byref(n_bad), ctypes.byref(first)) == 0
    assert n_bad.value == 0, f"{n_bad.value} patterns differ, first {first.value:#010x}"

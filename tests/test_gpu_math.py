"""The library's table-driven logarithm against the CUDA math library."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_log_fast_within_two_ulp_of_cuda_log():
    import torch
    assert torch.cuda.is_available()
    from paper_2205_03090_gb300 import build, ptflash
    build.build()
    lib = ptflash.load()
    lib.ptflash_check_math.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    lib.ptflash_check_math.restype = ctypes.c_int
    err = ctypes.c_double(-1.0)
    assert lib.ptflash_check_math(1 << 22, ctypes.byref(err)) == 0
    assert 0.0 <= err.value <= 3.0, err.value

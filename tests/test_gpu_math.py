"""The library's table-driven logarithm and exponential against the CUDA
math library."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_log_fast_and_exp_fast_within_a_few_ulp_of_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2205_03090_gb300 import build, ptflash
    build.build()
    lib = ptflash.load()
    lib.ptflash_check_math.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.ptflash_check_math.restype = ctypes.c_int
    el, ee = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    assert lib.ptflash_check_math(1 << 22, ctypes.byref(el), ctypes.byref(ee)) == 0
    print("max ulp: log", el.value, "exp", ee.value)
    assert 0.0 <= el.value <= 3.0, el.value
    assert 0.0 <= ee.value <= 2.0, ee.value

"""The no-allocation flash entry point against the regular one.

ptflash_flash_noalloc serves callers that cannot allocate device memory once
running (its scratch is a fixed device array inside the library).  Called
through the C ABI twice in a row, it must reproduce ptflash_flash: the same
phase labels and statuses, and beta, x, y, K within 1e-8 (the tolerance of
the parity tests).  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2205_03090_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-8


def test_noalloc_matches_flash_twice():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2205_03090_gb300 import build, ptflash
    build.build()
    lib = ptflash.load()
    lib.ptflash_noalloc_max_mixtures.argtypes = [ctypes.c_int]
    lib.ptflash_noalloc_max_mixtures.restype = ctypes.c_int64
    VP, D = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    lib.ptflash_flash_noalloc.argtypes = [ctypes.c_int, D, D, D, D, ctypes.c_int64] + [VP] * 11
    lib.ptflash_flash_noalloc.restype = ctypes.c_int

    comp, cond = wl.workload("nc8_1e6", 50_000)
    nc, n = comp.nc, cond.n
    assert n <= lib.ptflash_noalloc_max_mixtures(nc)
    dev = torch.device("cuda")
    P = torch.tensor(cond.P, device=dev)
    T = torch.tensor(cond.T, device=dev)
    z = torch.tensor(cond.z, device=dev).contiguous()
    fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij)
    ref = fl.ptflash_flash(P, T, z)
    torch.cuda.synchronize()
    refn = {k: getattr(ref, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "K", "status", "iters")}
    fl.close()

    host = [np.ascontiguousarray(a, np.float64) for a in (comp.Tc, comp.Pc, comp.omega, comp.kij)]
    hp = [a.ctypes.data_as(D) for a in host]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = ptflash.Flash.alloc_outputs(fl, n, dev)
        # poison the outputs so stale values cannot pass
        for t in (out.beta, out.x, out.y, out.K):
            t.fill_(float("nan"))
        out.nphase.fill_(-1)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.ptflash_flash_noalloc(nc, *hp, n, *(ctypes.c_void_p(t.data_ptr()) for t in (
            P, T, z, out.nphase, out.beta, out.x, out.y, out.K, out.status, out.iters)), stream)
        assert rc == 0, lib.ptflash_strerror(rc)
        torch.cuda.synchronize()
        if call == 1:
            # the defining property: once the first call has loaded the
            # library's kernels, a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        got = {k: getattr(out, k).cpu().numpy() for k in refn}
        np.testing.assert_array_equal(got["nphase"], refn["nphase"])
        np.testing.assert_array_equal(got["status"], refn["status"])
        for k in ("beta", "x", "y", "K"):
            assert np.all(np.isfinite(got[k])), (call, k)
            assert np.abs(got[k] - refn[k]).max() <= TOL, (call, k)

    # sizes beyond the scratch are rejected with an error, not run
    too_many = lib.ptflash_noalloc_max_mixtures(nc) + 1
    rc = lib.ptflash_flash_noalloc(nc, *hp, too_many, *([ctypes.c_void_p(P.data_ptr())] * 10), stream)
    assert rc == -1

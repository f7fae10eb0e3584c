"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(?:int|int64_t|const char\s*\*)\s+(ptflash_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2205_03090_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert {"ptflash_create", "ptflash_flash", "ptflash_stability", "ptflash_flash_host"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_strerror_without_gpu():
    from paper_2205_03090_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.ptflash_strerror.restype = ctypes.c_char_p
    assert lib.ptflash_strerror(0) == b"ok"
    assert lib.ptflash_strerror(-5).startswith(b"unsupported")
    # argument checks that fail before any CUDA call
    h = ctypes.c_void_p()
    assert lib.ptflash_create(None, 4, 10) == -1
    assert lib.ptflash_create(ctypes.byref(h), 17, 10) == -5
    assert lib.ptflash_destroy(None) == -1


def test_batch_argument_checks_without_gpu():
    """ptflash_batch_create validates every system's data on the host before
    any CUDA call: nc outside 2..16, an asymmetric or nonzero-diagonal k_ij, a
    non-positive critical constant, a negative mixture count."""
    import numpy as np
    from paper_2205_03090_gb300 import build
    lib = ctypes.CDLL(build.build())
    P = ctypes.c_void_p
    lib.ptflash_batch_create.argtypes = [P, ctypes.c_int, P, P, P, P, P, P]

    def create(nc, n, Tc, Pc, om, kij):
        h = ctypes.c_void_p()
        arrs = [np.ascontiguousarray(a) for a in (nc, n, Tc, Pc, om, kij)]
        rc = lib.ptflash_batch_create(ctypes.byref(h), len(nc), *[a.ctypes.data_as(P) for a in arrs])
        return rc, h

    nc = np.array([3], np.int32)
    n = np.array([10], np.int64)
    Tc, Pc, om = np.array([300.0, 400.0, 500.0]), np.array([4.0, 3.5, 3.0]), np.array([0.1, 0.2, 0.3])
    kij = np.zeros((3, 3))
    bad_k = kij.copy()
    bad_k[0, 1] = 0.05  # asymmetric
    diag_k = kij.copy()
    diag_k[1, 1] = 0.01  # nonzero diagonal
    assert create(np.array([1], np.int32), n, Tc[:1], Pc[:1], om[:1], kij[:1, :1])[0] == -5
    assert create(np.array([17], np.int32), n, np.ones(17), np.ones(17), np.ones(17), np.zeros((17, 17)))[0] == -5
    assert create(nc, n, Tc, Pc, om, bad_k)[0] == -1
    assert create(nc, n, Tc, Pc, om, diag_k)[0] == -1
    assert create(nc, n, Tc, np.array([4.0, -1.0, 3.0]), om, kij)[0] == -1
    assert create(nc, np.array([-1], np.int64), Tc, Pc, om, kij)[0] == -1
    h = ctypes.c_void_p()
    assert lib.ptflash_batch_create(None, 1, None, None, None, None, None, None) == -1
    assert lib.ptflash_batch_create(ctypes.byref(h), 0, None, None, None, None, None, None) == -1


def test_default_options_without_gpu():
    """ptflash_default_options fills the paper's caps and tolerances (and the
    readings' split caps) without touching the GPU; the binding's struct has
    the C layout."""
    from paper_2205_03090_gb300 import build, ptflash
    build.build()
    d = ptflash.default_options()
    assert d["max_ss_stab"] == 9 and d["max_tr_stab"] == 20  # K_ss, K_tr of Alg. 2
    assert d["max_ss_split"] == 9 and d["max_tr_split"] == 60 and d["max_polish"] == 10
    assert d["tol_stab"] == 1e-6 and d["tol_split_tr"] == 1e-8 and d["tol_fug"] == 0.98e-10
    assert d["p_l"] == 0.02 and d["p_r"] == 0.98 and d["nn_lnk_dev"] == 0.3
    assert d["tr_lanes"] == 0  # one lane per trust-region run, several in the drain
    assert ctypes.sizeof(ptflash.ptflash_options) == 88  # the C sizeof on LP64 (x86-64 and aarch64)
    assert ptflash.load().ptflash_default_options(None) == -1


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_options_layout_matches_header(tmp_path):
    """Every field of ptflash_options sits at the same offset in the C header
    (compiled by the host C compiler) and in the binding's ctypes mirror, so a
    field added on one side only is caught without a GPU."""
    from paper_2205_03090_gb300 import ptflash
    fields = [f for f, _ in ptflash.ptflash_options._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'    printf("%s %zu\\n", "{f}", offsetof(ptflash_options, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ptflash.h"\nint main(void) {\n'
                   f'{body}\n    printf("sizeof %zu\\n", sizeof(ptflash_options));\n    return 0;\n}}\n')
    exe = str(tmp_path / "layout")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe], check=True)
    out = dict(line.split() for line in subprocess.run([exe], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for f in fields:
        assert int(out[f]) == getattr(ptflash.ptflash_options, f).offset, f
    assert int(out["sizeof"]) == ctypes.sizeof(ptflash.ptflash_options)

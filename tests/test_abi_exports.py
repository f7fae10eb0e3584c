"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

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

"""CPU oracle for the batched isothermal two-phase flash (arXiv 2205.03090).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2205_03090_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``ptflash_oracle.c`` (plain FP64 C, one mixture at a
time, OpenMP over mixtures); this module only compiles it with gcc and
marshals NumPy arrays through ctypes.  ``mlp`` holds the FP64 reference of the
two networks (Sec. 4 of the paper).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptflash_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

# status bits (same values as the CUDA library documents)
ST_PRECHECK_UNSTABLE = 1
ST_STAB_RUN = 2
ST_STAB_TR = 4
ST_SPLIT_TR = 8
ST_MAXITER = 16
ST_COLLAPSE = 32
ST_NONFINITE = 64


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP).

    -ffp-contract=off keeps the x86 and Arm results identical (no FMA
    contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)


def _lib_handle():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        sysargs = [ctypes.c_int, _D, _D, _D, _D]
        lib.oracle_flash_batch.argtypes = sysargs + [ctypes.c_int64, _D, _D, _D, _I, _D, _D, _D, _D, _I, _I, _D,
                                                     _D, ctypes.c_int]
        lib.oracle_flash_batch.restype = ctypes.c_int
        lib.oracle_tpd_min_batch.argtypes = sysargs + [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int]
        lib.oracle_tpd_min_batch.restype = ctypes.c_int
        lib.oracle_stability_batch.argtypes = sysargs + [ctypes.c_int64, _D, _D, _D, _I, _D, _D, ctypes.c_int]
        lib.oracle_stability_batch.restype = ctypes.c_int
        lib.oracle_mix_consts.argtypes = sysargs + [ctypes.c_double, ctypes.c_double, _D, _D]
        lib.oracle_cubic_roots.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_cubic_roots.restype = ctypes.c_int
        lib.oracle_eos.argtypes = sysargs + [ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D]
        lib.oracle_eos.restype = ctypes.c_int
        lib.oracle_wilson.argtypes = sysargs + [ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_rr.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.oracle_rr.restype = ctypes.c_int
        lib.oracle_tr_subproblem.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, _D]
        lib.oracle_tr_subproblem.restype = ctypes.c_double
        lib.oracle_dlnphi_dPT.argtypes = sysargs + [ctypes.c_double, ctypes.c_double, _D, _D, _D]
        lib.oracle_dlnphi_dPT.restype = ctypes.c_int
        lib.oracle_flash_jacobian_batch.argtypes = sysargs + [ctypes.c_int64, _D, _D, _D, _I, _D, _D, _D, _D, _I,
                                                              ctypes.c_int]
        lib.oracle_flash_jacobian_batch.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _pi(a):
    return a.ctypes.data_as(_I) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class System:
    """Component data: Tc [K], Pc [any pressure unit, same as P], omega, k_ij."""

    def __init__(self, Tc, Pc, omega, kij):
        self.Tc = _f64(Tc)
        self.Pc = _f64(Pc)
        self.omega = _f64(omega)
        self.kij = _f64(kij).reshape(len(self.Tc), len(self.Tc))
        self.nc = len(self.Tc)

    def _args(self):
        return (self.nc, _p(self.Tc), _p(self.Pc), _p(self.omega), _p(self.kij))


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def flash(sysc: System, P, T, z, nthreads: int | None = None):
    """Plain flash (Sec. 2.2.3) of n mixtures; z is component-major [nc, n].

    Returns a dict of NumPy arrays: nphase, beta, x, y, K ([nc, n]), status,
    iters (packed: split SS | split TR << 8 | stab SS << 16 | stab TR << 24),
    tm_min (NaN where stability analysis did not run), ops: the algorithmic
    FP64 work summed over the batch, [stage, kind] with stages (prep+precheck,
    stability SS, stability TR, split SS, split TR) and kinds (flops: add and
    multiply 1, fused multiply-add 2; divisions; square roots; exponentials;
    logarithms), and flops = ops[:, 0]."""
    P = _f64(P)
    T = _f64(T)
    z = _f64(z)
    n = P.shape[0]
    nc = sysc.nc
    assert z.shape == (nc, n)
    out = dict(nphase=np.zeros(n, np.int32), beta=np.zeros(n), x=np.zeros((nc, n)), y=np.zeros((nc, n)),
               K=np.zeros((nc, n)), status=np.zeros(n, np.int32), iters=np.zeros(n, np.int32),
               tm_min=np.zeros(n), ops=np.zeros((5, 5)))
    rc = _lib_handle().oracle_flash_batch(*sysc._args(), n, _p(P), _p(T), _p(z), _pi(out["nphase"]),
                                          _p(out["beta"]), _p(out["x"]), _p(out["y"]), _p(out["K"]),
                                          _pi(out["status"]), _pi(out["iters"]), _p(out["tm_min"]),
                                          _p(out["ops"]), nthreads or default_threads())
    if rc:
        raise ValueError("oracle_flash_batch failed")
    out["flops"] = out["ops"][:, 0].copy()
    return out


def tpd_min(sysc: System, P, T, z, nthreads: int | None = None):
    """Minimum tpd over both trials, each converged to its stationary point."""
    P = _f64(P)
    T = _f64(T)
    z = _f64(z)
    n = P.shape[0]
    out = np.zeros(n)
    rc = _lib_handle().oracle_tpd_min_batch(*sysc._args(), n, _p(P), _p(T), _p(z), _p(out),
                                            nthreads or default_threads())
    if rc:
        raise ValueError("oracle_tpd_min_batch failed")
    return out


def stability(sysc: System, P, T, z, nthreads: int | None = None):
    """Stability analysis alone (Alg. 2, two Wilson trials): stable flag,
    min tm and the K re-estimate."""
    P = _f64(P)
    T = _f64(T)
    z = _f64(z)
    n = P.shape[0]
    stable = np.zeros(n, np.int32)
    tm = np.zeros(n)
    K = np.zeros((sysc.nc, n))
    rc = _lib_handle().oracle_stability_batch(*sysc._args(), n, _p(P), _p(T), _p(z), _pi(stable), _p(tm), _p(K),
                                              nthreads or default_threads())
    if rc:
        raise ValueError("oracle_stability_batch failed")
    return dict(stable=stable, tm_min=tm, K=K)


def mix_consts(sysc: System, P: float, T: float):
    Ai = np.zeros(sysc.nc)
    Bi = np.zeros(sysc.nc)
    _lib_handle().oracle_mix_consts(*sysc._args(), P, T, _p(Ai), _p(Bi))
    return Ai, Bi


def cubic_roots(A: float, B: float):
    r = np.zeros(3)
    n = _lib_handle().oracle_cubic_roots(A, B, _p(r))
    return r[:n].copy()


def eos(sysc: System, P: float, T: float, c, with_jac: bool = False):
    """Z, ln phi (Eq. lnphi) and optionally J = n_T d ln phi / d n."""
    c = _f64(c)
    lnphi = np.zeros(sysc.nc)
    J = np.zeros((sysc.nc, sysc.nc)) if with_jac else None
    Z = ctypes.c_double()
    AB = np.zeros(2)
    rc = _lib_handle().oracle_eos(*sysc._args(), P, T, _p(c), ctypes.byref(Z), _p(lnphi), _p(J), _p(AB))
    if rc:
        raise ValueError("no admissible root")
    return (Z.value, lnphi, J, AB) if with_jac else (Z.value, lnphi)


def wilson(sysc: System, P: float, T: float):
    lnK = np.zeros(sysc.nc)
    _lib_handle().oracle_wilson(*sysc._args(), P, T, _p(lnK))
    return lnK


def rr(z, K):
    z = _f64(z)
    K = _f64(K)
    th = ctypes.c_double()
    rc = _lib_handle().oracle_rr(len(z), _p(z), _p(K), ctypes.byref(th))
    return None if rc else th.value


def tr_subproblem(H, g, radius, mdiag=None):
    H = _f64(H)
    g = _f64(g)
    d = np.zeros(len(g))
    md = _f64(mdiag) if mdiag is not None else None
    pred = _lib_handle().oracle_tr_subproblem(len(g), _p(H), _p(g), _p(md), radius, _p(d))
    return d, pred


def dlnphi_dPT(sysc: System, P: float, T: float, c):
    """d ln phi_i / dP and d ln phi_i / dT at fixed composition c."""
    c = _f64(c)
    dP = np.zeros(sysc.nc)
    dT = np.zeros(sysc.nc)
    _lib_handle().oracle_dlnphi_dPT(*sysc._args(), P, T, _p(c), _p(dP), _p(dT))
    return dP, dT


def flash_jacobian(sysc: System, P, T, z, res, nthreads: int | None = None):
    """Jacobian of (beta, x, y) with respect to (P, T, z) at the converged
    results `res` (a flash() dict): array [n, 1 + 2 nc, nc + 2] (rows beta,
    x_1..x_nc, y_1..y_nc; columns P, T, z_1..z_nc, z read as mole numbers) and
    ok[n] (0, or -1 where the split Hessian is singular)."""
    P, T, z = _f64(P), _f64(T), _f64(z)
    n, nc = P.shape[0], sysc.nc
    jac = np.zeros((n, 1 + 2 * nc, nc + 2))
    ok = np.zeros(n, np.int32)
    nph = np.ascontiguousarray(res["nphase"], np.int32)
    rc = _lib_handle().oracle_flash_jacobian_batch(*sysc._args(), n, _p(P), _p(T), _p(z), _pi(nph),
                                                   _p(_f64(res["beta"])), _p(_f64(res["x"])), _p(_f64(res["y"])),
                                                   _p(jac), _pi(ok), nthreads or default_threads())
    if rc:
        raise ValueError("oracle_flash_jacobian_batch failed")
    return jac, ok

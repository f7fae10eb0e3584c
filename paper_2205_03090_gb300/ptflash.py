"""Thin Python binding of the C ABI in include/ptflash.h.

Argument marshalling only: every step of the flash runs in the CUDA library
(_build/libptflash.so).  torch supplies device memory and streams.  There is
no CPU fallback -- if the library is missing or CUDA is unavailable, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libptflash.so")

PTF_ST_PRECHECK_UNSTABLE = 1
PTF_ST_STAB_RUN = 2
PTF_ST_STAB_TR = 4
PTF_ST_SPLIT_TR = 8
PTF_ST_MAXITER = 16
PTF_ST_COLLAPSE = 32
PTF_ST_NONFINITE = 64
PTF_ST_NN_STABLE = 128
PTF_ST_NN_UNSTABLE = 256
PTF_ST_NN_INIT = 512
PTF_ST_NN_REJECTED = 1024

_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.POINTER(ctypes.c_double)


class PtflashError(RuntimeError):
    pass


class ptflash_options(ctypes.Structure):
    _fields_ = [("use_nn", ctypes.c_int32), ("p_l", ctypes.c_double), ("p_r", ctypes.c_double),
                ("max_ss_stab", ctypes.c_int32), ("max_tr_stab", ctypes.c_int32), ("max_ss_split", ctypes.c_int32),
                ("max_tr_split", ctypes.c_int32), ("max_polish", ctypes.c_int32), ("tol_stab", ctypes.c_double),
                ("tol_split_tr", ctypes.c_double), ("tol_fug", ctypes.c_double), ("nn_lnk_dev", ctypes.c_double),
                ("tr_lanes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# ptflash_options fields a caller may set through **opts (0 = default)
OPTION_FIELDS = ("max_ss_stab", "max_tr_stab", "max_ss_split", "max_tr_split", "max_polish", "tol_stab",
                 "tol_split_tr", "tol_fug", "nn_lnk_dev", "tr_lanes")


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PtflashError(f"CUDA library not built: {path} (run paper_2205_03090_gb300/build.py)")
    lib = ctypes.CDLL(path)
    lib.ptflash_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, _I64]
    lib.ptflash_destroy.argtypes = [_VP]
    lib.ptflash_set_components.argtypes = [_VP, ctypes.c_int, _D, _D, _D, _D]
    dev = [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ptflash_options), _VP]
    lib.ptflash_flash.argtypes = dev
    lib.ptflash_flash_host.argtypes = dev
    lib.ptflash_stability.argtypes = [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]
    lib.ptflash_last_counts.argtypes = [_VP, ctypes.POINTER(_I64)]
    lib.ptflash_set_profiling.argtypes = [_VP, ctypes.c_int]
    lib.ptflash_last_stage_ms.argtypes = [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    _F = ctypes.POINTER(ctypes.c_float)
    lib.ptflash_nn_set.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _F, _F, _F]
    lib.ptflash_nn_set_arch.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _F, _F, _F]
    lib.ptflash_nn_set_theta_loss.argtypes = [_VP, ctypes.c_int, ctypes.c_float]
    lib.ptflash_nn_param_count_arch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.ptflash_nn_param_count_arch.restype = ctypes.c_int64
    lib.ptflash_nn_get.argtypes = [_VP, ctypes.c_int, _F]
    lib.ptflash_nn_param_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.ptflash_nn_param_count.restype = ctypes.c_int64
    lib.ptflash_nn_features.argtypes = [_VP, ctypes.c_int, _I64, _VP, _VP, _VP, _VP, _VP]
    lib.ptflash_nn_infer.argtypes = [_VP, ctypes.c_int, _I64, _VP, _VP, _VP, _VP, _VP]
    lib.ptflash_nn_train_steps.argtypes = [_VP, ctypes.c_int, _I64, _VP, _VP, _VP, _I64, ctypes.c_int, _F,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP, _VP]
    lib.ptflash_nn_eval.argtypes = [_VP, ctypes.c_int, _I64, _VP, _VP, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), _VP]
    for f in ("ptflash_nn_set", "ptflash_nn_get", "ptflash_nn_features", "ptflash_nn_infer", "ptflash_nn_train_steps",
              "ptflash_nn_eval", "ptflash_nn_set_arch", "ptflash_nn_set_theta_loss"):
        getattr(lib, f).restype = ctypes.c_int
    lib.ptflash_flash_adjoint.argtypes = [_VP, _I64] + [_VP] * 15
    lib.ptflash_flash_adjoint.restype = ctypes.c_int
    _I32P = ctypes.POINTER(ctypes.c_int32)
    lib.ptflash_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, _I32P, ctypes.POINTER(_I64), _D, _D, _D,
                                         _D]
    lib.ptflash_batch_destroy.argtypes = [_VP]
    lib.ptflash_batch_flash.argtypes = [_VP] + [_VP] * 10 + [_VP]
    lib.ptflash_batch_tune.argtypes = [_VP] + [_VP] * 10 + [_I32P, ctypes.POINTER(ctypes.c_float)]
    lib.ptflash_batch_info.argtypes = [_VP, _I32P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]
    for f in ("ptflash_batch_create", "ptflash_batch_destroy", "ptflash_batch_flash", "ptflash_batch_tune",
              "ptflash_batch_info"):
        getattr(lib, f).restype = ctypes.c_int
    lib.ptflash_default_options.argtypes = [ctypes.POINTER(ptflash_options)]
    lib.ptflash_default_options.restype = ctypes.c_int
    lib.ptflash_phase_eos.argtypes = [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP]
    lib.ptflash_phase_eos.restype = ctypes.c_int
    lib.ptflash_fp64_fma_rate.argtypes = [_I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.ptflash_fp64_fma_rate.restype = ctypes.c_int
    lib.ptflash_strerror.argtypes = [ctypes.c_int]
    lib.ptflash_strerror.restype = ctypes.c_char_p
    lib.ptflash_last_cuda_error.restype = ctypes.c_char_p
    for f in ("ptflash_create", "ptflash_destroy", "ptflash_set_components", "ptflash_flash", "ptflash_flash_host",
              "ptflash_stability", "ptflash_last_counts", "ptflash_set_profiling", "ptflash_last_stage_ms"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        lib = load()
        msg = lib.ptflash_strerror(rc).decode()
        cuda = lib.ptflash_last_cuda_error().decode()
        raise PtflashError(f"ptflash error {rc}: {msg}" + (f" ({cuda})" if cuda else ""))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _opts(use_nn=False, p_l=0.02, p_r=0.98, **caps):
    o = ptflash_options()
    o.use_nn = 1 if use_nn else 0
    o.p_l = p_l
    o.p_r = p_r
    for k, v in caps.items():
        if k not in OPTION_FIELDS:
            raise TypeError(f"unknown flash option {k}")
        setattr(o, k, v)
    return o


def default_options() -> dict:
    """The library's default caps and tolerances (ptflash_default_options)."""
    o = ptflash_options()
    _check(load().ptflash_default_options(ctypes.byref(o)))
    return {k: getattr(o, k) for k in ("p_l", "p_r") + OPTION_FIELDS}


def fp64_fma_rate(iters: int = 6000):
    """FP64 FMA throughput of the current device (ptflash_fp64_fma_rate):
    (TFLOP/s, ms of the timed launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().ptflash_fp64_fma_rate(int(iters), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


@dataclass
class FlashResult:
    nphase: "object"
    beta: "object"
    x: "object"
    y: "object"
    K: "object"
    status: "object"
    iters: "object"


class Flash:
    """A flash context on the current CUDA device (ptflash_create / set_components)."""

    def __init__(self, Tc, Pc, omega, kij, n_max: int = 1 << 20, nc_max: int | None = None):
        lib = load()
        Tc = np.ascontiguousarray(Tc, np.float64)
        nc = int(Tc.shape[0])
        self.nc = nc
        self.n_max = int(n_max)
        self._nn_scaler = {}  # which -> (mean, std) of the network features
        h = _VP()
        _check(lib.ptflash_create(ctypes.byref(h), nc_max or nc, self.n_max))
        self._h = h
        arrs = [Tc, np.ascontiguousarray(Pc, np.float64), np.ascontiguousarray(omega, np.float64),
                np.ascontiguousarray(kij, np.float64).reshape(-1)]
        _check(lib.ptflash_set_components(h, nc, *[a.ctypes.data_as(_D) for a in arrs]))

    def close(self):
        if getattr(self, "_h", None):
            load().ptflash_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_outputs(self, n: int, device="cuda", with_iters=True):
        import torch
        f64 = dict(dtype=torch.float64, device=device)
        i32 = dict(dtype=torch.int32, device=device)
        return FlashResult(torch.empty(n, **i32), torch.empty(n, **f64), torch.empty(self.nc, n, **f64),
                           torch.empty(self.nc, n, **f64), torch.empty(self.nc, n, **f64), torch.empty(n, **i32),
                           torch.empty(n, **i32) if with_iters else None)

    def ptflash_flash(self, P, T, z, out: FlashResult | None = None, use_nn=False, p_l=0.02, p_r=0.98,
                      stream=None, **caps) -> FlashResult:
        """Device tensors P[n], T[n], z[nc, n] (float64, contiguous).  caps:
        ptflash_options caps and tolerances (OPTION_FIELDS; 0 = default)."""
        n = int(P.shape[0])
        assert z.shape == (self.nc, n) and P.is_cuda and z.is_contiguous()
        out = out or self.alloc_outputs(n, P.device)
        o = _opts(use_nn, p_l, p_r, **caps)
        _check(load().ptflash_flash(self._h, n, _ptr(P), _ptr(T), _ptr(z), _ptr(out.nphase), _ptr(out.beta),
                                    _ptr(out.x), _ptr(out.y), _ptr(out.K), _ptr(out.status), _ptr(out.iters),
                                    ctypes.byref(o), _stream_handle(stream)))
        return out

    def ptflash_flash_host(self, P, T, z, out=None, use_nn=False, p_l=0.02, p_r=0.98, stream=None, **caps):
        """Host tensors (pinned CPU torch tensors or NumPy arrays); returns host outputs."""
        import torch
        n = int(P.shape[0])
        if out is None:
            out = FlashResult(torch.empty(n, dtype=torch.int32), torch.empty(n, dtype=torch.float64),
                              torch.empty(self.nc, n, dtype=torch.float64),
                              torch.empty(self.nc, n, dtype=torch.float64),
                              torch.empty(self.nc, n, dtype=torch.float64), torch.empty(n, dtype=torch.int32),
                              torch.empty(n, dtype=torch.int32))
        o = _opts(use_nn, p_l, p_r, **caps)
        _check(load().ptflash_flash_host(self._h, n, _ptr(P), _ptr(T), _ptr(z), _ptr(out.nphase), _ptr(out.beta),
                                         _ptr(out.x), _ptr(out.y), _ptr(out.K), _ptr(out.status), _ptr(out.iters),
                                         ctypes.byref(o), _stream_handle(stream)))
        return out

    def ptflash_phase_eos(self, P, T, c, stream=None):
        """Z[n] and ln phi[nc, n] of the phase of composition c[nc, n] (device
        tensors) at P[n], T[n]."""
        import torch
        n = int(P.shape[0])
        assert c.shape == (self.nc, n) and c.is_contiguous()
        Z = torch.empty(n, dtype=torch.float64, device=P.device)
        lnphi = torch.empty(self.nc, n, dtype=torch.float64, device=P.device)
        _check(load().ptflash_phase_eos(self._h, n, _ptr(P), _ptr(T), _ptr(c), _ptr(Z), _ptr(lnphi),
                                        _stream_handle(stream)))
        return Z, lnphi

    def ptflash_stability(self, P, T, z, stream=None):
        import torch
        n = int(P.shape[0])
        dev = P.device
        stable = torch.empty(n, dtype=torch.int32, device=dev)
        tm = torch.empty(n, dtype=torch.float64, device=dev)
        K = torch.empty(self.nc, n, dtype=torch.float64, device=dev)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        _check(load().ptflash_stability(self._h, n, _ptr(P), _ptr(T), _ptr(z), _ptr(stable), _ptr(tm), _ptr(K),
                                        _ptr(status), _stream_handle(stream)))
        return stable, tm, K, status

    def ptflash_flash_adjoint(self, P, T, z, res: FlashResult, gbeta=None, gx=None, gy=None, stream=None):
        """dl/dP, dl/dT, dl/dz for l = gbeta.beta + gx.x + gy.y at the flash
        results `res` of (P, T, z); returns (gP[n], gT[n], gz[nc, n], astatus[n])."""
        import torch
        n = int(P.shape[0])
        dev = P.device
        gP = torch.empty(n, dtype=torch.float64, device=dev)
        gT = torch.empty(n, dtype=torch.float64, device=dev)
        gz = torch.empty(self.nc, n, dtype=torch.float64, device=dev)
        ast = torch.empty(n, dtype=torch.int32, device=dev)
        c = lambda t: t.contiguous() if t is not None else None
        gbeta, gx, gy = c(gbeta), c(gx), c(gy)
        _check(load().ptflash_flash_adjoint(self._h, n, _ptr(P), _ptr(T), _ptr(z), _ptr(res.nphase), _ptr(res.beta),
                                            _ptr(res.x), _ptr(res.y), _ptr(gbeta), _ptr(gx), _ptr(gy), _ptr(gP),
                                            _ptr(gT), _ptr(gz), _ptr(ast), _stream_handle(stream)))
        return gP, gT, gz, ast

    STAGES = ("prep_precheck", "stab_ss", "stab_tr", "stab_decide", "split_ss", "split_tr")

    def ptflash_set_profiling(self, enable: bool = True):
        _check(load().ptflash_set_profiling(self._h, 1 if enable else 0))

    def ptflash_last_stage_ms(self):
        ms = (ctypes.c_double * 6)()
        _check(load().ptflash_last_stage_ms(self._h, ms, 6))
        return dict(zip(self.STAGES, list(ms)))

    # ---- learned form (Sec. 4): which = 0 classifier, 1 initializer ----
    def ptflash_nn_set(self, which: int, hidden: int, theta, mean, std, arch: int = 0):
        F = ctypes.POINTER(ctypes.c_float)
        arrs = [np.ascontiguousarray(a, np.float32) for a in (theta, mean, std)]
        _check(load().ptflash_nn_set_arch(self._h, which, arch, hidden, *[a.ctypes.data_as(F) for a in arrs]))

    def ptflash_nn_set_theta_loss(self, which: int, weight: float):
        _check(load().ptflash_nn_set_theta_loss(self._h, which, float(weight)))

    def ptflash_nn_get(self, which: int, count: int):
        out = np.zeros(count, np.float32)
        _check(load().ptflash_nn_get(self._h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def ptflash_nn_features(self, which, P, T, z, X, stream=None):
        _check(load().ptflash_nn_features(self._h, which, int(P.shape[0]), _ptr(P), _ptr(T), _ptr(z), _ptr(X),
                                          _stream_handle(stream)))

    def ptflash_nn_infer(self, which, P, T, z, out, stream=None):
        _check(load().ptflash_nn_infer(self._h, which, int(P.shape[0]), _ptr(P), _ptr(T), _ptr(z), _ptr(out),
                                       _stream_handle(stream)))

    def ptflash_nn_train_steps(self, which, X, Y, perm, steps, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8,
                               loss=None, stream=None):
        lr = np.ascontiguousarray(lr, np.float32)
        _check(load().ptflash_nn_train_steps(self._h, which, int(X.shape[1]), _ptr(X), _ptr(Y), _ptr(perm), steps,
                                             batch, lr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), beta1, beta2,
                                             eps, _ptr(loss), _stream_handle(stream)))

    def ptflash_nn_eval(self, which, X, Y, stream=None):
        l, a = ctypes.c_double(), ctypes.c_double()
        _check(load().ptflash_nn_eval(self._h, which, int(X.shape[1]), _ptr(X), _ptr(Y), ctypes.byref(l),
                                      ctypes.byref(a), _stream_handle(stream)))
        return l.value, a.value

    def ptflash_last_counts(self):
        c = (_I64 * 4)()
        _check(load().ptflash_last_counts(self._h, c))
        return dict(stab=c[0], split=c[1], stab_tr=c[2], split_tr=c[3])


class Batch:
    """An uneven batch of fluid systems (ptflash_batch_create).

    systems: list of (Tc, Pc, omega, kij) per system; n: mixtures per system.
    Mixture arrays are packed by system: P, T and the per-mixture outputs hold
    sum(n) entries in system order; z, x, y, K are the concatenation of each
    system's flattened component-major [nc_s, n_s] block."""

    def __init__(self, systems, n):
        lib = load()
        self.nc = np.array([len(np.atleast_1d(s[0])) for s in systems], np.int32)
        self.n = np.array(n, np.int64)
        self.off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.zoff = np.concatenate([[0], np.cumsum(self.nc.astype(np.int64) * self.n)]).astype(np.int64)
        self.N = int(self.off[-1])
        self.Z = int(self.zoff[-1])
        cat = lambda k: np.ascontiguousarray(np.concatenate([np.ravel(np.asarray(s[k], np.float64)) for s in systems]))
        Tc, Pc, om, kij = cat(0), cat(1), cat(2), cat(3)
        h = _VP()
        _check(lib.ptflash_batch_create(ctypes.byref(h), len(systems), self.nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        self.n.ctypes.data_as(ctypes.POINTER(_I64)), Tc.ctypes.data_as(_D),
                                        Pc.ctypes.data_as(_D), om.ctypes.data_as(_D), kij.ctypes.data_as(_D)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().ptflash_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, parts, device="cuda"):
        """Pack per-system (P, T, z[nc, n]) NumPy arrays into device tensors."""
        import torch
        P = torch.tensor(np.concatenate([p[0] for p in parts]), dtype=torch.float64, device=device)
        T = torch.tensor(np.concatenate([p[1] for p in parts]), dtype=torch.float64, device=device)
        z = torch.tensor(np.concatenate([np.ravel(p[2]) for p in parts]), dtype=torch.float64, device=device)
        return P, T, z

    def alloc_outputs(self, device="cuda"):
        import torch
        f64 = dict(dtype=torch.float64, device=device)
        i32 = dict(dtype=torch.int32, device=device)
        return FlashResult(torch.empty(self.N, **i32), torch.empty(self.N, **f64), torch.empty(self.Z, **f64),
                           torch.empty(self.Z, **f64), torch.empty(self.Z, **f64), torch.empty(self.N, **i32),
                           torch.empty(self.N, **i32))

    def unpack(self, out: FlashResult, s: int):
        """System s's results as NumPy arrays (x, y, K shaped [nc, n])."""
        a, b = int(self.off[s]), int(self.off[s + 1])
        za, zb = int(self.zoff[s]), int(self.zoff[s + 1])
        nc, n = int(self.nc[s]), int(self.n[s])
        cpu = lambda t, lo, hi: t[lo:hi].cpu().numpy()
        return dict(nphase=cpu(out.nphase, a, b), beta=cpu(out.beta, a, b), status=cpu(out.status, a, b),
                    iters=cpu(out.iters, a, b), x=cpu(out.x, za, zb).reshape(nc, n), y=cpu(out.y, za, zb).reshape(nc, n),
                    K=cpu(out.K, za, zb).reshape(nc, n))

    def ptflash_batch_flash(self, P, T, z, out: FlashResult | None = None, stream=None) -> FlashResult:
        out = out or self.alloc_outputs(P.device)
        _check(load().ptflash_batch_flash(self._h, _ptr(P), _ptr(T), _ptr(z), _ptr(out.nphase), _ptr(out.beta),
                                          _ptr(out.x), _ptr(out.y), _ptr(out.K), _ptr(out.status), _ptr(out.iters),
                                          _stream_handle(stream)))
        return out

    def ptflash_batch_tune(self, P, T, z, out: FlashResult | None = None):
        """Returns ({nc: blocks per SM (0 = default)}, {nc: best group ms})."""
        out = out or self.alloc_outputs(P.device)
        bps = (ctypes.c_int32 * 17)()
        ms = (ctypes.c_float * 17)()
        _check(load().ptflash_batch_tune(self._h, _ptr(P), _ptr(T), _ptr(z), _ptr(out.nphase), _ptr(out.beta),
                                         _ptr(out.x), _ptr(out.y), _ptr(out.K), _ptr(out.status), _ptr(out.iters),
                                         bps, ms))
        present = sorted(set(int(k) for k, m in zip(self.nc, self.n) if m > 0))
        return {k: int(bps[k]) for k in present}, {k: float(ms[k]) for k in present}

    def ptflash_batch_info(self):
        g, nodes, n = ctypes.c_int32(), _I64(), _I64()
        _check(load().ptflash_batch_info(self._h, ctypes.byref(g), ctypes.byref(nodes), ctypes.byref(n)))
        return dict(groups=g.value, graph_nodes=nodes.value, mixtures=n.value)

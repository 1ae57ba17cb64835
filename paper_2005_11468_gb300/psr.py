"""ctypes binding of libpsr (include/psr.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback. Device arrays
are torch CUDA tensors (float64 / int32, contiguous), passed by pointer with the
current torch stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpsr.so")

PSR_OK = 0
PSR_CONVERGED, PSR_MAX_ITER, PSR_NONFINITE, PSR_TS_EXHAUSTED, PSR_REFINE_FALLBACK = 0, 1, 2, 4, 5
PSR_BAD_INPUT = 7
PSR_JAC_ANALYTIC, PSR_JAC_FD = 0, 1
CONVERGED_STATES = (PSR_CONVERGED, PSR_REFINE_FALLBACK)
PSR_FP64, PSR_MIXED = 0, 1
PSR_ADIABATIC, PSR_FIXED_T = 0, 1
PSR_PATH_AUTO, PSR_PATH_WARP, PSR_PATH_BLOCK = 0, 1, 2
PSR_LU_CUDA_CORES, PSR_LU_TF32, PSR_LU_3XTF32 = 0, 1, 3


class PsrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpsr error {code}: {msg}")
        self.code = code


class CMechInfo(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("I", ctypes.c_int32), ("n_elements", ctypes.c_int32),
                ("n_third_body", ctypes.c_int32), ("n_falloff", ctypes.c_int32),
                ("has_soot", ctypes.c_int32)]


class COptions(ctypes.Structure):
    _fields_ = [("ftol", ctypes.c_double), ("step_rtol", ctypes.c_double),
                ("step_atol_y", ctypes.c_double), ("step_atol_t", ctypes.c_double),
                ("ts_rtol", ctypes.c_double), ("ts_atol_y", ctypes.c_double),
                ("dt0_over_tau", ctypes.c_double), ("dt_shrink", ctypes.c_double),
                ("y_floor", ctypes.c_double), ("t_min", ctypes.c_double), ("t_max", ctypes.c_double),
                ("max_newton", ctypes.c_int32), ("max_damp", ctypes.c_int32),
                ("max_ts_rounds", ctypes.c_int32), ("ts_steps", ctypes.c_int32),
                ("ts_newton", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("energy", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("mixed_fallback", ctypes.c_int32),
                ("jacobian", ctypes.c_int32), ("mixed_max_newton", ctypes.c_int32),
                ("jac_age", ctypes.c_int32), ("ts_linear", ctypes.c_int32), ("path", ctypes.c_int32),
                ("handoff", ctypes.c_int32), ("lu_tensor", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("spin_limit", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libpsr; raises if it was not built (run __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        L.psr_mech_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
        L.psr_mech_load_mem.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.psr_mech_info_get.argtypes = [vp, ctypes.POINTER(CMechInfo)]
        L.psr_mech_weights.argtypes = [vp, dp]
        L.psr_mech_free.argtypes = [vp]
        L.psr_mech_free.restype = None
        L.psr_options_default.argtypes = [ctypes.POINTER(COptions)]
        L.psr_options_default.restype = None
        L.psr_last_error.restype = ctypes.c_char_p
        solve_args = [vp, i64] + [dp] * 7 + [dp] * 2 + [dp] * 5 + [ctypes.POINTER(COptions), vp]
        L.psr_batch_solve.argtypes = solve_args
        L.psr_batch_solve_host.argtypes = solve_args
        L.psr_batch_solve_noalloc.argtypes = solve_args
        L.psr_eval_residual.argtypes = [vp, i64] + [dp] * 7 + [dp, i32, vp]
        L.psr_eval_jacobian.argtypes = [vp, i64] + [dp] * 7 + [dp, i32, i32, vp]
        L.psr_batch_lu_solve.argtypes = [i64, i32, dp, dp, dp, dp, i32, vp]
        L.psr_batch_adjoint.argtypes = [vp, i64] + [dp] * 7 + [dp, dp, dp, dp, i32, vp]
        L.psr_batch_solve_soot.argtypes = [vp, i64] + [dp] * 9 + [dp] * 3 + [dp] * 5 + [ctypes.POINTER(COptions), vp]
        L.psr_eval_residual_soot.argtypes = [vp, i64] + [dp] * 9 + [dp, i32, vp]
        L.psr_eval_jacobian_soot.argtypes = [vp, i64] + [dp] * 9 + [dp, i32, i32, vp]
        L.psr_eval_jacobian_fd.argtypes = [vp, i64] + [dp] * 7 + [dp, i32, vp]
        L.psr_eval_rates.argtypes = [vp, i64] + [dp] * 8 + [vp]
        L.psr_autotune.argtypes = [vp, i64] + [dp] * 6 + [ctypes.POINTER(COptions), vp]
        L.psr_batch_solve_multi.argtypes = [ctypes.POINTER(vp), i32, i64, dp, dp] + [dp] * 8 + [dp] * 5 + \
            [ctypes.POINTER(COptions), vp]
        L.psr_pipe_probe.argtypes = [i32, i64, i32, i32, dp, vp]
        L.psr_batch_lu_solve_tc.argtypes = [i64, i32, dp, dp, dp, dp, i32, vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != PSR_OK:
        raise PsrError(rc, lib().psr_last_error().decode())


@dataclasses.dataclass
class Options:
    """Solver controls, field for field as psr_options (defaults from the library)."""
    ftol: float = 1e-8
    step_rtol: float = 1e-10
    step_atol_y: float = 1e-14
    step_atol_t: float = 1e-10
    ts_rtol: float = 1e-4
    ts_atol_y: float = 1e-10
    dt0_over_tau: float = 1e-6
    dt_shrink: float = 0.25
    y_floor: float = 1e-10
    t_min: float = 200.0
    t_max: float = 5000.0
    max_newton: int = 500
    max_damp: int = 8
    max_ts_rounds: int = 100
    ts_steps: int = 12
    ts_newton: int = 8
    precision: int = PSR_FP64
    energy: int = PSR_ADIABATIC
    warps_per_block: int = 0
    blocks_per_sm: int = 0
    mixed_fallback: int = 2
    jacobian: int = 0
    mixed_max_newton: int = -1
    jac_age: int = 1
    ts_linear: int = 150
    path: int = 0
    handoff: int = -1
    lu_tensor: int = 0
    block_threads: int = 0
    persistent: int = 0
    spin_limit: int = 0

    def to_c(self):
        o = COptions()
        lib().psr_options_default(ctypes.byref(o))
        for f in dataclasses.fields(self):
            setattr(o, f.name, getattr(self, f.name))
        return o


class Mechanism:
    """A mechanism loaded into libpsr (tables on the current CUDA device)."""

    def __init__(self, text: str):
        h = ctypes.c_void_p()
        raw = text.encode()
        _check(lib().psr_mech_load_mem(raw, len(raw), ctypes.byref(h)))
        self._h = h
        info = CMechInfo()
        _check(lib().psr_mech_info_get(h, ctypes.byref(info)))
        self.K, self.I = info.K, info.I
        self.n_third_body, self.n_falloff, self.has_soot = info.n_third_body, info.n_falloff, bool(info.has_soot)
        W = np.zeros(self.K)
        _check(lib().psr_mech_weights(h, W.ctypes.data))
        self.W = W

    @classmethod
    def from_file(cls, path):
        with open(path) as fh:
            return cls(fh.read())

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().psr_mech_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t, dtype, shape=None, name="array"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def batch_solve(mech: Mechanism, Y_in, T_in, tau, P, Y0, T0, rate_mult=None, opts: Options = None,
                out=None):
    """psr_batch_solve on torch CUDA tensors. Returns dict Y, T, iters, ts_steps, status, fnorm, nfev."""
    import torch
    f64, i32 = torch.float64, torch.int32
    B, K = Y_in.shape
    dev = Y_in.device
    if out is None:
        out = dict(Y=torch.empty((B, K), dtype=f64, device=dev), T=torch.empty(B, dtype=f64, device=dev),
                   iters=torch.empty(B, dtype=i32, device=dev), ts_steps=torch.empty(B, dtype=i32, device=dev),
                   status=torch.empty(B, dtype=i32, device=dev), fnorm=torch.empty(B, dtype=f64, device=dev),
                   nfev=torch.empty(B, dtype=i32, device=dev))
    o = (opts or Options()).to_c()
    _check(lib().psr_batch_solve(
        mech.handle, B, _ptr(Y_in, f64, (B, K), "Y_in"), _ptr(T_in, f64, (B,), "T_in"),
        _ptr(tau, f64, (B,), "tau"), _ptr(P, f64, (B,), "P"), _ptr(Y0, f64, (B, K), "Y0"),
        _ptr(T0, f64, (B,), "T0"), _ptr(rate_mult, f64, (mech.I,), "rate_mult"),
        _ptr(out["Y"], f64, (B, K)), _ptr(out["T"], f64, (B,)), _ptr(out["iters"], i32, (B,)),
        _ptr(out["ts_steps"], i32, (B,)), _ptr(out["status"], i32, (B,)), _ptr(out["fnorm"], f64, (B,)),
        _ptr(out["nfev"], i32, (B,)), ctypes.byref(o), _stream()))
    return out


def batch_solve_noalloc(mech: Mechanism, Y_in, T_in, tau, P, Y0, T0, rate_mult=None, opts: Options = None,
                        out=None):
    """psr_batch_solve_noalloc: as batch_solve, but the library allocates no device memory
    (its work-queue counter is a static device array). Output tensors must be passed in
    `out` by callers that cannot allocate; otherwise they are created here."""
    import torch
    f64, i32 = torch.float64, torch.int32
    B, K = Y_in.shape
    dev = Y_in.device
    if out is None:
        out = dict(Y=torch.empty((B, K), dtype=f64, device=dev), T=torch.empty(B, dtype=f64, device=dev),
                   iters=torch.empty(B, dtype=i32, device=dev), ts_steps=torch.empty(B, dtype=i32, device=dev),
                   status=torch.empty(B, dtype=i32, device=dev), fnorm=torch.empty(B, dtype=f64, device=dev),
                   nfev=torch.empty(B, dtype=i32, device=dev))
    o = (opts or Options()).to_c()
    _check(lib().psr_batch_solve_noalloc(
        mech.handle, B, _ptr(Y_in, f64, (B, K), "Y_in"), _ptr(T_in, f64, (B,), "T_in"),
        _ptr(tau, f64, (B,), "tau"), _ptr(P, f64, (B,), "P"), _ptr(Y0, f64, (B, K), "Y0"),
        _ptr(T0, f64, (B,), "T0"), _ptr(rate_mult, f64, (mech.I,), "rate_mult"),
        _ptr(out["Y"], f64, (B, K)), _ptr(out["T"], f64, (B,)), _ptr(out["iters"], i32, (B,)),
        _ptr(out["ts_steps"], i32, (B,)), _ptr(out["status"], i32, (B,)), _ptr(out["fnorm"], f64, (B,)),
        _ptr(out["nfev"], i32, (B,)), ctypes.byref(o), _stream()))
    return out


def batch_solve_host(mech: Mechanism, Y_in, T_in, tau, P, Y0, T0, rate_mult=None, opts: Options = None,
                     out=None, stream=None):
    """psr_batch_solve_host on host arrays (numpy float64, or CPU torch tensors, pinned
    for the fast path): the library copies inputs in, solves, copies results back and
    synchronises. Returns dict Y, T, iters, ts_steps, status, fnorm, nfev (host)."""
    def addr(x, dtype):
        if hasattr(x, "data_ptr"):
            import torch
            want = torch.float64 if dtype == np.float64 else torch.int32
            if x.is_cuda or x.dtype != want or not x.is_contiguous():
                raise TypeError("host arrays must be contiguous CPU tensors of the right dtype")
            return x.data_ptr()
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be contiguous numpy arrays of the right dtype")
        return x.ctypes.data
    B, K = Y_in.shape
    if out is None:
        out = dict(Y=np.empty((B, K)), T=np.empty(B), iters=np.empty(B, np.int32),
                   ts_steps=np.empty(B, np.int32), status=np.empty(B, np.int32), fnorm=np.empty(B),
                   nfev=np.empty(B, np.int32))
    ins = [v if hasattr(v, "data_ptr") else np.ascontiguousarray(v, dtype=np.float64)
           for v in (Y_in, T_in, tau, P, Y0, T0)]
    mult = None if rate_mult is None else np.ascontiguousarray(rate_mult, dtype=np.float64)
    o = (opts or Options()).to_c()
    _check(lib().psr_batch_solve_host(
        mech.handle, B, *[addr(v, np.float64) for v in ins], None if mult is None else mult.ctypes.data,
        addr(out["Y"], np.float64), addr(out["T"], np.float64), addr(out["iters"], np.int32),
        addr(out["ts_steps"], np.int32), addr(out["status"], np.int32), addr(out["fnorm"], np.float64),
        addr(out["nfev"], np.int32), ctypes.byref(o), stream if stream is not None else _stream()))
    return out


def eval_residual(mech: Mechanism, Y_in, T_in, tau, P, Y, T, rate_mult=None, energy=PSR_ADIABATIC):
    import torch
    f64 = torch.float64
    B, K = Y.shape
    F = torch.empty((B, K + 1), dtype=f64, device=Y.device)
    _check(lib().psr_eval_residual(
        mech.handle, B, _ptr(Y_in, f64, (B, K)), _ptr(T_in, f64, (B,)), _ptr(tau, f64, (B,)),
        _ptr(P, f64, (B,)), _ptr(Y, f64, (B, K)), _ptr(T, f64, (B,)), _ptr(rate_mult, f64, (mech.I,)),
        F.data_ptr(), energy, _stream()))
    return F


def eval_jacobian(mech: Mechanism, Y_in, T_in, tau, P, Y, T, rate_mult=None, energy=PSR_ADIABATIC,
                  precision=PSR_FP64):
    import torch
    f64 = torch.float64
    B, K = Y.shape
    J = torch.empty((B, K + 1, K + 1), dtype=f64, device=Y.device)
    _check(lib().psr_eval_jacobian(
        mech.handle, B, _ptr(Y_in, f64, (B, K)), _ptr(T_in, f64, (B,)), _ptr(tau, f64, (B,)),
        _ptr(P, f64, (B,)), _ptr(Y, f64, (B, K)), _ptr(T, f64, (B,)), _ptr(rate_mult, f64, (mech.I,)),
        J.data_ptr(), energy, precision, _stream()))
    return J


def eval_jacobian_fd(mech: Mechanism, Y_in, T_in, tau, P, Y, T, rate_mult=None, energy=PSR_ADIABATIC):
    """psr_eval_jacobian_fd: the central-difference Jacobian [B][K+1][K+1] (FP64)."""
    import torch
    f64 = torch.float64
    B, K = Y.shape
    J = torch.empty((B, K + 1, K + 1), dtype=f64, device=Y.device)
    _check(lib().psr_eval_jacobian_fd(
        mech.handle, B, _ptr(Y_in, f64, (B, K)), _ptr(T_in, f64, (B,)), _ptr(tau, f64, (B,)),
        _ptr(P, f64, (B,)), _ptr(Y, f64, (B, K)), _ptr(T, f64, (B,)), _ptr(rate_mult, f64, (mech.I,)),
        J.data_ptr(), energy, _stream()))
    return J


def batch_lu_solve(A, r, precision=PSR_FP64):
    """Solve A_b x_b = r_b for a batch of n x n systems (n <= 512) by the solver's LU."""
    import torch
    B, n, _ = A.shape
    x = torch.empty((B, n), dtype=torch.float64, device=A.device)
    ok = torch.empty(B, dtype=torch.int32, device=A.device)
    _check(lib().psr_batch_lu_solve(B, n, _ptr(A, torch.float64, (B, n, n), "A"), _ptr(r, torch.float64, (B, n), "r"),
                                    x.data_ptr(), ok.data_ptr(), precision, _stream()))
    return x, ok


def batch_lu_solve_tc(A, r, lu_tensor=PSR_LU_TF32):
    """psr_batch_lu_solve_tc: the FP32 LU with the trailing update on the tensor cores
    (TF32 or 3xTF32) for n >= 96 (smaller n: CUDA cores)."""
    import torch
    B, n, _ = A.shape
    x = torch.empty((B, n), dtype=torch.float64, device=A.device)
    ok = torch.empty(B, dtype=torch.int32, device=A.device)
    _check(lib().psr_batch_lu_solve_tc(B, n, _ptr(A, torch.float64, (B, n, n), "A"),
                                       _ptr(r, torch.float64, (B, n), "r"), x.data_ptr(), ok.data_ptr(), lu_tensor,
                                       _stream()))
    return x, ok


def batch_adjoint(mech: Mechanism, Y_in, T_in, tau, P, Y, T, g, rate_mult=None, energy=PSR_ADIABATIC):
    """psr_batch_adjoint: dL/d ln(rate multiplier) [B, I] for dL/d(Y, T) = g [B, K+1] at
    converged states. Returns (grad, lambda, ok)."""
    import torch
    f64 = torch.float64
    B, K = Y.shape
    grad = torch.empty((B, mech.I), dtype=f64, device=Y.device)
    lam = torch.empty((B, K + 1), dtype=f64, device=Y.device)
    ok = torch.empty(B, dtype=torch.int32, device=Y.device)
    _check(lib().psr_batch_adjoint(
        mech.handle, B, _ptr(Y_in, f64, (B, K)), _ptr(T_in, f64, (B,)), _ptr(tau, f64, (B,)),
        _ptr(P, f64, (B,)), _ptr(Y, f64, (B, K)), _ptr(T, f64, (B,)), _ptr(rate_mult, f64, (mech.I,)),
        _ptr(g, f64, (B, K + 1), "g"), grad.data_ptr(), lam.data_ptr(), ok.data_ptr(), energy, _stream()))
    return grad, lam, ok


def batch_solve_soot(mech: Mechanism, Y_in, T_in, tau, P, M_in, Y0, T0, M0=None, rate_mult=None,
                     opts: Options = None, out=None):
    """psr_batch_solve_soot on torch CUDA tensors (gas + six MOMIC moments). Returns the
    batch_solve dict plus M [B, 6]."""
    import torch
    f64, i32 = torch.float64, torch.int32
    B, K = Y_in.shape
    dev = Y_in.device
    if out is None:
        out = dict(Y=torch.empty((B, K), dtype=f64, device=dev), T=torch.empty(B, dtype=f64, device=dev),
                   M=torch.empty((B, 6), dtype=f64, device=dev),
                   iters=torch.empty(B, dtype=i32, device=dev), ts_steps=torch.empty(B, dtype=i32, device=dev),
                   status=torch.empty(B, dtype=i32, device=dev), fnorm=torch.empty(B, dtype=f64, device=dev),
                   nfev=torch.empty(B, dtype=i32, device=dev))
    o = (opts or Options()).to_c()
    _check(lib().psr_batch_solve_soot(
        mech.handle, B, _ptr(Y_in, f64, (B, K), "Y_in"), _ptr(T_in, f64, (B,), "T_in"),
        _ptr(tau, f64, (B,), "tau"), _ptr(P, f64, (B,), "P"), _ptr(M_in, f64, (B, 6), "M_in"),
        _ptr(Y0, f64, (B, K), "Y0"), _ptr(T0, f64, (B,), "T0"), _ptr(M0, f64, (B, 6), "M0"),
        _ptr(rate_mult, f64, (mech.I,), "rate_mult"),
        _ptr(out["Y"], f64, (B, K)), _ptr(out["T"], f64, (B,)), _ptr(out["M"], f64, (B, 6)),
        _ptr(out["iters"], i32, (B,)), _ptr(out["ts_steps"], i32, (B,)), _ptr(out["status"], i32, (B,)),
        _ptr(out["fnorm"], f64, (B,)), _ptr(out["nfev"], i32, (B,)), ctypes.byref(o), _stream()))
    return out


def eval_residual_soot(mech: Mechanism, Y_in, T_in, tau, P, M_in, Y, T, M, rate_mult=None, energy=PSR_ADIABATIC):
    import torch
    f64 = torch.float64
    B, K = Y.shape
    F = torch.empty((B, K + 7), dtype=f64, device=Y.device)
    _check(lib().psr_eval_residual_soot(
        mech.handle, B, _ptr(Y_in, f64, (B, K)), _ptr(T_in, f64, (B,)), _ptr(tau, f64, (B,)), _ptr(P, f64, (B,)),
        _ptr(M_in, f64, (B, 6)), _ptr(Y, f64, (B, K)), _ptr(T, f64, (B,)), _ptr(M, f64, (B, 6)),
        _ptr(rate_mult, f64, (mech.I,)), F.data_ptr(), energy, _stream()))
    return F


def eval_jacobian_soot(mech: Mechanism, Y_in, T_in, tau, P, M_in, Y, T, M, rate_mult=None, energy=PSR_ADIABATIC,
                       precision=PSR_FP64):
    import torch
    f64 = torch.float64
    B, K = Y.shape
    J = torch.empty((B, K + 7, K + 7), dtype=f64, device=Y.device)
    _check(lib().psr_eval_jacobian_soot(
        mech.handle, B, _ptr(Y_in, f64, (B, K)), _ptr(T_in, f64, (B,)), _ptr(tau, f64, (B,)), _ptr(P, f64, (B,)),
        _ptr(M_in, f64, (B, 6)), _ptr(Y, f64, (B, K)), _ptr(T, f64, (B,)), _ptr(M, f64, (B, 6)),
        _ptr(rate_mult, f64, (mech.I,)), J.data_ptr(), energy, precision, _stream()))
    return J


def batch_solve_multi(mechs, mech_id, row_off, Y_in, T_in, tau, P, Y0, T0, opts: Options = None, out=None):
    """psr_batch_solve_multi: B reactors of several mechanisms in one call. mech_id (int32
    [B]) picks mechs[mech_id[r]]; row_off (int64 [B]) locates reactor r's row in the packed
    float64 arrays Y_in, Y0 (and the returned Y). Returns dict Y (packed), T, iters,
    ts_steps, status, fnorm, nfev."""
    import torch
    f64, i32, i64 = torch.float64, torch.int32, torch.int64
    B = mech_id.shape[0]
    L = Y_in.shape[0]
    dev = Y_in.device
    if out is None:
        out = dict(Y=torch.empty(L, dtype=f64, device=dev), T=torch.empty(B, dtype=f64, device=dev),
                   iters=torch.empty(B, dtype=i32, device=dev), ts_steps=torch.empty(B, dtype=i32, device=dev),
                   status=torch.empty(B, dtype=i32, device=dev), fnorm=torch.empty(B, dtype=f64, device=dev),
                   nfev=torch.empty(B, dtype=i32, device=dev))
    handles = (ctypes.c_void_p * len(mechs))(*[m.handle for m in mechs])
    o = (opts or Options()).to_c()
    _check(lib().psr_batch_solve_multi(
        handles, len(mechs), B, _ptr(mech_id, i32, (B,), "mech_id"), _ptr(row_off, i64, (B,), "row_off"),
        _ptr(Y_in, f64, (L,), "Y_in"), _ptr(T_in, f64, (B,), "T_in"), _ptr(tau, f64, (B,), "tau"),
        _ptr(P, f64, (B,), "P"), _ptr(Y0, f64, (L,), "Y0"), _ptr(T0, f64, (B,), "T0"),
        _ptr(out["Y"], f64, (L,)), _ptr(out["T"], f64, (B,)), _ptr(out["iters"], i32, (B,)),
        _ptr(out["ts_steps"], i32, (B,)), _ptr(out["status"], i32, (B,)), _ptr(out["fnorm"], f64, (B,)),
        _ptr(out["nfev"], i32, (B,)), ctypes.byref(o), _stream()))
    return out


def autotune(mech: Mechanism, Y_in, T_in, tau, P, Y0, T0, opts: Options = None) -> Options:
    """psr_autotune on a sample batch (torch CUDA tensors): returns a copy of `opts` with
    the fastest launch shape (warps_per_block, blocks_per_sm) for this mechanism."""
    import torch
    f64 = torch.float64
    B, K = Y_in.shape
    base = opts or Options()
    o = base.to_c()
    _check(lib().psr_autotune(
        mech.handle, B, _ptr(Y_in, f64, (B, K), "Y_in"), _ptr(T_in, f64, (B,), "T_in"), _ptr(tau, f64, (B,), "tau"),
        _ptr(P, f64, (B,), "P"), _ptr(Y0, f64, (B, K), "Y0"), _ptr(T0, f64, (B,), "T0"), ctypes.byref(o),
        _stream()))
    return dataclasses.replace(base, warps_per_block=o.warps_per_block, blocks_per_sm=o.blocks_per_sm, path=o.path,
                               block_threads=o.block_threads)


def eval_rates(mech: Mechanism, Y, T, P, rate_mult=None, out=None):
    """psr_eval_rates on torch CUDA tensors: dict kf, kr, q [B][I] (mechanism-file order)
    and wdot [B][K]."""
    import torch
    f64 = torch.float64
    B, K = Y.shape
    dev = Y.device
    if out is None:
        out = dict(kf=torch.empty((B, mech.I), dtype=f64, device=dev), kr=torch.empty((B, mech.I), dtype=f64, device=dev),
                   q=torch.empty((B, mech.I), dtype=f64, device=dev), wdot=torch.empty((B, K), dtype=f64, device=dev))
    _check(lib().psr_eval_rates(
        mech.handle, B, _ptr(Y, f64, (B, K), "Y"), _ptr(T, f64, (B,), "T"), _ptr(P, f64, (B,), "P"),
        _ptr(rate_mult, f64, (mech.I,), "rate_mult"), _ptr(out.get("kf"), f64, (B, mech.I)),
        _ptr(out.get("kr"), f64, (B, mech.I)), _ptr(out.get("q"), f64, (B, mech.I)),
        _ptr(out.get("wdot"), f64, (B, K)), _stream()))
    return out


PROBE_FMA64, PROBE_FMA32, PROBE_EXP64, PROBE_LOG64, PROBE_DIV64 = 0, 1, 2, 3, 4
PROBE_SATOM32, PROBE_SATOM32_SAME, PROBE_SATOM64, PROBE_SATOM64_SAME = 5, 6, 7, 8
# operations per thread and iteration of each probe (psr_probe.h): flops for the FMA
# probes, calls for exp / log / division, atomics for the shared-memory atomic probes
PROBE_OPS = {PROBE_FMA64: 16, PROBE_FMA32: 32, PROBE_EXP64: 8, PROBE_LOG64: 8, PROBE_DIV64: 8,
             PROBE_SATOM32: 8, PROBE_SATOM32_SAME: 8, PROBE_SATOM64: 8, PROBE_SATOM64_SAME: 8}


def pipe_probe(kind, iters, blocks, threads, sink):
    """psr_pipe_probe: one probe launch on the current stream; `sink` is a float64 CUDA
    tensor of at least blocks x threads elements. Returns the operation count."""
    import torch
    if sink.numel() < blocks * threads:
        raise ValueError("sink too small")
    _check(lib().psr_pipe_probe(kind, iters, blocks, threads, _ptr(sink, torch.float64, None, "sink"), _stream()))
    return PROBE_OPS[kind] * blocks * threads * iters

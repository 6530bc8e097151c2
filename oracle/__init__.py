"""CPU oracle for AMP-PCG / DS-PCG -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and the
two share no code: the oracle is plain C (``ampcg_oracle.c``) plus this ctypes
wrapper, compiled with ``gcc -ffp-contract=off`` so that every rounding is the
one written in the source.

Functions follow the paper (Guo, de Sturler, Warburton, arXiv 2505.04155):
``pcg64`` is Algorithm 1 in native FP64; ``ampcg`` is Algorithm 3 (and
Algorithm 2 under the FIXED criterion) with software-rounded FP32/FP16 storage;
``select``/``eta_window``/``eta_linear`` are Eq. (precision_selector),
Eq. (eta_k) and Eq. (linear criterion).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ampcg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

FP64, FP32, FP16 = 0, 1, 2
WINDOW, LINEAR, FIXED = 0, 1, 2
SCALE_NONE, SCALE_L2, SCALE_LINF_POW2, SCALE_LINF_POW2_LAG = 0, 1, 2, 3
M_NONE, M_JACOBI, M_CHEBYSHEV = 0, 1, 2
OK, NOT_CONVERGED, ERR_INVALID, ERR_BREAKDOWN, ERR_NONFINITE = 0, 1, -1, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, C11)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Policy(C.Structure):
    _fields_ = [("u0", C.c_int), ("criterion", C.c_int), ("d", C.c_int), ("ell", C.c_int),
                ("C", C.c_double), ("tau_zs", C.c_double), ("tau_zh", C.c_double),
                ("scale", C.c_int), ("latch", C.c_int), ("verify_refresh", C.c_int),
                ("fixed_uz", C.c_int), ("fixed_ur", C.c_int)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("converged", C.c_int),
                ("refreshes", C.c_int), ("true_relres", C.c_double),
                ("updated_relres", C.c_double), ("switch_iter", C.c_int * 3),
                ("scale_retries", C.c_int), ("y16_small", C.c_int64), ("y16_total", C.c_int64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp, ip, i64 = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_int64
        u8p = C.POINTER(C.c_uint8)
        lib.oracle_round16.restype = C.c_double
        lib.oracle_round16.argtypes = [C.c_double]
        lib.oracle_round32.restype = C.c_double
        lib.oracle_round32.argtypes = [C.c_double]
        lib.oracle_round_array.argtypes = [C.c_int, dp, dp, i64]
        lib.oracle_spmv.argtypes = [i64, ip, ip, dp, C.c_int, dp, dp]
        lib.oracle_residual64.argtypes = [i64, ip, ip, dp, dp, dp, dp]
        lib.oracle_dot.restype = C.c_double
        lib.oracle_dot.argtypes = [i64, dp, dp]
        lib.oracle_scale.restype = C.c_double
        lib.oracle_scale.argtypes = [C.c_int, C.c_double, C.c_double]
        for nm in ("oracle_eta_window", "oracle_eta_linear"):
            getattr(lib, nm).restype = C.c_double
            getattr(lib, nm).argtypes = [dp, C.c_int, C.c_int, C.c_double]
        lib.oracle_eta_hat.restype = C.c_double
        lib.oracle_eta_hat.argtypes = [dp, C.c_int, C.c_int, C.c_double]
        lib.oracle_select.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.oracle_pcg64.restype = C.c_int
        lib.oracle_pcg64.argtypes = [i64, ip, ip, dp, C.c_int, dp, dp, C.c_double, C.c_int,
                                     dp, C.POINTER(_Result)]
        lib.oracle_ampcg.restype = C.c_int
        lib.oracle_ampcg.argtypes = [i64, ip, ip, dp, C.c_int, C.c_int, C.c_double, C.c_double,
                                     dp, dp, C.c_double, C.c_int, C.POINTER(_Policy), dp, u8p,
                                     C.POINTER(_Result)]
        lib.oracle_selector_trace.argtypes = [dp, C.c_int, C.c_double, C.c_double,
                                              C.POINTER(_Policy), u8p]
        lib.oracle_scale_precond.restype = C.c_int
        lib.oracle_scale_precond.argtypes = [i64, ip, ip, dp, C.c_int, C.c_int, C.c_int, C.c_double,
                                             dp, dp]
        lib.oracle_grad_log_coeff.argtypes = [i64, ip, ip, dp, dp, dp, dp]
        lib.oracle_direction.argtypes = [i64, C.c_int, C.c_int, C.c_double, dp, dp]
        lib.oracle_update_xr.argtypes = [i64, C.c_int, C.c_double, dp, dp, dp, dp]
        lib.oracle_scale_cheb.restype = C.c_int
        lib.oracle_scale_cheb.argtypes = [i64, ip, ip, dp, C.c_int, C.c_double, C.c_double, C.c_int,
                                          C.c_int, C.c_double, dp, dp]
        lib.oracle_cheb_apply_public.restype = C.c_int
        lib.oracle_cheb_apply_public.argtypes = [i64, i64, ip, ip, dp, dp, C.c_int, C.c_double,
                                                 C.c_double, C.c_int, dp, dp]
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Policy:
    """Precision policy; defaults are the paper's constants (d=10, C=1, ell=5,
    tau_zs=1e-4, tau_zh=1e-6) with the AMP-PCG(FP16) variant."""
    u0: int = FP16
    criterion: int = LINEAR
    d: int = 10
    ell: int = 5
    C: float = 1.0
    tau_zs: float = 1e-4
    tau_zh: float = 1e-6
    scale: int = SCALE_LINF_POW2
    latch: int = 1
    verify_refresh: int = 0
    fixed_uz: int = FP64
    fixed_ur: int = FP64

    def _c(self) -> _Policy:
        return _Policy(self.u0, self.criterion, self.d, self.ell, self.C, self.tau_zs,
                       self.tau_zh, self.scale, self.latch, self.verify_refresh,
                       self.fixed_uz, self.fixed_ur)


@dataclass
class Result:
    status: int
    iters: int
    converged: bool
    refreshes: int
    true_relres: float
    updated_relres: float
    switch_iter: tuple
    x: np.ndarray
    relres_hist: np.ndarray = field(repr=False)
    prec_hist: np.ndarray = field(repr=False)
    scale_retries: int = 0
    y16_small: int = 0      # binary16 y_i below the normal range while r_i != 0 (summed over iterations)
    y16_total: int = 0      # binary16 y_i with r_i != 0


def round16(v):
    """IEEE binary16 round-to-nearest-even of float64 values (from the definition)."""
    a = _f64(np.atleast_1d(v))
    out = np.empty_like(a)
    _load().oracle_round_array(FP16, _d(a), _d(out), a.size)
    return out if np.ndim(v) else float(out[0])


def round32(v):
    """IEEE binary32 round-to-nearest-even of float64 values (from the definition)."""
    a = _f64(np.atleast_1d(v))
    out = np.empty_like(a)
    _load().oracle_round_array(FP32, _d(a), _d(out), a.size)
    return out if np.ndim(v) else float(out[0])


def round_to(prec, v):
    return {FP64: lambda x: _f64(x).copy(), FP32: round32, FP16: round16}[prec](v)


def spmv(rowptr, col, aval, prec, p):
    """q = A p in precision `prec`; `aval` must already be rounded to `prec`."""
    rowptr, col, aval, p = _i32(rowptr), _i32(col), _f64(aval), _f64(p)
    n = rowptr.size - 1
    q = np.empty(n)
    _load().oracle_spmv(n, _i(rowptr), _i(col), _d(aval), prec, _d(p), _d(q))
    return q


def residual64(rowptr, col, val, b, x):
    rowptr, col, val, b, x = _i32(rowptr), _i32(col), _f64(val), _f64(b), _f64(x)
    n = rowptr.size - 1
    r = np.empty(n)
    _load().oracle_residual64(n, _i(rowptr), _i(col), _d(val), _d(b), _d(x), _d(r))
    return r


def dot(a, b):
    a, b = _f64(a), _f64(b)
    return _load().oracle_dot(a.size, _d(a), _d(b))


def scale_precond(rowptr, col, val, mtype, uz, ur, omega, r):
    """Alg. 3 scaling and preconditioning: z = M^-1 round_uz(fl_ur(omega r)), M none or Jacobi."""
    rowptr, col, val, r = _i32(rowptr), _i32(col), _f64(val), _f64(r)
    n = rowptr.size - 1
    z = np.empty(n)
    st = _load().oracle_scale_precond(n, _i(rowptr), _i(col), _d(val), mtype, uz, ur, omega, _d(r), _d(z))
    assert st == 0
    return z


def scale_cheb(rowptr, col, val, degree, lmin, lmax, uz, ur, omega, r):
    """Alg. 3 scaling and preconditioning with the Chebyshev preconditioner (reading R8)."""
    rowptr, col, val, r = _i32(rowptr), _i32(col), _f64(val), _f64(r)
    n = rowptr.size - 1
    z = np.empty(n)
    st = _load().oracle_scale_cheb(n, _i(rowptr), _i(col), _d(val), degree, lmin, lmax, uz, ur,
                                   omega, _d(r), _d(z))
    assert st == 0
    return z


def direction(uz, first, beta, z, p_prev):
    """Alg. 3 search direction p = z + beta p_prev in u_z (p_prev rounded to u_z first)."""
    z = _f64(z)
    p = _f64(p_prev).copy()
    _load().oracle_direction(z.size, uz, int(first), beta, _d(z), _d(p))
    return p


def update_xr(ur, alpha, p, q, x, r):
    """Alg. 3 updates: returns (x + alpha p in FP64, r - alpha q in u_r)."""
    p, q = _f64(p), _f64(q)
    x, r = _f64(x).copy(), _f64(r).copy()
    _load().oracle_update_xr(p.size, ur, alpha, _d(p), _d(q), _d(x), _d(r))
    return x, r


def grad_log_coeff(rowptr, col, val, x, lam):
    """dL/dtheta for the log-coefficient field from x and the adjoint lambda."""
    rowptr, col, val, x, lam = _i32(rowptr), _i32(col), _f64(val), _f64(x), _f64(lam)
    n = rowptr.size - 1
    out = np.empty(n)
    _load().oracle_grad_log_coeff(n, _i(rowptr), _i(col), _d(val), _d(x), _d(lam), _d(out))
    return out


def scale(mode, delta, maxabs):
    return _load().oracle_scale(mode, delta, maxabs)


def eta_window(delta, k, d=10, C=1.0):
    delta = _f64(delta)
    return _load().oracle_eta_window(_d(delta), k, d, C)


def eta_linear(delta, k, ell=5, C=1.0):
    delta = _f64(delta)
    return _load().oracle_eta_linear(_d(delta), k, ell, C)


def eta_hat(delta, k, m, C=1.0):
    delta = _f64(delta)
    return _load().oracle_eta_hat(_d(delta), k, m, C)


def select(nu, u0, tau_zs, tau_zh, eta, tol_nb):
    uz, ur = C.c_int(), C.c_int()
    _load().oracle_select(nu, u0, tau_zs, tau_zh, eta, tol_nb, C.byref(uz), C.byref(ur))
    return uz.value, ur.value


def selector_trace(delta, nb, tol, policy: Policy):
    delta = _f64(delta)
    out = np.zeros(delta.size, dtype=np.uint8)
    pol = policy._c()
    _load().oracle_selector_trace(_d(delta), delta.size - 1, nb, tol, C.byref(pol),
                                  out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def cheb_apply(rowptr, col, ahat64, dsqrt_inv64, degree, lmin, lmax, prec, y):
    rowptr, col, ahat64, dsi, y = _i32(rowptr), _i32(col), _f64(ahat64), _f64(dsqrt_inv64), _f64(y)
    n = rowptr.size - 1
    z = np.empty(n)
    st = _load().oracle_cheb_apply_public(n, col.size, _i(rowptr), _i(col), _d(ahat64), _d(dsi),
                                          degree, lmin, lmax, prec, _d(y), _d(z))
    assert st == 0
    return z


def _result(res, x, rh, ph):
    it = res.iters
    return Result(res.status, it, bool(res.converged), res.refreshes, res.true_relres,
                  res.updated_relres, tuple(res.switch_iter), x, rh[: it + 1].copy(),
                  ph[:it].copy(), res.scale_retries, res.y16_small, res.y16_total)


def pcg64(rowptr, col, val, b, x0=None, tol=1e-10, maxit=2000, jacobi=True) -> Result:
    """Algorithm 1 (PCG) in native FP64 with Jacobi (or identity) M."""
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.size - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    rh = np.zeros(maxit + 1)
    res = _Result()
    _load().oracle_pcg64(n, _i(rowptr), _i(col), _d(val), M_JACOBI if jacobi else M_NONE,
                         _d(b), _d(x), tol, maxit, _d(rh), C.byref(res))
    return _result(res, x, rh, np.zeros(max(maxit, 1), dtype=np.uint8))


def ampcg(rowptr, col, val, b, x0=None, tol=1e-10, maxit=2000, policy: Policy | None = None,
          precond=M_JACOBI, cheb_degree=0, cheb_lmin=0.0, cheb_lmax=0.0) -> Result:
    """Algorithm 3 (AMP-PCG) with software-rounded storage precisions."""
    policy = policy or Policy()
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.size - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    rh = np.zeros(maxit + 2)
    ph = np.zeros(max(maxit, 1), dtype=np.uint8)
    res = _Result()
    pol = policy._c()
    _load().oracle_ampcg(n, _i(rowptr), _i(col), _d(val), precond, cheb_degree, cheb_lmin,
                         cheb_lmax, _d(b), _d(x), tol, maxit, C.byref(pol), _d(rh),
                         ph.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(res))
    return _result(res, x, rh, ph)

"""Python binding of libampcg (include/ampcg.h): adaptive mixed-precision,
dynamically scaled PCG (Guo, de Sturler, Warburton, arXiv 2505.04155) on B300.

Argument marshalling only: every step of the solver runs in the CUDA library.
There is no CPU fallback; if the library has not been built (``build.py``) or
no CUDA device is visible, the calls raise.

Arrays may be NumPy arrays (host) or CUDA torch tensors (device); the library
asks the CUDA runtime which kind each pointer is.  Contexts created while
torch has CUDA available are bound to torch's current stream, so library work
is ordered with torch work on that stream.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libampcg.so")

FP64, FP32, FP16 = 0, 1, 2
CRIT_WINDOW, CRIT_LINEAR, CRIT_FIXED = 0, 1, 2
SCALE_NONE, SCALE_L2, SCALE_LINF_POW2, SCALE_LINF_POW2_LAG = 0, 1, 2, 3
M_NONE, M_JACOBI, M_CHEBYSHEV = 0, 1, 2

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NONFINITE = -1, -2, -3, -4
ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NO_DEVICE, ERR_UNSUPPORTED = -5, -6, -7, -8, -9


class AmpcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class PrecondSpec(C.Structure):
    _fields_ = [("type", C.c_int), ("degree", C.c_int), ("lmin", C.c_double), ("lmax", C.c_double)]


class LayoutC(C.Structure):
    _fields_ = [("n", C.c_int64), ("nslices", C.c_int64), ("stored", C.c_int64),
                ("stored_uniform", C.c_int64), ("maxw", C.c_int32), ("idx16", C.c_int32),
                ("stream_hint", C.c_int32), ("block3", C.c_int32)]


class PolicyC(C.Structure):
    _fields_ = [("u0", C.c_int), ("criterion", C.c_int), ("d", C.c_int), ("ell", C.c_int),
                ("C", C.c_double), ("tau_zs", C.c_double), ("tau_zh", C.c_double),
                ("scale", C.c_int), ("latch", C.c_int), ("verify_refresh", C.c_int),
                ("fixed_uz", C.c_int), ("fixed_ur", C.c_int), ("graph_chunk", C.c_int)]


class ResultC(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("refreshes", C.c_int),
                ("status", C.c_int), ("true_relres", C.c_double), ("updated_relres", C.c_double),
                ("switch_iter", C.c_int * 3), ("seconds", C.c_double),
                ("relres_hist", C.POINTER(C.c_double)), ("prec_hist", C.POINTER(C.c_uint8)),
                ("kernel_launches", C.c_int64)]


class TuningC(C.Structure):
    _fields_ = [("fused", C.c_int * 6), ("us_plain", C.c_double * 6), ("us_fused", C.c_double * 6),
                ("iters", C.c_int), ("cached", C.c_int), ("reserved", C.c_int), ("pad", C.c_int)]


class BatchTuningC(C.Structure):
    _fields_ = [("block", C.c_int * 2), ("ms", C.c_double * 2), ("chosen", C.c_int), ("iters", C.c_int)]


class KernelTimesC(C.Structure):
    _fields_ = [("ms", (C.c_double * 6) * 4), ("launches", (C.c_int * 6) * 4), ("total_ms", C.c_double)]


# event-timed slots of an iteration in the launch-by-launch mode: the
# precondition step (with Jacobi or no preconditioner also rho, beta and the
# search direction, one cooperative kernel), the search direction (Chebyshev
# only), SpMV + gamma, update + norm.  Where the whole iteration is one
# cooperative launch (k_loop: Jacobi or none, narrow slices) its time is
# reported as "iteration".
KERNEL_NAMES = ("precond", "search_dir", "spmv_gamma", "update_norm")


def phase_name(phase: int) -> str:
    """Phase index 2*u_z + u_r -> e.g. 'uz16_ur64'."""
    bits = {FP64: "64", FP32: "32", FP16: "16"}
    return f"uz{bits[phase // 2]}_ur{bits[phase % 2]}"


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libampcg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libampcg.so not built ({path}); run paper_2505_04155_b300/build.py")
    lib = C.CDLL(path)
    vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
    lib.ampcg_policy_default.argtypes = [C.POINTER(PolicyC)]
    lib.ampcg_policy_default.restype = None
    lib.ampcg_create_csr.argtypes = [C.POINTER(vp), i64, i64, vp, vp, vp, C.POINTER(PrecondSpec), vp]
    lib.ampcg_create_csr.restype = C.c_int
    lib.ampcg_create_bsr.argtypes = [C.POINTER(vp), i64, C.c_int, i64, vp, vp, vp,
                                     C.POINTER(PrecondSpec), vp]
    lib.ampcg_create_bsr.restype = C.c_int
    lib.ampcg_destroy.argtypes = [vp]
    lib.ampcg_destroy.restype = None
    lib.ampcg_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(PolicyC), C.POINTER(ResultC)]
    lib.ampcg_solve.restype = C.c_int
    lib.ampcg_solve_timed.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(PolicyC),
                                      C.POINTER(ResultC), C.POINTER(KernelTimesC)]
    lib.ampcg_solve_timed.restype = C.c_int
    lib.ampcg_precond_interval.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.ampcg_precond_interval.restype = C.c_int
    lib.ampcg_update_values.argtypes = [vp, vp]
    lib.ampcg_update_values.restype = C.c_int
    lib.ampcg_adjoint.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(PolicyC), vp, vp,
                                  C.POINTER(ResultC)]
    lib.ampcg_adjoint.restype = C.c_int
    lib.ampcg_assemble_log_coeff.argtypes = [vp, vp, vp]
    lib.ampcg_assemble_log_coeff.restype = C.c_int
    lib.ampcg_grad_log_coeff.argtypes = [vp, vp, vp, vp]
    lib.ampcg_grad_log_coeff.restype = C.c_int
    lib.ampcg_solve_batched.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                        C.c_double, C.c_int, C.POINTER(PolicyC), C.POINTER(ResultC)]
    lib.ampcg_solve_batched.restype = C.c_int
    lib.ampcg_spmv.argtypes = [vp, C.c_int, vp, vp]
    lib.ampcg_spmv.restype = C.c_int
    lib.ampcg_precond_apply.argtypes = [vp, C.c_int, C.c_int, C.c_double, vp, vp]
    lib.ampcg_precond_apply.restype = C.c_int
    lib.ampcg_spmv_loop_step.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.POINTER(C.c_double)]
    lib.ampcg_spmv_loop_step.restype = C.c_int
    lib.ampcg_spmv_block.argtypes = [vp, C.c_int, vp, vp]
    lib.ampcg_spmv_block.restype = C.c_int
    lib.ampcg_residual.argtypes = [vp, vp, vp, vp]
    lib.ampcg_residual.restype = C.c_int
    lib.ampcg_selector_trace.argtypes = [C.POINTER(PolicyC), dp, C.c_int, C.c_double, C.c_double,
                                         C.POINTER(C.c_uint8)]
    lib.ampcg_selector_trace.restype = C.c_int
    lib.ampcg_selector_trace_noalloc.argtypes = [C.POINTER(PolicyC), dp, C.c_int, C.c_double,
                                                 C.c_double, C.POINTER(C.c_uint8)]
    lib.ampcg_selector_trace_noalloc.restype = C.c_int
    lib.ampcg_tune.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.POINTER(TuningC)]
    lib.ampcg_tune.restype = C.c_int
    lib.ampcg_set_tuning.argtypes = [vp, C.c_int, C.POINTER(TuningC)]
    lib.ampcg_set_tuning.restype = C.c_int
    lib.ampcg_tune_batched.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(PolicyC), C.c_int,
                                       C.POINTER(BatchTuningC)]
    lib.ampcg_tune_batched.restype = C.c_int
    lib.ampcg_set_batch_block.argtypes = [C.c_int, C.POINTER(vp), C.c_int]
    lib.ampcg_set_batch_block.restype = C.c_int
    lib.ampcg_barrier_check.argtypes = [C.c_int, C.c_int, C.c_longlong]
    lib.ampcg_barrier_check.restype = C.c_int
    lib.ampcg_rows.argtypes = [vp]
    lib.ampcg_rows.restype = i64
    lib.ampcg_layout_stats.argtypes = [vp, C.POINTER(LayoutC)]
    lib.ampcg_layout_stats.restype = C.c_int
    lib.ampcg_status_string.argtypes = [C.c_int]
    lib.ampcg_status_string.restype = C.c_char_p
    lib.ampcg_last_error.argtypes = []
    lib.ampcg_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load_library().ampcg_status_string(s).decode()


def _check(status: int, ok=(OK,)):
    if status not in ok:
        raise AmpcgError(status, load_library().ampcg_last_error().decode())
    return status


def _ptr(a):
    """Raw pointer of a NumPy array or torch tensor (contiguity is required)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


@dataclass
class Policy:
    """Precision policy (ampcg_policy); defaults are the paper's constants for
    AMP-PCG(FP16) with the linear-convergence criterion."""
    u0: int = FP16
    criterion: int = CRIT_LINEAR
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
    graph_chunk: int = 0     # 0: automatic (256 with the persistent kernel, else 16)

    def to_c(self) -> PolicyC:
        return PolicyC(self.u0, self.criterion, self.d, self.ell, self.C, self.tau_zs, self.tau_zh,
                       self.scale, self.latch, self.verify_refresh, self.fixed_uz, self.fixed_ur,
                       self.graph_chunk)

    @staticmethod
    def pcg64(**kw) -> "Policy":
        """Plain PCG (Algorithm 1) on the same kernels: FIXED (FP64, FP64), no scaling."""
        return Policy(criterion=CRIT_FIXED, fixed_uz=FP64, fixed_ur=FP64, scale=SCALE_NONE, **kw)


def default_policy() -> Policy:
    pc = PolicyC()
    load_library().ampcg_policy_default(C.byref(pc))
    return Policy(pc.u0, pc.criterion, pc.d, pc.ell, pc.C, pc.tau_zs, pc.tau_zh, pc.scale, pc.latch,
                  pc.verify_refresh, pc.fixed_uz, pc.fixed_ur, pc.graph_chunk)


@dataclass
class SolveInfo:
    status: int
    iters: int
    converged: bool
    refreshes: int
    true_relres: float
    updated_relres: float
    switch_iter: tuple
    seconds: float
    kernel_launches: int = 0
    relres_hist: np.ndarray | None = field(default=None, repr=False)
    prec_hist: np.ndarray | None = field(default=None, repr=False)
    kernel_ms: dict | None = field(default=None, repr=False)
    kernel_launches_by: dict | None = field(default=None, repr=False)
    kernel_total_ms: float | None = None


class Solver:
    """One SPD matrix (CSR) with its preconditioner on the GPU (ampcg_create_csr)."""

    def __init__(self, rowptr, col, val, precond: int = M_JACOBI, degree: int = 0,
                 lmin: float = 0.0, lmax: float = 0.0, stream=None):
        lib = load_library()
        if isinstance(rowptr, np.ndarray):
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = int(rowptr.shape[0]) - 1
        self.nnz = int(col.shape[0])
        spec = PrecondSpec(precond, degree, lmin, lmax)
        h = C.c_void_p()
        st = _torch_stream() if stream is None else stream
        _check(lib.ampcg_create_csr(C.byref(h), self.n, self.nnz, _ptr(rowptr), _ptr(col), _ptr(val),
                                    C.byref(spec), st))
        self._h = h

    @classmethod
    def from_bsr(cls, browptr, bcol, bval, bs: int, precond: int = M_JACOBI, degree: int = 0,
                 lmin: float = 0.0, lmax: float = 0.0, stream=None) -> "Solver":
        """Context from block CSR (ampcg_create_bsr): bval holds nnzb row-major
        bs x bs blocks; the solver works on the scalar system of nb*bs rows."""
        lib = load_library()
        if isinstance(browptr, np.ndarray):
            browptr = np.ascontiguousarray(browptr, dtype=np.int32)
            bcol = np.ascontiguousarray(bcol, dtype=np.int32)
            bval = np.ascontiguousarray(bval, dtype=np.float64)
        self = cls.__new__(cls)
        nb = int(browptr.shape[0]) - 1
        nnzb = int(bcol.shape[0])
        self.n = nb * bs
        self.nnz = nnzb * bs * bs
        spec = PrecondSpec(precond, degree, lmin, lmax)
        h = C.c_void_p()
        st = _torch_stream() if stream is None else stream
        _check(lib.ampcg_create_bsr(C.byref(h), nb, bs, nnzb, _ptr(browptr), _ptr(bcol), _ptr(bval),
                                    C.byref(spec), st))
        self._h = h
        return self

    def close(self):
        if getattr(self, "_h", None):
            load_library().ampcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, x=None, tol: float = 1e-10, maxit: int = 2000, policy: Policy | None = None,
              history: bool = True, raise_on_breakdown: bool = False, timed: bool = False):
        """Solve A x = b.  `x` (same kind of array as b) holds x_0 on entry and
        the result on exit; if None, x_0 = 0 and a new array is returned.
        timed=True uses ampcg_solve_timed and adds per-kernel, per-phase
        device times to the returned info (info.kernel_ms, info.kernel_launches_by)."""
        if x is None:
            if isinstance(b, np.ndarray):
                x = np.zeros(self.n)
            else:
                import torch
                x = torch.zeros_like(b)
        pol = (policy or Policy()).to_c()
        res = ResultC()
        rh = ph = None
        if history:
            rh = np.zeros(maxit + 2)
            ph = np.zeros(max(maxit, 1), dtype=np.uint8)
            res.relres_hist = rh.ctypes.data_as(C.POINTER(C.c_double))
            res.prec_hist = ph.ctypes.data_as(C.POINTER(C.c_uint8))
        kt = KernelTimesC()
        if timed:
            s = load_library().ampcg_solve_timed(self._h, _ptr(b), _ptr(x), tol, maxit, C.byref(pol),
                                                 C.byref(res), C.byref(kt))
        else:
            s = load_library().ampcg_solve(self._h, _ptr(b), _ptr(x), tol, maxit, C.byref(pol),
                                           C.byref(res))
        ok = (OK, NOT_CONVERGED) if raise_on_breakdown else (OK, NOT_CONVERGED, ERR_BREAKDOWN, ERR_NONFINITE)
        _check(s, ok)
        it = res.iters
        info = SolveInfo(res.status, it, bool(res.converged), res.refreshes, res.true_relres,
                         res.updated_relres, tuple(res.switch_iter), res.seconds,
                         res.kernel_launches, rh[: it + 1].copy() if history else None, ph[:it].copy() if history else None)
        if timed:
            def slot_name(j, ph_):
                # one launch in slot 0 only: the whole iteration (k_loop)
                if j == 0 and not any(kt.launches[i][ph_] for i in (1, 2, 3)):
                    return "iteration"
                return KERNEL_NAMES[j]
            info.kernel_ms = {(slot_name(j, ph_), phase_name(ph_)): kt.ms[j][ph_]
                              for j in range(4) for ph_ in range(6) if kt.launches[j][ph_]}
            info.kernel_launches_by = {(slot_name(j, ph_), phase_name(ph_)): kt.launches[j][ph_]
                                    for j in range(4) for ph_ in range(6) if kt.launches[j][ph_]}
            info.kernel_total_ms = kt.total_ms
        return x, info

    def tune(self, scale: int = SCALE_LINF_POW2_LAG, iters: int = 20, pairs=None) -> dict:
        """Autotune the persistent iteration kernel's form per precision pair
        for solves under `scale` (SCALE_NONE, SCALE_LINF_POW2_LAG or
        SCALE_LINF_POW2, each tuned on its own; ampcg_tune): pairs is an iterable of phase indices 2*u_z + u_r, or
        None for all six.  Returns the choices and the measured times."""
        mask = 0 if pairs is None else sum(1 << p for p in pairs)
        t = TuningC()
        _check(load_library().ampcg_tune(self._h, scale, iters, mask, C.byref(t)))
        return {"fused": {phase_name(p): t.fused[p] for p in range(6) if t.fused[p] >= 0},
                "us_four_barrier": {phase_name(p): round(t.us_plain[p], 2) for p in range(6) if t.us_plain[p] > 0},
                "us_three_barrier": {phase_name(p): round(t.us_fused[p], 2) for p in range(6) if t.us_fused[p] > 0},
                "iters": t.iters, "cached": bool(t.cached)}

    def set_tuning(self, fused, scale: int = SCALE_LINF_POW2_LAG):
        """Set the kernel form per pair for solves under `scale`
        (ampcg_set_tuning): fused is a sequence of six values -1 (automatic),
        0 (four barriers) or 1 (three)."""
        t = TuningC()
        for p in range(6):
            t.fused[p] = int(fused[p])
        _check(load_library().ampcg_set_tuning(self._h, scale, C.byref(t)))

    def layout(self) -> dict:
        """Storage statistics of the sliced layout (ampcg_layout_stats)."""
        out = LayoutC()
        _check(load_library().ampcg_layout_stats(self._h, C.byref(out)))
        return {k: getattr(out, k) for k, _ in LayoutC._fields_}

    def interval(self):
        """The Chebyshev interval (lmin, lmax) in use (ampcg_precond_interval)."""
        lo, hi = C.c_double(), C.c_double()
        _check(load_library().ampcg_precond_interval(self._h, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def update_values(self, vals):
        """New FP64 values on the same pattern, CSR order (ampcg_update_values)."""
        _check(load_library().ampcg_update_values(self._h, _ptr(vals)))

    def adjoint(self, x, dLdx, tol: float = 1e-10, maxit: int = 2000, policy: Policy | None = None,
                want_dA: bool = True):
        """Adjoint solve A lambda = dL/dx (ampcg_adjoint): returns (lambda = dL/db,
        dL/dA on the pattern in CSR order or None, info)."""
        like = dLdx
        if isinstance(like, np.ndarray):
            lam = np.zeros(self.n)
            dA = np.zeros(self.nnz) if want_dA else None
        else:
            import torch
            lam = torch.zeros_like(like)
            dA = torch.zeros(self.nnz, dtype=like.dtype, device=like.device) if want_dA else None
        pol = (policy or Policy()).to_c()
        res = ResultC()
        s = load_library().ampcg_adjoint(self._h, _ptr(x), _ptr(dLdx), tol, maxit, C.byref(pol),
                                         _ptr(lam), _ptr(dA) if want_dA else None, C.byref(res))
        _check(s, (OK, NOT_CONVERGED))
        info = SolveInfo(res.status, res.iters, bool(res.converged), res.refreshes, res.true_relres,
                         res.updated_relres, tuple(res.switch_iter), res.seconds, res.kernel_launches)
        return lam, dA, info

    def assemble_log_coeff(self, theta, nbound):
        """Values from a log-coefficient field (ampcg_assemble_log_coeff)."""
        _check(load_library().ampcg_assemble_log_coeff(self._h, _ptr(theta), _ptr(nbound)))

    def grad_log_coeff(self, x, lam, out=None):
        """dL/dtheta from the forward solution and the adjoint (ampcg_grad_log_coeff)."""
        if out is None:
            if isinstance(x, np.ndarray):
                out = np.zeros(self.n)
            else:
                import torch
                out = torch.zeros_like(x)
        _check(load_library().ampcg_grad_log_coeff(self._h, _ptr(x), _ptr(lam), _ptr(out)))
        return out

    def spmv(self, p, q, prec: int = FP64):
        """q = A p in FP64 or FP32 (device arrays)."""
        _check(load_library().ampcg_spmv(self._h, prec, _ptr(p), _ptr(q)))
        return q

    def spmv_block(self, p, q, prec: int = FP64):
        """q = A p with the 3 x 3 block-row layout (ampcg_spmv_block; device arrays)."""
        _check(load_library().ampcg_spmv_block(self._h, prec, _ptr(p), _ptr(q)))
        return q

    def spmv_loop_step(self, p, q, uz: int, ur: int) -> float:
        """q = A p as the persistent iteration kernel computes it (its launch
        shape and work split): p in u_z, q in u_r (device arrays); returns
        gamma = q^T p as that kernel accumulates it (ampcg_spmv_loop_step)."""
        g = C.c_double()
        _check(load_library().ampcg_spmv_loop_step(self._h, uz, ur, _ptr(p), _ptr(q), C.byref(g)))
        return g.value

    def precond_apply(self, r, z, uz: int, ur: int, omega: float = 1.0):
        """z = M^-1 round_uz(omega r) with r in u_r and z in u_z (device arrays)."""
        _check(load_library().ampcg_precond_apply(self._h, uz, ur, omega, _ptr(r), _ptr(z)))
        return z

    def residual(self, b, x, r):
        """r = b - A x in FP64 (device arrays)."""
        _check(load_library().ampcg_residual(self._h, _ptr(b), _ptr(x), _ptr(r)))
        return r


def selector_trace(delta, nb: float, tol: float, policy: Policy | None = None) -> np.ndarray:
    """Device precision selector replayed over delta[0..m]; (u_z << 4) | u_r per k."""
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    out = np.zeros(delta.size, dtype=np.uint8)
    pol = (policy or Policy()).to_c()
    _check(load_library().ampcg_selector_trace(C.byref(pol), delta.ctypes.data_as(C.POINTER(C.c_double)),
                                               delta.size - 1, nb, tol,
                                               out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


def selector_trace_noalloc(delta, nb: float, tol: float, policy: Policy | None = None) -> np.ndarray:
    """selector_trace without any device allocation (ampcg_selector_trace_noalloc):
    for callers that must not call cudaMalloc.  At most 65536 residual norms;
    concurrent calls share one static device array and must be serialised."""
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    out = np.zeros(delta.size, dtype=np.uint8)
    pol = (policy or Policy()).to_c()
    _check(load_library().ampcg_selector_trace_noalloc(
        C.byref(pol), delta.ctypes.data_as(C.POINTER(C.c_double)), delta.size - 1, nb, tol,
        out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


def solve_batched(solvers, bs, xs, tol: float = 1e-10, maxit: int = 2000,
                  policy: Policy | None = None, history: bool = False):
    """Solve independent systems in one call (ampcg_solve_batched); xs hold
    the initial guesses and receive the solutions.  Returns a list of
    SolveInfo (with relres/precision histories when history=True)."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s._h.value for s in solvers])
    bp = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    xp = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    res = (ResultC * n)()
    hist = []
    if history:
        for r in res:
            rh, ph = np.zeros(maxit + 2), np.zeros(max(maxit, 1), dtype=np.uint8)
            r.relres_hist = rh.ctypes.data_as(C.POINTER(C.c_double))
            r.prec_hist = ph.ctypes.data_as(C.POINTER(C.c_uint8))
            hist.append((rh, ph))
    pol = (policy or Policy()).to_c()
    st = load_library().ampcg_solve_batched(n, hs, bp, xp, tol, maxit, C.byref(pol), res)
    _check(st, (OK, NOT_CONVERGED, ERR_BREAKDOWN, ERR_NONFINITE))
    out = []
    for j, r in enumerate(res):
        rh, ph = hist[j] if history else (None, None)
        out.append(SolveInfo(r.status, r.iters, bool(r.converged), r.refreshes, r.true_relres,
                             r.updated_relres, tuple(r.switch_iter), r.seconds, r.kernel_launches,
                             rh[: r.iters + 1].copy() if history else None,
                             ph[: r.iters].copy() if history else None))
    return out


def barrier_check(nblocks: int = 2, absent_block: int = -1, spin_limit: int = 1 << 21) -> int:
    """One bounded grid barrier of the iteration kernel's kind (ampcg_barrier_check):
    returns OK when every arriving block passed, ERR_TIMEOUT when a wait ran out
    (absent_block in [0, nblocks) never arrives).  Other statuses raise."""
    return _check(load_library().ampcg_barrier_check(nblocks, absent_block, spin_limit),
                  ok=(OK, ERR_TIMEOUT))


def tune_batched(solvers, iters: int = 20, policy: Policy | None = None) -> dict:
    """Autotune ampcg_solve_batched's block size for this batch (ampcg_tune_batched)."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s._h.value for s in solvers])
    pol = (policy or Policy()).to_c()
    t = BatchTuningC()
    _check(load_library().ampcg_tune_batched(n, hs, C.byref(pol), iters, C.byref(t)))
    return {"ms": {t.block[j]: round(t.ms[j], 3) for j in range(2)}, "chosen": t.chosen, "iters": t.iters}


def set_batch_block(solvers, block: int):
    """Block size of the batched kernel for batches led by these solvers (0, 1024 or 512)."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s._h.value for s in solvers])
    _check(load_library().ampcg_set_batch_block(n, hs, block))

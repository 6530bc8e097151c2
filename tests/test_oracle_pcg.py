"""Pins for the oracle's PCG (Algorithm 1), DS-PCG (Algorithm 2) and the
FP64 path of AMP-PCG (Algorithm 3) against mathematics that does not depend on
the oracle: direct solves (dense Cholesky, sparse LU), SciPy's CG iteration
count, CG's finite termination on a matrix with few distinct eigenvalues, the
monotone A-norm error of CG, and the exact-arithmetic equivalence of DS-PCG and
PCG (Theorem 3.2), which holds bit for bit when omega is a power of two."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workloads as W


def _sp(a):
    return sp.csr_matrix((a.val, a.col, a.rowptr), shape=(a.n, a.n))


@pytest.mark.parametrize("n,kappa,seed", [(60, 1e2, 1), (200, 1e3, 2), (300, 1e4, 3)])
def test_pcg64_matches_dense_cholesky(n, kappa, seed):
    eigs = np.geomspace(1.0 / kappa, 1.0, n)
    a = W.dense_spd_csr(eigs, seed)
    b = W.rhs_uniform(n, seed)
    dense = a.to_dense()
    x_star = sla.cho_solve(sla.cho_factor(dense), b)
    tol = 1e-12
    r = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=tol, maxit=20 * n)
    assert r.converged
    err = np.linalg.norm(r.x - x_star) / np.linalg.norm(x_star)
    assert err <= 10 * kappa * tol
    assert r.true_relres <= 10 * tol


def test_pcg64_config1_against_splu_and_scipy_cg():
    a = W.poisson2d(64)
    b = W.rhs_uniform(a.n, 0)
    A = _sp(a)
    x_star = spla.spsolve(A.tocsc(), b)
    r = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=2000)
    assert r.converged and r.status == oracle.OK
    # kappa(A) of the 64x64 5-point Laplacian < 1.8e3
    err = np.linalg.norm(r.x - x_star) / np.linalg.norm(x_star)
    assert err <= 1.8e3 * 1e-10
    assert r.true_relres <= 1e-10 * 1.01
    # SciPy's CG with the same Jacobi M, rtol, x0 = 0 counts the same steps
    dinv = 1.0 / A.diagonal()
    M = spla.LinearOperator(A.shape, matvec=lambda v: dinv * v)
    count = [0]
    spla.cg(A, b, rtol=1e-10, atol=0.0, maxiter=2000, M=M, callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert abs(count[0] - r.iters) <= 1


def test_cg_terminates_in_distinct_eigenvalue_count():
    # A with 4 distinct eigenvalues: the Krylov space has dimension <= 4
    eigs = np.repeat([0.1, 0.5, 2.0, 7.0], 20)
    a = W.dense_spd_csr(eigs, 4)
    b = W.rhs_uniform(a.n, 4)
    r = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=100, jacobi=False)
    assert r.converged and r.iters <= 5


def test_a_norm_error_is_monotone():
    eigs = np.linspace(1e-2, 1.0, 120)
    a = W.dense_spd_csr(eigs, 5)
    b = W.rhs_uniform(a.n, 5)
    A = a.to_dense()
    x_star = np.linalg.solve(A, b)
    errs = []
    for k in range(1, 40):
        xk = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-30, maxit=k, jacobi=False).x
        e = x_star - xk
        errs.append(np.sqrt(e @ A @ e))
    assert np.all(np.diff(errs) < 0)


def _amp(a, b, **kw):
    tol = kw.pop("tol", 1e-10)
    maxit = kw.pop("maxit", 3000)
    precond = kw.pop("precond", oracle.M_JACOBI)
    return oracle.ampcg(a.rowptr, a.col, a.val, b, tol=tol, maxit=maxit, precond=precond,
                        policy=oracle.Policy(**kw))


def test_ampcg_fixed64_equals_alg1_bitwise():
    a = W.diffusion3d(16, 2.0, 0)
    b = W.rhs_uniform(a.n, 1)
    ref = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=3000)
    amp = _amp(a, b, criterion=oracle.FIXED, fixed_uz=oracle.FP64, fixed_ur=oracle.FP64,
               scale=oracle.SCALE_NONE)
    assert amp.iters == ref.iters
    assert np.array_equal(amp.x, ref.x)
    assert np.array_equal(amp.relres_hist, ref.relres_hist)


@pytest.mark.parametrize("scale", [oracle.SCALE_LINF_POW2, oracle.SCALE_LINF_POW2_LAG])
@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_dspcg_pow2_scaling_is_bitwise_pcg(prec, scale):
    # Theorem 3.2: every DS-PCG quantity is PCG's times an exact power of two,
    # whichever powers of two the omega_k are (the current or the previous
    # iteration's max|r|, reading R20)
    a = W.diffusion3d(12, 1.0, 3)
    b = W.rhs_uniform(a.n, 2) * 1e3
    base = dict(criterion=oracle.FIXED, fixed_uz=prec, fixed_ur=prec, tol=1e-6)
    plain = _amp(a, b, scale=oracle.SCALE_NONE, **base)
    scaled = _amp(a, b, scale=scale, **base)
    assert plain.iters == scaled.iters
    assert np.array_equal(plain.x, scaled.x)
    assert np.array_equal(plain.relres_hist, scaled.relres_hist)


def test_dspcg_l2_scaling_close_to_pcg():
    a = W.diffusion3d(12, 1.0, 3)
    b = W.rhs_uniform(a.n, 2)
    base = dict(criterion=oracle.FIXED, fixed_uz=oracle.FP64, fixed_ur=oracle.FP64)
    plain = _amp(a, b, scale=oracle.SCALE_NONE, **base)
    l2 = _amp(a, b, scale=oracle.SCALE_L2, **base)
    assert abs(plain.iters - l2.iters) <= 1
    assert np.linalg.norm(plain.x - l2.x) / np.linalg.norm(plain.x) < 1e-8


def test_breakdown_and_nonfinite_statuses():
    a = W.poisson2d(8)
    b = W.rhs_uniform(a.n, 0)
    bad = a.val.copy()
    diag = a.col == np.repeat(np.arange(a.n), np.diff(a.rowptr))
    bad[diag] = -bad[diag]          # negative definite: gamma < 0 at once
    r = oracle.ampcg(a.rowptr, a.col, bad, b, precond=oracle.M_NONE,
                     policy=oracle.Policy(criterion=oracle.FIXED))
    assert r.status == oracle.ERR_BREAKDOWN
    bn = b.copy()
    bn[3] = np.nan
    r = oracle.ampcg(a.rowptr, a.col, a.val, bn, policy=oracle.Policy())
    assert r.status == oracle.ERR_NONFINITE
    r = oracle.ampcg(a.rowptr, a.col, a.val, b, maxit=3, policy=oracle.Policy())
    assert r.status == oracle.NOT_CONVERGED and r.iters == 3


def test_refresh_reaches_true_residual():
    a = W.diffusion3d(24, 2.0, 0)
    b = W.rhs_uniform(a.n, 1)
    plain = _amp(a, b, u0=oracle.FP16, criterion=oracle.WINDOW, maxit=5000)
    fixed = _amp(a, b, u0=oracle.FP16, criterion=oracle.WINDOW, verify_refresh=3, maxit=5000)
    assert fixed.converged
    assert fixed.true_relres <= 1e-10 or fixed.refreshes == 3
    assert fixed.iters >= plain.iters


def _growth_system():
    """A 2 x 2 SPD matrix on which one Jacobi-PCG step takes the residual norm
    from 1 to 8.9e4, beyond binary16's 65504: draw 13211 (from 0) of a seeded
    random family Q diag(e^u) Q^T scaled by D A D, b with spread magnitudes."""
    rng = np.random.default_rng(1)
    for _ in range(13212):
        th = rng.uniform(0, np.pi)
        ev = np.exp(rng.uniform(-12, 2, 2))
        sc = np.exp(rng.uniform(-6, 6, 2))
        b = rng.standard_normal(2) * np.exp(rng.uniform(-6, 0, 2))
    q = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    m = q @ np.diag(ev) @ q.T
    m = (m + m.T) / 2 * np.outer(sc, sc)
    a = W.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), m.ravel().copy(), {})
    return a, b


def test_lagged_scale_retries_with_the_exact_power_after_overflow():
    # reading R20: omega_1 from max|r_0| makes y_1 overflow binary16; rho_1 is
    # then formed again with omega_1 = 2^-ceil(log2 max|r_1|), the non-lagged
    # mode's omega_1, so both runs agree bit for bit (no binary16 subnormals
    # occur here, so the different powers of two of iteration 0 change nothing)
    a, b = _growth_system()
    assert np.all(np.linalg.eigvalsh(a.val.reshape(2, 2)) > 0)
    base = dict(criterion=oracle.FIXED, fixed_uz=oracle.FP16, fixed_ur=oracle.FP64, tol=1e-30,
                maxit=2, precond=oracle.M_JACOBI)
    lag = _amp(a, b, scale=oracle.SCALE_LINF_POW2_LAG, **base)
    exact = _amp(a, b, scale=oracle.SCALE_LINF_POW2, **base)
    assert lag.relres_hist[1] / lag.relres_hist[0] > 65504
    assert lag.scale_retries == 1 and exact.scale_retries == 0
    assert lag.status == exact.status == oracle.NOT_CONVERGED and lag.iters == 2
    assert np.array_equal(lag.x, exact.x) and np.array_equal(lag.relres_hist, exact.relres_hist)


def test_binary16_underflow_count_of_the_scaling_step():
    # one iteration on a diagonal system: the counts cover y_0 = round16(omega_0 r_0)
    # with r_0 = b, omega_0 = 2^-ceil(log2 max|b|) = 2^-1 here
    b = np.array([1.5, 2.0 ** -20, 2.0 ** -10, 0.0, 3e-5, -1e-6, 0.25, 2.0 ** -13])
    n = b.size
    a = W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n), {})
    r = _amp(a, b, criterion=oracle.FIXED, fixed_uz=oracle.FP16, fixed_ur=oracle.FP64, maxit=1, tol=1e-30,
             scale=oracle.SCALE_LINF_POW2, precond=oracle.M_NONE)
    y = b * 0.5
    assert r.y16_total == np.count_nonzero(b)
    assert r.y16_small == np.count_nonzero((b != 0) & (np.abs(y) < 2.0 ** -14))

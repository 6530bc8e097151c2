"""Pins for the oracle's Chebyshev preconditioner (reading R8): the
three-term recurrence of the Chebyshev iteration against the closed-form
polynomial evaluated on the eigen-decomposition of Ahat = D^-1/2 A D^-1/2,
  z = D^-1/2 V P(L) V^T D^-1/2 y,  P(l) = (1 - T_m((t - l)/d) / T_m(t/d)) / l,
t = (lmax + lmin)/2, d = (lmax - lmin)/2, and positivity of P on the spectrum
(M SPD) whenever lmax bounds the spectrum from above."""
import numpy as np
import pytest

import oracle
import workloads as W


def _T(m, x):
    x = np.asarray(x, dtype=np.float64)
    t0, t1 = np.ones_like(x), x.copy()
    if m == 0:
        return t0
    for _ in range(m - 1):
        t0, t1 = t1, 2 * x * t1 - t0
    return t1


@pytest.mark.parametrize("m", [1, 2, 5, 8])
def test_recurrence_matches_closed_form(m):
    a = W.diffusion3d(5, 1.5, 2)
    dense = a.to_dense()
    d = np.diag(dense)
    dsi = 1.0 / np.sqrt(d)
    ah = dsi[:, None] * dense * dsi[None, :]
    lam, V = np.linalg.eigh(ah)
    lmax = 1.05 * lam[-1]
    lmin = lmax / 30.0
    t, dd = (lmax + lmin) / 2, (lmax - lmin) / 2
    P = (1.0 - _T(m, (t - lam) / dd) / _T(m, t / dd)) / lam
    assert np.all(P > 0)                        # M is SPD
    y = W.rhs_uniform(a.n, 3)
    want = dsi * (V @ (P * (V.T @ (dsi * y))))
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    ahat_csr = dsi[rows] * a.val * dsi[a.col]
    got = oracle.cheb_apply(a.rowptr, a.col, ahat_csr, dsi, m, lmin, lmax, oracle.FP64, y)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_degree_one_is_scaled_jacobi():
    # one step: z = D^-1/2 (D^-1/2 y / theta) = D^-1 y / theta
    a = W.poisson2d(6)
    y = W.rhs_uniform(a.n, 1)
    d = 4.0
    lmin, lmax = 0.1, 2.0
    theta = (lmax + lmin) / 2
    z = oracle.scale_cheb(a.rowptr, a.col, a.val, 1, lmin, lmax, oracle.FP64, oracle.FP64, 1.0, y)
    assert np.allclose(z, y / d / theta, rtol=1e-15, atol=0)


def test_ampcg_with_chebyshev_converges_fewer_iterations():
    a = W.diffusion3d(10, 1.0, 4)
    b = W.rhs_uniform(a.n, 5)
    jac = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=5000,
                       policy=oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW))
    ch = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=5000, precond=oracle.M_CHEBYSHEV,
                      cheb_degree=6, cheb_lmin=2.0 / 30, cheb_lmax=2.0,
                      policy=oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW))
    assert ch.converged and jac.converged
    assert ch.iters < 0.6 * jac.iters
    assert ch.true_relres <= 2e-10

"""Pin for the oracle's coefficient-field gradient (the adjoint identity
dL/da_ij = -lambda_i x_j pushed through the log-coefficient assembly):
central finite differences of L(theta) = 0.5 ||x(theta) - x_t||^2 along random
directions, with FP64 oracle solves to 1e-14 and the generator's assembly."""
import numpy as np

import oracle
import workloads as W


def _solve(a, b):
    r = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-14, maxit=20000)
    assert r.converged
    return r.x


def test_grad_log_coeff_matches_central_differences():
    n = 6
    theta, theta_t, a, a_t, b = W.log_coeff_problem(n, sigma=1.0, seed=3)
    x_t = _solve(a_t, b)
    x = _solve(a, b)
    lam = _solve(a, x - x_t)                 # A lambda = dL/dx
    g = oracle.grad_log_coeff(a.rowptr, a.col, a.val, x, lam)
    rng = np.random.default_rng(5)
    h = 1e-6

    def loss(th):
        aa = W.diffusion3d_from_field(th.reshape(n, n, n))
        xx = _solve(aa, b)
        return 0.5 * np.sum((xx - x_t) ** 2)

    for _ in range(4):
        d = rng.standard_normal(theta.size)
        fd = (loss(theta + h * d) - loss(theta - h * d)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), 1e-12)


def test_adjoint_identity_on_values():
    # dL/db = lambda and dL/da_ij = -lambda_i x_j against differences in b and A
    a = W.poisson2d(7)
    b = W.rhs_uniform(a.n, 4)
    c = W.rhs_uniform(a.n, 5)
    x = _solve(a, b)
    lam = _solve(a, c)                       # L = c^T x, dL/dx = c
    h = 1e-6
    rng = np.random.default_rng(6)
    db = rng.standard_normal(a.n)
    fd_b = (c @ _solve(a, b + h * db) - c @ _solve(a, b - h * db)) / (2 * h)
    assert abs(fd_b - lam @ db) <= 1e-7 * abs(fd_b)
    # symmetric perturbation of the values keeps A SPD
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    dv = rng.standard_normal(a.nnz) * 0.1
    dense = np.zeros((a.n, a.n))
    dense[rows, a.col] = dv
    dense = 0.5 * (dense + dense.T)
    dv = dense[rows, a.col]
    ap = W.CSR(a.n, a.rowptr, a.col, a.val + h * dv, {})
    am = W.CSR(a.n, a.rowptr, a.col, a.val - h * dv, {})
    fd_a = (c @ _solve(ap, b) - c @ _solve(am, b)) / (2 * h)
    dLdA = -lam[rows] * x[a.col]
    assert abs(fd_a - dLdA @ dv) <= 1e-6 * abs(fd_a)

"""Adjoint and autograd through the C ABI (ampcg_adjoint, ampcg_update_values,
ampcg_assemble_log_coeff, ampcg_grad_log_coeff) against the FP64 oracle
(oracle solves to 1e-13/1e-14 and the oracle's gradient definition, itself
pinned by finite differences on the CPU) and against central finite
differences of the loss L(theta) = 0.5 ||x(theta) - x_t||^2.

Tolerances: with FP64 PCG at tol 1e-13 the gradient agrees with the oracle's
to 1e-8 (norm-wise); with AMP-PCG(FP16) at an FP64-verified 1e-10 the error
is bounded by kappa * 1e-10 relative (kappa <= 1e4 for these fields), so 1e-4."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")
from paper_2505_04155_b300 import autograd as AG  # noqa: E402


def _osolve(a, b, tol=1e-14):
    r = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=tol, maxit=50000)
    assert r.converged
    return r.x


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def test_assemble_log_coeff_matches_generator():
    theta, _, a, _, _ = W.log_coeff_problem(9, sigma=1.5, seed=4)
    s = P.Solver(a.rowptr, a.col, np.ones_like(a.val) * -1 + 8 * (a.col == np.repeat(
        np.arange(a.n), np.diff(a.rowptr))))                  # a different SPD start
    s.assemble_log_coeff(_dev(theta), torch.as_tensor(a.info["nbound"], device="cuda"))
    p = np.random.default_rng(1).standard_normal(a.n)
    q = torch.empty(a.n, dtype=torch.float64, device="cuda")
    s.spmv(_dev(p), q, P.FP64)
    torch.cuda.synchronize()
    want = oracle.spmv(a.rowptr, a.col, a.val, oracle.FP64, p)
    assert _rel(q.cpu().numpy(), want) < 1e-13
    s.close()


@pytest.mark.parametrize("policy,tol,rtol", [(P.Policy.pcg64(), 1e-13, 1e-8),
                                             (P.Policy(verify_refresh=3), 1e-10, 1e-4)])
def test_adjoint_lambda_and_pattern_gradient(policy, tol, rtol):
    a = W.diffusion3d(14, 1.0, 7)
    b = W.rhs_uniform(a.n, 8)
    g = W.rhs_uniform(a.n, 9)                 # dL/dx
    x = _osolve(a, b)
    s = P.Solver(a.rowptr, a.col, a.val)
    lam, dA, info = s.adjoint(_dev(x), _dev(g), tol=tol, maxit=20000, policy=policy)
    s.close()
    assert info.converged
    lam_ref = _osolve(a, g)
    assert _rel(lam.cpu().numpy(), lam_ref) < rtol
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    assert _rel(dA.cpu().numpy(), -lam_ref[rows] * x[a.col]) < rtol


def test_update_values_matches_fresh_context():
    a = W.diffusion3d(10, 2.0, 1)
    a2 = W.diffusion3d(10, 2.0, 2)             # same pattern, other values
    b = _dev(W.rhs_uniform(a.n, 3))
    s = P.Solver(a.rowptr, a.col, a.val)
    s.update_values(_dev(a2.val))
    x1, i1 = s.solve(b, tol=1e-10, maxit=5000)
    s2 = P.Solver(a2.rowptr, a2.col, a2.val)
    x2, i2 = s2.solve(b, tol=1e-10, maxit=5000)
    assert i1.iters == i2.iters and torch.equal(x1, x2)
    bad = a2.val.copy()
    bad[0] = -1.0
    with pytest.raises(P.AmpcgError):
        s.update_values(_dev(bad))
    s.close()
    s2.close()


@pytest.mark.parametrize("which", ["fp64", "amp"])
def test_log_coeff_autograd_vs_oracle_and_fd(which):
    n = 12
    theta, theta_t, a, a_t, b = W.log_coeff_problem(n, sigma=1.0, seed=11)
    x_t = _osolve(a_t, b)
    policy, tol, rtol = ((P.Policy.pcg64(), 1e-13, 1e-8) if which == "fp64"
                         else (P.Policy(verify_refresh=3), 1e-10, 1e-4))
    s = P.Solver(a.rowptr, a.col, a.val)
    nb = torch.as_tensor(a.info["nbound"], device="cuda")
    th = _dev(theta).requires_grad_(True)
    bd = _dev(b).requires_grad_(True)
    x = AG.solve_log_coeff(th, bd, s, nb, tol=tol, maxit=20000, policy=policy)
    L = 0.5 * torch.sum((x - _dev(x_t)) ** 2)
    L.backward()
    # FP64 oracle gradient (definition, pinned by finite differences on the CPU)
    xo = _osolve(a, b)
    lam = _osolve(a, xo - x_t)
    g_ref = oracle.grad_log_coeff(a.rowptr, a.col, a.val, xo, lam)
    assert _rel(th.grad.cpu().numpy(), g_ref) < rtol
    assert _rel(bd.grad.cpu().numpy(), lam) < rtol
    # central differences along random directions (oracle forward solves)
    rng = np.random.default_rng(12)
    h = 1e-6

    def loss(t):
        aa = W.diffusion3d_from_field(t.reshape(n, n, n))
        return 0.5 * np.sum((_osolve(aa, b) - x_t) ** 2)

    gd = th.grad.cpu().numpy()
    for _ in range(3):
        d = rng.standard_normal(theta.size)
        fd = (loss(theta + h * d) - loss(theta - h * d)) / (2 * h)
        assert abs(fd - gd @ d) <= max(rtol, 1e-6) * abs(fd) * 10
    s.close()


def test_values_autograd_matches_adjoint_formula():
    a = W.diffusion3d(8, 1.0, 5)
    b = W.rhs_uniform(a.n, 6)
    s = P.Solver(a.rowptr, a.col, a.val)
    vals = _dev(a.val).requires_grad_(True)
    x = AG.solve_values(vals, _dev(b), s, tol=1e-13, policy=P.Policy.pcg64())
    c = _dev(W.rhs_uniform(a.n, 7))
    (c @ x).backward()
    xo = _osolve(a, b)
    lam = _osolve(a, c.cpu().numpy())
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    assert _rel(vals.grad.cpu().numpy(), -lam[rows] * xo[a.col]) < 1e-8
    s.close()


def test_coefficient_field_64cubed():
    # the coefficient-field workload at full size: 64^3 nodes, sigma = 1
    theta, theta_t, a, a_t, b = W.log_coeff_problem(64, sigma=1.0, seed=0)
    s = P.Solver(a.rowptr, a.col, a.val)
    nb = torch.as_tensor(a.info["nbound"], device="cuda")
    st = P.Solver(a_t.rowptr, a_t.col, a_t.val)
    x_t, _ = st.solve(_dev(b), tol=1e-13, maxit=50000, policy=P.Policy.pcg64())
    st.close()
    th = _dev(theta).requires_grad_(True)
    x = AG.solve_log_coeff(th, _dev(b), s, nb, tol=1e-10, maxit=50000,
                           policy=P.Policy(verify_refresh=3))
    L = 0.5 * torch.sum((x - x_t) ** 2)
    L.backward()
    g = th.grad.cpu().numpy()
    xo = _osolve(a, b, 1e-13)
    lam = _osolve(a, xo - x_t.cpu().numpy(), 1e-13)
    g_ref = oracle.grad_log_coeff(a.rowptr, a.col, a.val, xo, lam)
    assert _rel(g, g_ref) < 1e-4
    # central differences along two directions with GPU FP64 forward solves
    rng = np.random.default_rng(0)
    h = 1e-4   # larger step: the FP64 forward solves stop at 1e-13
    f64 = P.Solver(a.rowptr, a.col, a.val)

    def loss(t):
        f64.assemble_log_coeff(_dev(t), nb)
        xx, _ = f64.solve(_dev(b), tol=1e-13, maxit=50000, policy=P.Policy.pcg64())
        return 0.5 * float(torch.sum((xx - x_t) ** 2))

    for _ in range(2):
        d = rng.standard_normal(theta.size)
        fd = (loss(theta + h * d) - loss(theta - h * d)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-4 * abs(fd)
    f64.close()
    s.close()

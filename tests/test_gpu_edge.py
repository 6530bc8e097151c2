"""Degenerate sizes and structures of the solve against the oracle: a 1 x 1
system, one full slice plus a one-row ragged tail, and a diagonal matrix (on
which Jacobi-preconditioned PCG in FP64 is exact after one iteration, Alg. 1:
z_0 = D^-1 r_0 is the solution's direction and alpha_0 = 1)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


def _solve(a, b, pol, tol=1e-10, maxit=2000):
    s = P.Solver(a.rowptr, a.col, a.val)
    bd = torch.as_tensor(b, device="cuda")
    x, info = s.solve(bd, tol=tol, maxit=maxit, policy=pol)
    s.close()
    return x.cpu().numpy(), info


def _opol(p):
    return oracle.Policy(u0=p.u0, criterion=p.criterion, d=p.d, ell=p.ell, C=p.C, tau_zs=p.tau_zs,
                         tau_zh=p.tau_zh, scale=p.scale, latch=p.latch, verify_refresh=p.verify_refresh,
                         fixed_uz=p.fixed_uz, fixed_ur=p.fixed_ur)


def _diag(n, seed):
    rng = np.random.default_rng(seed)
    d = np.exp(rng.uniform(-3.0, 3.0, n))
    return W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d, {})


def _lap1d(n):
    mid = np.arange(1, n - 1)
    col = np.concatenate([[0, 1], np.stack([mid - 1, mid, mid + 1], 1).ravel(), [n - 2, n - 1]])
    val = np.concatenate([[2.0, -1.0], np.tile([-1.0, 2.0, -1.0], n - 2), [-1.0, 2.0]])
    rowptr = np.concatenate([[0, 2], 2 + 3 * np.arange(1, n - 1), [3 * n - 2]]).astype(np.int32)
    return W.CSR(n, rowptr, col.astype(np.int32), val, {})


@pytest.mark.parametrize("variant", ["pcg64", "amp16"])
def test_one_by_one_system(variant):
    a = W.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]), {})
    b = np.array([2.0])
    pol = P.Policy.pcg64() if variant == "pcg64" else P.Policy(verify_refresh=3)
    x, info = _solve(a, b, pol)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=2000, policy=_opol(pol))
    assert info.converged and ref.converged
    assert info.iters == ref.iters
    assert x[0] == ref.x[0] == 0.5     # every quantity of the one iteration is exact here


@pytest.mark.parametrize("variant", ["pcg64", "amp16"])
def test_one_slice_and_a_ragged_row(variant):
    a = _lap1d(33)                      # 32 rows of one slice, one row of the next
    b = W.rhs_uniform(a.n, 3)
    pol = P.Policy.pcg64() if variant == "pcg64" else P.Policy(verify_refresh=3)
    x, info = _solve(a, b, pol)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=2000, policy=_opol(pol))
    assert info.converged and ref.converged
    assert abs(info.iters - ref.iters) <= (1 if variant == "pcg64" else max(2, 0.05 * ref.iters))
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    assert info.true_relres <= 1.01e-10


def test_diagonal_matrix_pcg64_is_exact_in_one_iteration():
    a = _diag(5000, 7)
    b = W.rhs_uniform(a.n, 8)
    x, info = _solve(a, b, P.Policy.pcg64())
    ref = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=2000)
    assert info.converged and info.iters == ref.iters == 1
    # alpha_0 = rho_0 / gamma_0 is 1 up to the rounding of two sums (taken in
    # another order than the oracle's), D^-1 and x each one rounding
    exact = b / a.val
    assert np.max(np.abs(x - exact) / np.abs(exact)) <= 2e-15
    assert np.max(np.abs(x - ref.x) / np.abs(ref.x)) <= 2e-15


def test_diagonal_matrix_amp16_matches_oracle():
    a = _diag(5000, 9)
    b = W.rhs_uniform(a.n, 10)
    pol = P.Policy(verify_refresh=3)
    x, info = _solve(a, b, pol)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=2000, policy=_opol(pol))
    assert info.converged and ref.converged
    assert abs(info.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    assert info.true_relres <= 1e-10
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8

"""The Chebyshev polynomial preconditioner (reading R8) on the GPU against
the oracle: the scale-and-precondition step bit for bit in every precision
pair and degree (same interval, read back from the library), and whole
AMP-PCG solves with it (trajectory tolerances as in test_gpu_solve)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")

TT = {P.FP64: torch.float64, P.FP32: torch.float32, P.FP16: torch.float16}


def _eq(gpu, ref):
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    bad = ~(gpu == ref)
    assert not bad.any(), f"{bad.sum()} mismatches: {gpu[bad][:3]} vs {ref[bad][:3]}"


CASES = {"poisson_33x33": lambda: W.poisson2d(33), "diffusion_11cubed": lambda: W.diffusion3d(11, 2.0, 3),
         "varlen": lambda: W.dense_spd_csr(W.eigs_uniform(40, 100.0), 2)}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("degree", [1, 3, 8])
@pytest.mark.parametrize("uz,ur", [(P.FP64, P.FP64), (P.FP32, P.FP64), (P.FP16, P.FP64),
                                   (P.FP32, P.FP32), (P.FP16, P.FP32)])
def test_cheb_apply_bitwise(name, degree, uz, ur):
    a = CASES[name]()
    s = P.Solver(a.rowptr, a.col, a.val, precond=P.M_CHEBYSHEV, degree=degree)
    lmin, lmax = s.interval()
    assert 0 < lmin < lmax
    rng = np.random.default_rng(degree)
    r = rng.standard_normal(a.n) * np.exp2(rng.integers(-8, 3, a.n))
    if ur == P.FP32:
        r = oracle.round32(r)
    z = torch.empty(a.n, dtype=TT[uz], device="cuda")
    omega = 2.0 ** -3
    s.precond_apply(torch.as_tensor(r, dtype=TT[ur], device="cuda"), z, uz, ur, omega)
    want = oracle.scale_cheb(a.rowptr, a.col, a.val, degree, lmin, lmax, uz, ur, omega, r)
    _eq(z.double().cpu().numpy(), want)
    s.close()


def test_gershgorin_interval_bounds_spectrum():
    a = W.diffusion3d(7, 2.0, 1)
    s = P.Solver(a.rowptr, a.col, a.val, precond=P.M_CHEBYSHEV, degree=4)
    lmin, lmax = s.interval()
    d = np.sqrt(np.diag(a.to_dense()))
    lam = np.linalg.eigvalsh(a.to_dense() / d[:, None] / d[None, :])
    assert lam[-1] <= lmax * (1 + 1e-12) and lmin == pytest.approx(lmax / 30)
    s2 = P.Solver(a.rowptr, a.col, a.val, precond=P.M_CHEBYSHEV, degree=4, lmin=0.05, lmax=2.5)
    assert s2.interval() == (0.05, 2.5)
    s.close()
    s2.close()


@pytest.mark.parametrize("variant", ["amp16", "amp64", "pcg64"])
def test_cheb_solve_matches_oracle(variant):
    a = W.diffusion3d(16, 2.0, 0)
    b = W.rhs_uniform(a.n, 1)
    s = P.Solver(a.rowptr, a.col, a.val, precond=P.M_CHEBYSHEV, degree=8)
    lmin, lmax = s.interval()
    gp = {"amp16": P.Policy(u0=P.FP16, criterion=P.CRIT_WINDOW),
          "amp64": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW),
          "pcg64": P.Policy.pcg64()}[variant]
    x, info = s.solve(torch.as_tensor(b, device="cuda"), tol=1e-10, maxit=3000, policy=gp)
    op = oracle.Policy(u0=gp.u0, criterion=gp.criterion, scale=gp.scale, fixed_uz=gp.fixed_uz,
                       fixed_ur=gp.fixed_ur)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=3000, precond=oracle.M_CHEBYSHEV,
                       cheb_degree=8, cheb_lmin=lmin, cheb_lmax=lmax, policy=op)
    assert info.converged and ref.converged
    assert abs(info.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    m = min(10, info.iters, ref.iters)
    np.testing.assert_allclose(info.relres_hist[:m], ref.relres_hist[:m], rtol=1e-6)
    assert info.true_relres <= 3e-10
    s.close()


def test_cheb_after_value_update():
    a = W.diffusion3d(9, 1.0, 2)
    a2 = W.diffusion3d(9, 1.0, 3)
    b = torch.as_tensor(W.rhs_uniform(a.n, 4), device="cuda")
    s = P.Solver(a.rowptr, a.col, a.val, precond=P.M_CHEBYSHEV, degree=5)
    s.solve(b, tol=1e-10, maxit=2000)
    s.update_values(torch.as_tensor(a2.val, device="cuda"))
    x1, i1 = s.solve(b, tol=1e-10, maxit=2000)
    s2 = P.Solver(a2.rowptr, a2.col, a2.val, precond=P.M_CHEBYSHEV, degree=5)
    x2, i2 = s2.solve(b, tol=1e-10, maxit=2000)
    assert s.interval() == s2.interval()
    assert i1.iters == i2.iters and torch.equal(x1, x2)
    s.close()
    s2.close()


def test_lagged_scale_is_refused_with_chebyshev():
    a = W.diffusion3d(8, 1.0, 0)
    s = P.Solver(a.rowptr, a.col, a.val, precond=P.M_CHEBYSHEV, degree=4)
    b = torch.as_tensor(W.rhs_uniform(a.n, 1), device="cuda")
    with pytest.raises(P.AmpcgError) as e:
        s.solve(b, tol=1e-10, maxit=100, policy=P.Policy(scale=P.SCALE_LINF_POW2_LAG))
    assert e.value.status == P.ERR_UNSUPPORTED
    s.close()

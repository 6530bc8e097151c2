"""The paper's synthetic examples rebuilt from their closed-form spectra (our
own seeds for the random orthonormal eigenvectors, which the paper does not
give), checked against the behaviour the paper reports in words.

  Sec. 2 / Sec. 5.1, motivating example: PCG run entirely in FP16 breaks down
    (z underflows, rho = 0) before 1e-10, while AMP-PCG(FP64) converges with a
    true residual close to PCG(FP64)'s.
  Sec. 5.3, linear convergence example (kappa = 10): AMP-PCG(FP16) converges
    like PCG(FP64).
  Sec. 5.4, example without large outlying eigenvalues (kappa = 1e3):
    AMP-PCG(FP64) tracks PCG(FP64); AMP-PCG(FP16) is slower.
  Sec. 5.6, limitation example (n = 10, rho = 1/4): u_z is lowered to FP32
    at iteration 9 and to FP16 at iteration 11; more than n = 10 iterations.
  Sec. 4.1: the final true residual satisfies ||b - A x|| <~ 2 tol ||b||.
Iteration counts from the paper's figures are not printed in the text, so the
checks are the qualitative ones above (parity unpinned beyond them)."""
import numpy as np

import oracle
import workloads as W

TOL = 1e-10


def _run(a, b, **kw):
    maxit = kw.pop("maxit", 2000)
    return oracle.ampcg(a.rowptr, a.col, a.val, b, tol=kw.pop("tol", TOL), maxit=maxit,
                        precond=oracle.M_NONE, policy=oracle.Policy(**kw))


def _pcg(a, b, tol=TOL):
    return oracle.pcg64(a.rowptr, a.col, a.val, b, tol=tol, maxit=2000, jacobi=False)


def test_motivating_example_fp16_breakdown_vs_ampcg():
    a = W.dense_spd_csr(W.eigs_motivating(100), seed=11)
    b = np.ones(100)
    naive16 = _run(a, b, criterion=oracle.FIXED, fixed_uz=oracle.FP16, fixed_ur=oracle.FP16,
                   scale=oracle.SCALE_NONE)
    assert not naive16.converged
    assert naive16.status in (oracle.ERR_BREAKDOWN, oracle.ERR_NONFINITE, oracle.NOT_CONVERGED)
    ref = _pcg(a, b)
    amp = _run(a, b, u0=oracle.FP64, criterion=oracle.WINDOW)
    assert ref.converged and amp.converged
    assert amp.true_relres <= 2 * TOL
    assert abs(amp.iters - ref.iters) <= max(2, 0.1 * ref.iters)
    # with dynamic scaling, FP16 z and p no longer underflow
    ds16 = _run(a, b, criterion=oracle.FIXED, fixed_uz=oracle.FP16, fixed_ur=oracle.FP64,
                scale=oracle.SCALE_LINF_POW2)
    assert ds16.converged


def test_linear_convergence_example_fp16_tracks_fp64():
    a = W.dense_spd_csr(W.eigs_uniform(100, 10.0), seed=12)
    b = W.rhs_uniform(a.n, 12)
    ref = _pcg(a, b)
    amp = _run(a, b, u0=oracle.FP16, criterion=oracle.LINEAR)
    assert amp.converged and abs(amp.iters - ref.iters) <= 2
    assert amp.switch_iter[2] > 0            # u_r was lowered to FP32 on the way
    assert amp.true_relres <= 2 * TOL


def test_no_outlying_eigenvalues_example():
    a = W.dense_spd_csr(W.eigs_uniform(100, 1000.0), seed=13)
    b = W.rhs_uniform(a.n, 13)
    ref = _pcg(a, b)
    amp64 = _run(a, b, u0=oracle.FP64, criterion=oracle.WINDOW)
    amp16 = _run(a, b, u0=oracle.FP16, criterion=oracle.WINDOW)
    assert amp64.converged and amp16.converged
    assert abs(amp64.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    assert amp16.iters > amp64.iters
    assert 0 < amp64.switch_iter[0] < amp64.switch_iter[1]
    assert amp64.true_relres <= 2 * TOL


def test_limitation_example_switch_points():
    a = W.dense_spd_csr(W.eigs_limitation(10, 0.25), seed=14)
    b = np.ones(10)
    ref = _pcg(a, b)
    amp = _run(a, b, u0=oracle.FP64, criterion=oracle.WINDOW)
    assert ref.iters > 10 and amp.iters > 10
    assert abs(amp.switch_iter[0] - 9) <= 2
    assert abs(amp.switch_iter[1] - 11) <= 2
    assert amp.switch_iter[0] < amp.switch_iter[1]

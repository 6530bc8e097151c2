"""Full-solve parity through the C ABI (ampcg_solve) against the CPU oracle.

The reductions (rho, gamma, ||r||) run in a different order on the device, so
trajectories agree to rounding, not bit for bit.  Bars:
  - FP64 PCG: iteration count +-1, residual history to 1e-8 relative over the
    first iterations, solution to 1e-10 relative of the oracle's;
  - AMP-PCG: iteration count within +-5% (and +-2), switch iterations within
    +-2, the paper's final-residual bound ||b - A x|| <~ 2 tol ||b|| (Sec. 4.1),
    and with the FP64 verify-and-replace step (reading R9) a true relative
    residual <= tol;
  - status codes for the failure modes (breakdown, non-finite input, maxit,
    invalid or non-SPD matrices)."""
import functools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")

TOL = 1e-10


def _gpu_solve(a, b, policy, tol=TOL, maxit=5000, x0=None):
    s = P.Solver(a.rowptr, a.col, a.val)
    bd = torch.as_tensor(b, device="cuda")
    xd = torch.zeros_like(bd) if x0 is None else torch.as_tensor(x0, device="cuda").clone()
    xd, info = s.solve(bd, xd, tol=tol, maxit=maxit, policy=policy)
    x = xd.cpu().numpy()
    s.close()
    return x, info


def _opol(gp: "P.Policy"):
    return oracle.Policy(u0=gp.u0, criterion=gp.criterion, d=gp.d, ell=gp.ell, C=gp.C,
                         tau_zs=gp.tau_zs, tau_zh=gp.tau_zh, scale=gp.scale, latch=gp.latch,
                         verify_refresh=gp.verify_refresh, fixed_uz=gp.fixed_uz, fixed_ur=gp.fixed_ur)


def _kappa(a):
    """2-norm condition number of A (extreme eigenvalues by Lanczos; the
    smallest through shift-invert at 0, A being SPD)."""
    m = sp.csr_matrix((a.val, a.col, a.rowptr), shape=(a.n, a.n))
    lmax = spla.eigsh(m, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(m.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return float(lmax / lmin)


@functools.lru_cache(maxsize=None)
def _problem(prob):
    if prob == "poisson64":
        a, b = W.poisson2d(64), W.rhs_uniform(4096, 0)
    else:
        a = W.diffusion3d(24, 2.0, 0)
        b = W.rhs_uniform(a.n, 1)
    return a, b, _kappa(a)


def _x_error_ok(x, ref, kappa, relres_gpu):
    """Solution error against the oracle's (reading R11): at most 1e-8, or the
    bound kappa(A) (relres_gpu + relres_oracle) that two solutions with these
    true residuals can be apart by."""
    err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    bound = max(1e-8, kappa * (relres_gpu + ref.true_relres))
    assert err <= bound, (err, bound)
    return err


def test_pcg64_config1_matches_oracle():
    a = W.poisson2d(64)
    b = W.rhs_uniform(a.n, 0)
    x, info = _gpu_solve(a, b, P.Policy.pcg64(), maxit=2000)
    ref = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=TOL, maxit=2000)
    assert info.status == P.OK and info.converged
    assert abs(info.iters - ref.iters) <= 1
    m = min(info.iters, ref.iters, 60)
    np.testing.assert_allclose(info.relres_hist[:m], ref.relres_hist[:m], rtol=1e-8)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-10
    assert info.true_relres <= TOL * 1.01
    assert all(v == (P.FP64 << 4 | P.FP64) for v in info.prec_hist)


@pytest.mark.parametrize("variant", ["amp16_linear", "amp16_window", "amp64_window", "amp_ur", "ds16",
                                     "amp16_l2", "amp64_window_l2", "amp16_lag", "amp64_window_lag",
                                     "ds16_lag"])
@pytest.mark.parametrize("prob", ["poisson64", "diffusion24"])
def test_ampcg_matches_oracle(variant, prob):
    a, b, kappa = _problem(prob)
    gp = {
        "amp16_linear": P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR),
        # omega_k = 1/||r_k|| as printed in Alg. 3 (reading R5's paper-faithful mode)
        "amp16_l2": P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, scale=P.SCALE_L2),
        "amp64_window_l2": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, scale=P.SCALE_L2),
        # lagged power of two (reading R20): the persistent kernel's three-barrier form
        "amp16_lag": P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, scale=P.SCALE_LINF_POW2_LAG),
        "amp64_window_lag": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, scale=P.SCALE_LINF_POW2_LAG),
        "ds16_lag": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64,
                             scale=P.SCALE_LINF_POW2_LAG),
        "amp16_window": P.Policy(u0=P.FP16, criterion=P.CRIT_WINDOW),
        "amp64_window": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW),
        "amp_ur": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, tau_zs=0.0, tau_zh=0.0),
        "ds16": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64),
    }[variant]
    x, info = _gpu_solve(a, b, gp)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=TOL, maxit=5000, policy=_opol(gp))
    assert info.converged and ref.converged
    assert abs(info.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    for j in range(3):
        if ref.switch_iter[j] < 0:
            assert info.switch_iter[j] < 0
        else:
            assert abs(info.switch_iter[j] - ref.switch_iter[j]) <= 2
    assert info.true_relres <= 2 * TOL * 1.5 or info.true_relres <= 2 * ref.true_relres
    _x_error_ok(x, ref, kappa, info.true_relres)
    # the early trajectory agrees closely (reductions differ only in order)
    m = min(20, info.iters, ref.iters)
    np.testing.assert_allclose(info.relres_hist[:m], ref.relres_hist[:m], rtol=1e-6)
    # precisions used agree except within 2 iterations of a switch point
    k = min(info.iters, ref.iters)
    diff = np.nonzero(info.prec_hist[:k] != ref.prec_hist[:k])[0]
    sw = [s for s in ref.switch_iter if s >= 0]
    assert all(any(abs(d - s) <= 2 for s in sw) for d in diff)


def test_first_iterations_close_to_oracle():
    a = W.diffusion3d(20, 2.0, 1)
    b = W.rhs_uniform(a.n, 3)
    for gp in (P.Policy(), P.Policy.pcg64(), P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16,
                                                       fixed_ur=P.FP32)):
        for k in (1, 2, 5):
            x, info = _gpu_solve(a, b, gp, maxit=k)
            ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=TOL, maxit=k, policy=_opol(gp))
            assert info.iters == ref.iters == k
            assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-12
            np.testing.assert_allclose(info.relres_hist, ref.relres_hist, rtol=1e-12)


@pytest.fixture(scope="module")
def bench_system():
    a = W.diffusion3d(128, 2.0, seed=0)
    b = W.rhs_uniform(a.n, seed=1)
    s = P.Solver(a.rowptr, a.col, a.val)
    yield a, b, s
    s.close()


@pytest.mark.parametrize("which", ["amp16_linear", "phase2", "pcg64", "amp16_lag", "phase2_lag"])
def test_first_iterations_at_benchmark_size(bench_system, which):
    # the 128^3 benchmark system: every warp of the persistent kernel owns 14
    # slices (two-slice trips, stage refills) and the matrix streams with the
    # L2 evict-first hint; x and the residual history after 1, 2 and 5
    # iterations agree with the oracle to rounding
    a, b, s = bench_system
    gp = {"amp16_linear": P.Policy(verify_refresh=3),
          "phase2": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32),
          "pcg64": P.Policy.pcg64(),
          "amp16_lag": P.Policy(verify_refresh=3, scale=P.SCALE_LINF_POW2_LAG),
          "phase2_lag": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32,
                                 scale=P.SCALE_LINF_POW2_LAG)}[which]
    assert s.layout()["stream_hint"] == 1
    bd = torch.as_tensor(b, device="cuda")
    for k in (1, 2, 5):
        x, info = s.solve(bd, tol=TOL, maxit=k, policy=gp)
        ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=TOL, maxit=k, policy=_opol(gp))
        assert info.iters == ref.iters == k
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) < 1e-12
        np.testing.assert_allclose(info.relres_hist, ref.relres_hist, rtol=1e-12)
        assert np.array_equal(info.prec_hist, ref.prec_hist)


def test_refresh_gives_fp64_verified_tolerance():
    a = W.diffusion3d(32, 2.0, 0)
    b = W.rhs_uniform(a.n, 1)
    gp = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3)
    x, info = _gpu_solve(a, b, gp)
    assert info.converged
    assert info.true_relres <= TOL or info.refreshes == 3
    r = oracle.residual64(a.rowptr, a.col, a.val, b, x)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - info.true_relres) <= 1e-3 * info.true_relres


def test_host_and_device_buffers_agree():
    a = W.poisson2d(40)
    b = W.rhs_uniform(a.n, 2)
    s = P.Solver(a.rowptr, a.col, a.val)
    xh, ih = s.solve(b.copy(), np.zeros(a.n), tol=TOL, maxit=3000)
    xd, idv = s.solve(torch.as_tensor(b, device="cuda"), tol=TOL, maxit=3000)
    s.close()
    assert ih.iters == idv.iters
    assert np.array_equal(xh, xd.cpu().numpy())      # deterministic reductions


def test_repeated_solves_are_deterministic():
    a = W.diffusion3d(16, 2.0, 2)
    b = torch.as_tensor(W.rhs_uniform(a.n, 4), device="cuda")
    s = P.Solver(a.rowptr, a.col, a.val)
    outs = [s.solve(b, tol=TOL, maxit=3000) for _ in range(3)]
    s.close()
    for x, info in outs[1:]:
        assert info.iters == outs[0][1].iters
        assert torch.equal(x, outs[0][0])


@pytest.mark.parametrize("kind", ["amp16", "amp16_lag", "amp64_window", "amp64_window_lag", "cheb",
                                  "wide_jacobi", "wide_jacobi_lag", "pcg64", "bsr_cheb", "bsr_jacobi"])
def test_loop_graph_equals_kernel_by_kernel(kind):
    # the loop graph (SWITCH per precision change, inner loop of chunks) runs
    # the same kernels in the same order as the host-driven launches, for any
    # chunk length, including chunks that straddle a precision change or the
    # stop: the persistent iteration kernel (Jacobi, narrow slices), the
    # Chebyshev sequence, and the sequence with the cooperative precondition
    # + direction kernel (Jacobi, slices wider than 8)
    if kind.startswith("wide_jacobi"):
        a = W.elasticity_q1(7, seed=2).to_csr()
    else:
        a = W.diffusion3d(20, 2.0, 6)
    if kind.startswith("bsr"):
        a = W.elasticity_q1(7, seed=2)   # 3 x 3 blocks: the block-row kernels
    b = torch.as_tensor(W.rhs_uniform(a.n if not kind.startswith("bsr") else a.nb * 3, 8), device="cuda")
    kw = dict(precond=P.M_CHEBYSHEV, degree=4) if kind in ("cheb", "bsr_cheb") else {}
    if kind.startswith("bsr"):
        s = P.Solver.from_bsr(a.browptr, a.bcol, a.bval.reshape(-1), 3, **kw)
        assert s.layout()["block3"] == 1
    else:
        s = P.Solver(a.rowptr, a.col, a.val, **kw)
    lag = P.SCALE_LINF_POW2_LAG
    pol = {"amp64_window": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, verify_refresh=3),
           "amp64_window_lag": P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, verify_refresh=3, scale=lag),
           "amp16_lag": P.Policy(verify_refresh=3, scale=lag),
           "wide_jacobi_lag": P.Policy(verify_refresh=3, scale=lag),
           "pcg64": P.Policy.pcg64(verify_refresh=3)}.get(kind, P.Policy(verify_refresh=3))
    x0, i0 = s.solve(b, tol=TOL, maxit=5000, policy=pol, timed=True)
    assert i0.converged
    assert kind in ("cheb", "wide_jacobi", "wide_jacobi_lag", "pcg64", "bsr_cheb", "bsr_jacobi") or \
        any(k >= 0 for k in i0.switch_iter)
    for chunk in (1, 3, 16, 64):
        pol.graph_chunk = chunk
        x1, i1 = s.solve(b, tol=TOL, maxit=5000, policy=pol)
        assert i1.iters == i0.iters and i1.refreshes == i0.refreshes
        assert list(i1.switch_iter) == list(i0.switch_iter)
        assert np.array_equal(i1.prec_hist, i0.prec_hist)
        assert torch.equal(x1, x0)
    s.close()


@pytest.mark.parametrize("variant", ["pcg64", "amp16"])
def test_wide_rows_jacobi_matches_oracle(variant):
    # Jacobi on rows wider than the staged SpMV's slices (Q1 elasticity, ~81
    # entries per row): the kernel sequence with the cooperative precondition
    # + direction kernel, against the oracle
    a = W.elasticity_q1(7, seed=3).to_csr()
    b = W.rhs_uniform(a.n, 4)
    gp = P.Policy.pcg64() if variant == "pcg64" else P.Policy(verify_refresh=3)
    x, info = _gpu_solve(a, b, gp, tol=1e-8)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-8, maxit=5000, policy=_opol(gp))
    assert info.converged and ref.converged
    if variant == "pcg64":
        assert abs(info.iters - ref.iters) <= 1
    else:
        assert abs(info.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    t = oracle.residual64(a.rowptr, a.col, a.val, b, x)
    assert np.linalg.norm(t) / np.linalg.norm(b) <= (1.01e-8 if variant == "pcg64" else 1e-8)


def test_loop_graph_launch_count():
    # one precision pair, no replacement: k_init, one outer body (k_phase,
    # k_loop_ctl), ceil(iters / chunk) chunks, each one k_loop launch (Jacobi,
    # narrow slices: the whole chunk in one cooperative launch) plus
    # k_chunk_ctl, and the true residual
    a = W.diffusion3d(16, 1.0, 3)
    b = torch.as_tensor(W.rhs_uniform(a.n, 2), device="cuda")
    s = P.Solver(a.rowptr, a.col, a.val)
    for chunk in (1, 7, 16):
        pol = P.Policy.pcg64(graph_chunk=chunk)
        _, info = s.solve(b, tol=TOL, maxit=5000, policy=pol)
        chunks = -(-info.iters // chunk)
        assert info.kernel_launches == 1 + 2 + chunks * 2 + 1
    s.close()


def test_warm_start_and_zero_rhs():
    a = W.poisson2d(32)
    b = W.rhs_uniform(a.n, 5)
    x, info = _gpu_solve(a, b, P.Policy.pcg64())
    x2, info2 = _gpu_solve(a, b, P.Policy.pcg64(), x0=x)
    assert info2.iters <= 2
    x3, info3 = _gpu_solve(a, np.zeros(a.n), P.Policy())
    assert info3.iters == 0 and info3.status == P.OK and not np.any(x3)


def test_status_codes():
    a = W.poisson2d(8)
    b = W.rhs_uniform(a.n, 0)
    # maxit reached
    x, info = _gpu_solve(a, b, P.Policy(), maxit=3)
    assert info.status == P.NOT_CONVERGED and info.iters == 3 and not info.converged
    # non-finite right-hand side
    bn = b.copy()
    bn[5] = np.nan
    x, info = _gpu_solve(a, bn, P.Policy())
    assert info.status == P.ERR_NONFINITE
    # indefinite with a positive diagonal: gamma <= 0 at some step
    ind = W.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
                np.array([1.0, 3.0, 3.0, 1.0]), {})
    x, info = _gpu_solve(ind, np.array([1.0, -1.0]), P.Policy.pcg64())
    ref = oracle.ampcg(ind.rowptr, ind.col, ind.val, np.array([1.0, -1.0]), policy=oracle.Policy(
        criterion=oracle.FIXED, scale=oracle.SCALE_NONE))
    assert info.status == P.ERR_BREAKDOWN == ref.status
    # create-time validation
    with pytest.raises(P.AmpcgError) as e:
        P.Solver(a.rowptr, a.col[::-1].copy(), a.val)
    assert e.value.status == P.ERR_INVALID_ARG
    neg = a.val.copy()
    neg[0] = -4.0
    with pytest.raises(P.AmpcgError) as e:
        P.Solver(a.rowptr, a.col, neg)
    assert e.value.status == P.ERR_NOT_SPD
    bad = a.col.copy()
    bad[3] = a.n + 5
    with pytest.raises(P.AmpcgError) as e:
        P.Solver(a.rowptr, bad, a.val)
    assert e.value.status == P.ERR_INVALID_ARG


def _growth_system():
    """The 2 x 2 system on which one Jacobi-PCG step takes the residual norm
    from 1 to 8.9e4 (draw 13211 of the seeded family of the oracle's pin)."""
    rng = np.random.default_rng(1)
    for _ in range(13212):
        th = rng.uniform(0, np.pi)
        ev = np.exp(rng.uniform(-12, 2, 2))
        sc = np.exp(rng.uniform(-6, 6, 2))
        b = rng.standard_normal(2) * np.exp(rng.uniform(-6, 0, 2))
    q = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    m = q @ np.diag(ev) @ q.T
    m = (m + m.T) / 2 * np.outer(sc, sc)
    return W.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), m.ravel().copy(), {}), b


@pytest.mark.parametrize("timed", [False, True])
def test_lagged_scale_retry_after_overflow(timed):
    # y_1 = omega_1 r_1 with omega_1 from max|r_0| overflows binary16: the
    # fused update's rho_1 is non-finite, the head step forms y_1, z_1, rho_1
    # again with the exact power of two (reading R20); the run then equals the
    # non-lagged one bit for bit, and the oracle's to rounding
    a, b = _growth_system()
    s = P.Solver(a.rowptr, a.col, a.val)
    bd = torch.as_tensor(b, device="cuda")
    base = dict(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64)
    xl, il = s.solve(bd, tol=1e-30, maxit=2, policy=P.Policy(scale=P.SCALE_LINF_POW2_LAG, **base), timed=timed)
    xe, ie = s.solve(bd, tol=1e-30, maxit=2, policy=P.Policy(scale=P.SCALE_LINF_POW2, **base), timed=timed)
    s.close()
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-30, maxit=2, policy=oracle.Policy(
        scale=oracle.SCALE_LINF_POW2_LAG, criterion=oracle.FIXED, fixed_uz=oracle.FP16, fixed_ur=oracle.FP64))
    assert ref.scale_retries == 1
    assert il.status == ie.status == P.NOT_CONVERGED and il.iters == ie.iters == 2
    assert torch.equal(xl, xe) and np.array_equal(il.relres_hist, ie.relres_hist)
    np.testing.assert_allclose(il.relres_hist, ref.relres_hist, rtol=1e-12)
    np.testing.assert_allclose(xl.cpu().numpy(), ref.x, rtol=1e-12)

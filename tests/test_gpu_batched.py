"""Batched solves (ampcg_solve_batched).

Small Jacobi/unpreconditioned systems run in the persistent kernel (one block
per system, block-level reductions): each system is checked against the
oracle's run of Alg. 3 on the same input (iteration count within 5% or 3,
FP64-verified residual at tol, precision switches near the oracle's), and a
system's result does not depend on the rest of the batch (bitwise).  Larger
or Chebyshev systems run as independent device loops, bitwise equal to
single solves."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


def _dev(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")


def _solve_batched(solvers, rhs, pol, tol=1e-10, maxit=5000):
    bs = [_dev(b) for b in rhs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = P.solve_batched(solvers, bs, xs, tol=tol, maxit=maxit, policy=pol)
    return xs, infos


@pytest.mark.parametrize("kind", ["amp16", "amp16_lag", "amp64_window", "fp64"])
def test_persistent_path_matches_oracle(kind):
    mats, rhs = W.batch_2d(10, seed=3, smin=16, smax=90)
    gp, op = {
        "amp16": (P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3),
                  oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, verify_refresh=3)),
        # lagged power-of-two scale (reading R20)
        "amp16_lag": (P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3,
                               scale=P.SCALE_LINF_POW2_LAG),
                      oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, verify_refresh=3,
                                    scale=oracle.SCALE_LINF_POW2_LAG)),
        "amp64_window": (P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, verify_refresh=3),
                         oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW, verify_refresh=3)),
        "fp64": (P.Policy.pcg64(), oracle.Policy(criterion=oracle.FIXED, fixed_uz=oracle.FP64,
                                                 fixed_ur=oracle.FP64)),
    }[kind]
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs, infos = _solve_batched(solvers, rhs, gp)
    for m, b, x, info in zip(mats, rhs, xs, infos):
        ref = oracle.ampcg(m.rowptr, m.col, m.val, b, tol=1e-10, maxit=5000, policy=op)
        assert info.converged and ref.converged
        assert abs(info.iters - ref.iters) <= max(3, 0.05 * ref.iters)
        t = oracle.residual64(m.rowptr, m.col, m.val, b, x.cpu().numpy())
        relres = np.linalg.norm(t) / np.linalg.norm(b)
        assert abs(relres - info.true_relres) <= 1e-3 * relres
        if kind == "fp64":
            assert relres <= 1.01e-10 and info.iters == ref.iters
        else:
            assert relres <= 1e-10
        for g, o in zip(info.switch_iter, ref.switch_iter):
            assert (g < 0) == (o < 0) and abs(g - o) <= 3
    assert len({i.iters for i in infos}) > 1      # systems stop independently
    for s in solvers:
        s.close()


def test_persistent_result_independent_of_batch():
    mats, rhs = W.batch_2d(6, seed=5, smin=20, smax=70)
    pol = P.Policy(verify_refresh=3)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs, infos = _solve_batched(solvers, rhs, pol)
    for i in (0, 3, 5):
        x1, i1 = _solve_batched([solvers[i]], [rhs[i]], pol)
        assert torch.equal(x1[0], xs[i]) and i1[0].iters == infos[i].iters
    for s in solvers:
        s.close()


def test_persistent_histories_and_host_arrays():
    mats, rhs = W.batch_2d(3, seed=4, smin=10, smax=20)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs = [np.zeros(m.n) for m in mats]
    infos = P.solve_batched(solvers, [r.copy() for r in rhs], xs, tol=1e-10, maxit=2000,
                            policy=P.Policy(verify_refresh=3), history=True)
    for x, m, r, info in zip(xs, mats, rhs, infos):
        t = oracle.residual64(m.rowptr, m.col, m.val, r, x)
        assert np.linalg.norm(t) / np.linalg.norm(r) < 1e-10
        h = info.relres_hist
        assert h.shape == (info.iters + 1,) and h[0] == pytest.approx(1.0) and h[-1] <= 1e-10
        assert info.prec_hist.shape == (info.iters,)
        assert (info.prec_hist[-1] & 0xF) == P.FP32
    with pytest.raises(P.AmpcgError):
        P.solve_batched([solvers[0], solvers[0]], rhs[:1] * 2, xs[:1] * 2)
    for s in solvers:
        s.close()


def test_stream_path_equals_single_solves():
    # Chebyshev contexts are not taken by the persistent kernel: each system
    # runs the single-system device loop on a library stream
    mats, rhs = W.batch_2d(5, seed=6, smin=24, smax=64)
    pol = P.Policy(verify_refresh=3)
    solvers = [P.Solver(m.rowptr, m.col, m.val, precond=P.M_CHEBYSHEV, degree=4) for m in mats]
    xs, infos = _solve_batched(solvers, rhs, pol)
    for s, b, x, info in zip(solvers, rhs, xs, infos):
        x1, i1 = s.solve(_dev(b), tol=1e-10, maxit=5000, policy=pol)
        assert info.converged and info.iters == i1.iters
        assert torch.equal(x, x1)
    for s in solvers:
        s.close()


def test_mixed_batch():
    mats, rhs = W.batch_2d(4, seed=7, smin=24, smax=48)
    big = W.diffusion3d(52, 1.0, 3)            # 140,608 rows: above the persistent kernel's limit
    mats.append(big)
    rhs.append(W.rhs_uniform(big.n, 9))
    pol = P.Policy(verify_refresh=3)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs, infos = _solve_batched(solvers, rhs, pol, maxit=20000)
    for m, b, x, info in zip(mats, rhs, xs, infos):
        t = oracle.residual64(m.rowptr, m.col, m.val, b, x.cpu().numpy())
        assert info.converged and np.linalg.norm(t) / np.linalg.norm(b) <= 1e-10
    xb, ib = solvers[-1].solve(_dev(rhs[-1]), tol=1e-10, maxit=20000, policy=pol)
    assert torch.equal(xb, xs[-1]) and ib.iters == infos[-1].iters
    for s in solvers:
        s.close()


def test_larger_systems_match_oracle_and_are_independent():
    # the batch's larger sizes (17K-33K rows) next to a small one
    sides = [130, 150, 181, 40]
    mats = [W.diffusion2d_cells(s, 2000 + i) for i, s in enumerate(sides)]
    rhs = [W.rhs_uniform(m.n, 30 + i) for i, m in enumerate(mats)]
    gp = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3)
    op = oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, verify_refresh=3)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs, infos = _solve_batched(solvers, rhs, gp)
    for m, b, x, info in zip(mats, rhs, xs, infos):
        ref = oracle.ampcg(m.rowptr, m.col, m.val, b, tol=1e-10, maxit=5000, policy=op)
        assert info.converged and ref.converged
        assert abs(info.iters - ref.iters) <= max(3, 0.05 * ref.iters)
        t = oracle.residual64(m.rowptr, m.col, m.val, b, x.cpu().numpy())
        assert np.linalg.norm(t) / np.linalg.norm(b) <= 1e-10
    x1, i1 = _solve_batched([solvers[1]], [rhs[1]], gp)
    assert torch.equal(x1[0], xs[1]) and i1[0].iters == infos[1].iters
    for s in solvers:
        s.close()


def test_batched_statuses():
    # per-system statuses in the persistent kernel: converged, zero right-hand
    # side (done at iteration 0), maxit reached, non-finite input
    mats, rhs = W.batch_2d(4, seed=8, smin=12, smax=24)
    rhs[1] = np.zeros_like(rhs[1])
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs, infos = _solve_batched(solvers, rhs, P.Policy(verify_refresh=3))
    assert infos[0].status == P.OK and infos[1].status == P.OK and infos[1].iters == 0
    assert not torch.any(xs[1])
    xs, infos = _solve_batched(solvers[:1], rhs[:1], P.Policy(), maxit=3)
    assert infos[0].status == P.NOT_CONVERGED and infos[0].iters == 3
    bad = rhs[2].copy()
    bad[4] = np.nan
    xs, infos = _solve_batched([solvers[2], solvers[3]], [bad, rhs[3]], P.Policy())
    assert infos[0].status == P.ERR_NONFINITE and infos[1].status == P.OK
    for s in solvers:
        s.close()


@pytest.mark.parametrize("block", [1024, 512])
@pytest.mark.parametrize("kind", ["amp16_lag", "fp64"])
def test_each_block_size_matches_oracle(block, kind):
    # the batched kernel's block sizes the tuner chooses between: both run
    # Alg. 3 per system (reductions over other thread counts), each system
    # meets the parity bars against the oracle
    mats, rhs = W.batch_2d(12, seed=7, smin=16, smax=100)
    gp, op = {
        "amp16_lag": (P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3, scale=P.SCALE_LINF_POW2_LAG),
                      oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, verify_refresh=3,
                                    scale=oracle.SCALE_LINF_POW2_LAG)),
        "fp64": (P.Policy.pcg64(), oracle.Policy(criterion=oracle.FIXED, fixed_uz=oracle.FP64,
                                                 fixed_ur=oracle.FP64, scale=oracle.SCALE_NONE)),
    }[kind]
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    P.set_batch_block(solvers, block)
    xs, infos = _solve_batched(solvers, rhs, gp)
    for m, b, x, info in zip(mats, rhs, xs, infos):
        ref = oracle.ampcg(m.rowptr, m.col, m.val, b, tol=1e-10, maxit=5000, policy=op)
        assert info.converged and ref.converged
        if kind == "fp64":
            assert abs(info.iters - ref.iters) <= 1
        else:
            assert abs(info.iters - ref.iters) <= max(3, 0.05 * ref.iters)
        t = oracle.residual64(m.rowptr, m.col, m.val, b, x.cpu().numpy())
        assert np.linalg.norm(t) / np.linalg.norm(b) <= (1.01e-10 if kind == "fp64" else 1e-10)
    for s in solvers:
        s.close()


def test_tune_batched_stores_the_faster_block():
    mats, rhs = W.batch_2d(40, seed=9, smin=16, smax=128)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    t = P.tune_batched(solvers, iters=10, policy=P.Policy(scale=P.SCALE_LINF_POW2_LAG))
    assert set(t["ms"]) == {1024, 512} and all(v > 0 for v in t["ms"].values())
    assert t["chosen"] == min(t["ms"], key=t["ms"].get)
    xs, infos = _solve_batched(solvers, rhs, P.Policy(verify_refresh=3, scale=P.SCALE_LINF_POW2_LAG))
    assert all(i.converged and i.true_relres <= 1e-10 for i in infos)
    for s in solvers:
        s.close()

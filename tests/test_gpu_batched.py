"""Batched solves (ampcg_solve_batched): every system's result equals its
single solve bit for bit (same kernels, deterministic reductions), systems
stop independently, and the results match the oracle per system."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


def test_batched_equals_single_solves():
    mats, rhs = W.batch_2d(12, seed=3, smin=16, smax=90)
    pol = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    bs = [torch.as_tensor(b, device="cuda") for b in rhs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = P.solve_batched(solvers, bs, xs, tol=1e-10, maxit=5000, policy=pol)
    for s, b, x, info, m, bh in zip(solvers, bs, xs, infos, mats, rhs):
        x1, i1 = s.solve(b, tol=1e-10, maxit=5000, policy=pol)
        assert info.converged and info.iters == i1.iters
        assert torch.equal(x, x1)
        ref = oracle.ampcg(m.rowptr, m.col, m.val, bh, tol=1e-10, maxit=5000,
                           policy=oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR))
        assert abs(info.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    iters = [i.iters for i in infos]
    assert len(set(iters)) > 1           # uneven systems stop at different iterations
    for s in solvers:
        s.close()


def test_batched_host_arrays_and_errors():
    mats, rhs = W.batch_2d(3, seed=4, smin=10, smax=20)
    solvers = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
    xs = [np.zeros(m.n) for m in mats]
    infos = P.solve_batched(solvers, [r.copy() for r in rhs], xs, tol=1e-10, maxit=2000)
    for x, m, r in zip(xs, mats, rhs):
        t = oracle.residual64(m.rowptr, m.col, m.val, r, x)
        assert np.linalg.norm(t) / np.linalg.norm(r) < 3e-10
    with pytest.raises(P.AmpcgError):
        P.solve_batched([solvers[0], solvers[0]], rhs[:1] * 2, xs[:1] * 2)
    for s in solvers:
        s.close()

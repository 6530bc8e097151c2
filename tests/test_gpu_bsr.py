"""Block CSR input (ampcg_create_bsr): the device expansion gives the same
scalar system as the expanded CSR (solves identical bit for bit), and AMP-PCG
with the FP16 Chebyshev preconditioner on Q1 elasticity matches the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


@pytest.mark.parametrize("precond,degree", [(P.M_JACOBI, 0), (P.M_CHEBYSHEV, 8)])
def test_bsr_equals_expanded_csr(precond, degree):
    B = W.elasticity_q1(7, seed=2)
    A = B.to_csr()
    b = torch.as_tensor(W.rhs_uniform(A.n, 1), device="cuda")
    sb = P.Solver.from_bsr(B.browptr, B.bcol, B.bval.reshape(-1), 3, precond=precond, degree=degree)
    sc = P.Solver(A.rowptr, A.col, A.val, precond=precond, degree=degree)
    pol = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR)
    xb, ib = sb.solve(b, tol=1e-8, maxit=5000, policy=pol)
    xc, ic = sc.solve(b, tol=1e-8, maxit=5000, policy=pol)
    assert ib.converged and ib.iters == ic.iters and torch.equal(xb, xc)
    q = torch.empty(A.n, dtype=torch.float64, device="cuda")
    p = np.random.default_rng(0).standard_normal(A.n)
    sb.spmv(torch.as_tensor(p, device="cuda"), q, P.FP64)
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy(), oracle.spmv(A.rowptr, A.col, A.val, oracle.FP64, p))
    sb.close()
    sc.close()


def test_elasticity_chebyshev_fp16_matches_oracle():
    B = W.elasticity_q1(8, seed=0)
    A = B.to_csr()
    b = W.rhs_uniform(A.n, 1)
    s = P.Solver.from_bsr(B.browptr, B.bcol, B.bval.reshape(-1), 3, precond=P.M_CHEBYSHEV, degree=8)
    lmin, lmax = s.interval()
    pol = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR)
    x, info = s.solve(torch.as_tensor(b, device="cuda"), tol=1e-8, maxit=5000, policy=pol)
    ref = oracle.ampcg(A.rowptr, A.col, A.val, b, tol=1e-8, maxit=5000, precond=oracle.M_CHEBYSHEV,
                       cheb_degree=8, cheb_lmin=lmin, cheb_lmax=lmax,
                       policy=oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR))
    assert info.converged and ref.converged
    assert abs(info.iters - ref.iters) <= max(2, 0.05 * ref.iters)
    assert info.true_relres <= 3e-8
    s.close()


def test_bsr_invalid_input():
    B = W.elasticity_q1(4, seed=0)
    bad = B.browptr.copy()
    bad[-1] += 1
    with pytest.raises(P.AmpcgError) as e:
        P.Solver.from_bsr(bad, B.bcol, B.bval.reshape(-1), 3)
    assert e.value.status == P.ERR_INVALID_ARG

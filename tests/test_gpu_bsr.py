"""Block CSR input (ampcg_create_bsr) and the 3 x 3 block-row kernels.

A context created from 3 x 3 block CSR with wide rows keeps a block-row layout
that the Chebyshev steps and the SpMV of the kernel sequence use (one thread
per block row, each block's 3 operands gathered once for its 3 rows).  The
products are accumulated in the same order as on the scalar layout, so:
  - q = A p with the block layout is bitwise the oracle's SpMV on the expanded
    matrix (FP64 and FP32), also after a value update;
  - the Chebyshev preconditioner applied through the block layout is bitwise
    the scalar layout's, and the oracle's (reading R8);
  - whole solves agree with the expanded-CSR context and the oracle to the
    parity bars (the inner product gamma is summed over another partition)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")

TT = {P.FP64: torch.float64, P.FP32: torch.float32, P.FP16: torch.float16}


def _bsr(n, seed, precond=P.M_JACOBI, degree=0):
    B = W.elasticity_q1(n, seed=seed)
    return B, B.to_csr(), P.Solver.from_bsr(B.browptr, B.bcol, B.bval.reshape(-1), 3, precond=precond,
                                            degree=degree)


@pytest.mark.parametrize("n", [7, 12])
def test_block_spmv_bitwise(n):
    B, A, s = _bsr(n, seed=1)
    assert s.layout()["block3"] == 1
    rng = np.random.default_rng(n)
    for prec, aval in ((P.FP64, A.val), (P.FP32, oracle.round32(A.val))):
        p = oracle.round_to(prec, rng.standard_normal(A.n))
        q = torch.empty(A.n, dtype=TT[prec], device="cuda")
        s.spmv_block(torch.as_tensor(p, device="cuda").to(TT[prec]), q, prec)
        torch.cuda.synchronize()
        ref = oracle.spmv(A.rowptr, A.col, aval, prec, p)
        assert np.array_equal(q.double().cpu().numpy(), ref)
    # new values on the same pattern: the block layout follows
    s.update_values(2.0 * A.val)
    p = rng.standard_normal(A.n)
    q = torch.empty(A.n, dtype=torch.float64, device="cuda")
    s.spmv_block(torch.as_tensor(p, device="cuda"), q, P.FP64)
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy(), oracle.spmv(A.rowptr, A.col, 2.0 * A.val, oracle.FP64, p))
    s.close()


def test_narrow_block_matrix_keeps_the_scalar_layout():
    # 3 x 3 blocks in rows of at most 8 entries run the persistent kernel
    # (staged SpMV); no block layout is built
    nb = 40
    browptr = np.arange(nb + 1, dtype=np.int32)
    bcol = np.arange(nb, dtype=np.int32)
    bval = np.tile(np.eye(3) * 4.0, (nb, 1, 1))
    s = P.Solver.from_bsr(browptr, bcol, bval.reshape(-1), 3)
    assert s.layout()["block3"] == 0
    s.close()


@pytest.mark.parametrize("uz,ur", [(P.FP64, P.FP64), (P.FP32, P.FP64), (P.FP16, P.FP64), (P.FP16, P.FP32)])
def test_block_chebyshev_apply_bitwise(uz, ur):
    B, A, sb = _bsr(9, seed=3, precond=P.M_CHEBYSHEV, degree=8)
    sc = P.Solver(A.rowptr, A.col, A.val, precond=P.M_CHEBYSHEV, degree=8)
    assert sb.layout()["block3"] == 1 and sc.layout()["block3"] == 0
    lmin, lmax = sb.interval()
    assert (lmin, lmax) == sc.interval()
    r = oracle.round_to(ur, np.random.default_rng(5).standard_normal(A.n))
    omega = 2.0 ** -2
    zs = []
    for s in (sb, sc):
        z = torch.empty(A.n, dtype=TT[uz], device="cuda")
        s.precond_apply(torch.as_tensor(r, device="cuda").to(TT[ur]), z, uz, ur, omega)
        torch.cuda.synchronize()
        zs.append(z.double().cpu().numpy())
    ref = oracle.scale_cheb(A.rowptr, A.col, A.val, 8, lmin, lmax, uz, ur, omega, r)
    assert np.array_equal(zs[0], zs[1])
    assert np.array_equal(zs[0], ref)
    sb.close()
    sc.close()


@pytest.mark.parametrize("precond,degree", [(P.M_JACOBI, 0), (P.M_CHEBYSHEV, 8)])
@pytest.mark.parametrize("variant", ["amp16", "pcg64"])
def test_bsr_solve_matches_expanded_csr_and_oracle(precond, degree, variant):
    B, A, sb = _bsr(7, seed=2, precond=precond, degree=degree)
    sc = P.Solver(A.rowptr, A.col, A.val, precond=precond, degree=degree)
    b = W.rhs_uniform(A.n, 1)
    bd = torch.as_tensor(b, device="cuda")
    pol = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3) if variant == "amp16" else P.Policy.pcg64()
    xb, ib = sb.solve(bd, tol=1e-8, maxit=5000, policy=pol)
    xc, ic = sc.solve(bd, tol=1e-8, maxit=5000, policy=pol)
    lmin, lmax = sb.interval() if precond == P.M_CHEBYSHEV else (0.0, 0.0)
    ref = oracle.ampcg(A.rowptr, A.col, A.val, b, tol=1e-8, maxit=5000, precond=precond, cheb_degree=degree,
                       cheb_lmin=lmin, cheb_lmax=lmax,
                       policy=oracle.Policy(u0=pol.u0, criterion=pol.criterion, scale=pol.scale,
                                            verify_refresh=pol.verify_refresh, fixed_uz=pol.fixed_uz,
                                            fixed_ur=pol.fixed_ur))
    assert ib.converged and ic.converged and ref.converged
    tol_it = 1 if variant == "pcg64" else max(2, 0.05 * ref.iters)
    assert abs(ib.iters - ref.iters) <= tol_it and abs(ib.iters - ic.iters) <= tol_it
    xbn, xcn = xb.cpu().numpy(), xc.cpu().numpy()
    t = oracle.residual64(A.rowptr, A.col, A.val, b, xbn)
    assert np.linalg.norm(t) / np.linalg.norm(b) <= 1.01e-8
    assert np.linalg.norm(xbn - ref.x) / np.linalg.norm(ref.x) <= 1e-5
    sb.close()
    sc.close()


def test_elasticity_chebyshev_fp16_matches_oracle():
    B, A, s = _bsr(8, seed=0, precond=P.M_CHEBYSHEV, degree=8)
    b = W.rhs_uniform(A.n, 1)
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

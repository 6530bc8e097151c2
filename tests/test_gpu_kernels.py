"""Kernel-level parity through the C ABI: the device's SpMV of Alg. 3, its
FP64 initial residual, the scale-and-precondition step and the precision
selector (Eq. precision_selector with Eq. eta_k / linear criterion) against
the CPU oracle on the same seeded inputs.  All of these are elementwise or
scalar computations with a fixed operation order, so the bar is bit-for-bit
equality (IEEE equality; the sign of an exact zero may differ)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


def _csr_from_dense(a):
    n = a.shape[0]
    rows, cols = np.nonzero(a)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    return W.CSR(n, np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32), a[rows, cols], {})


def _varlen(n, seed):
    """SPD, rows of 1..20 entries (some rows hold only the diagonal)."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    for i in range(n):
        k = rng.integers(0, 10)
        js = rng.choice(n, size=k, replace=False)
        for j in js:
            if j != i:
                v = -rng.uniform(0.1, 1.0)
                a[i, j] = a[j, i] = v
    a[np.diag_indices(n)] = np.abs(a).sum(axis=1) + rng.uniform(0.5, 2.0, n)
    return _csr_from_dense(a)


def _long_range(n):
    """1D Laplacian plus a (0, n-1) coupling: column offsets exceed int16."""
    a = W.poisson2d(n, 1)
    rp, col, val = list(a.rowptr), list(a.col), list(a.val)
    dense_rows = []
    for i in range(n):
        lo, hi = rp[i], rp[i + 1]
        entries = dict(zip(col[lo:hi], val[lo:hi]))
        if i == 0:
            entries[n - 1] = -0.5
        if i == n - 1:
            entries[0] = -0.5
        entries[i] = entries[i] + 0.5 if i in (0, n - 1) else entries[i]
        dense_rows.append(sorted(entries.items()))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in dense_rows])
    cols = np.array([c for r in dense_rows for c, _ in r], dtype=np.int32)
    vals = np.array([v for r in dense_rows for _, v in r])
    return W.CSR(n, rowptr, cols, vals, {})


CASES = {
    "n1": lambda: _csr_from_dense(np.array([[3.0]])),
    "n7_1d": lambda: W.poisson2d(7, 1),
    "n33_1d": lambda: W.poisson2d(33, 1),
    "poisson_37x37": lambda: W.poisson2d(37),
    "diffusion_17cubed": lambda: W.diffusion3d(17, 2.0, 0),
    "dense_101": lambda: W.dense_spd_csr(W.eigs_uniform(100, 10.0), 3),
    "varlen_300": lambda: _varlen(300, 5),
    "long_range_40000": lambda: _long_range(40000),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    a = CASES[request.param]()
    s = P.Solver(a.rowptr, a.col, a.val)
    yield a, s
    s.close()


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda")


def _eq(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    bad = ~((gpu == ref) | (np.isnan(gpu) & np.isnan(ref)))
    assert not bad.any(), f"{bad.sum()} mismatches, first at {np.argmax(bad)}: {gpu[bad][:3]} vs {ref[bad][:3]}"


def test_spmv_fp64_fp32_bitwise(case):
    a, s = case
    rng = np.random.default_rng(1)
    p = rng.standard_normal(a.n)
    q = torch.empty(a.n, dtype=torch.float64, device="cuda")
    s.spmv(_dev(p), q, P.FP64)
    torch.cuda.synchronize()
    _eq(q.cpu().numpy(), oracle.spmv(a.rowptr, a.col, a.val, oracle.FP64, p))
    p32 = oracle.round32(p)
    q32 = torch.empty(a.n, dtype=torch.float32, device="cuda")
    s.spmv(_dev(p32, torch.float32), q32, P.FP32)
    torch.cuda.synchronize()
    _eq(q32.cpu().numpy(), oracle.spmv(a.rowptr, a.col, oracle.round32(a.val), oracle.FP32, p32))


def test_residual_fp64_bitwise(case):
    a, s = case
    rng = np.random.default_rng(2)
    b, x = rng.uniform(-1, 1, a.n), rng.standard_normal(a.n)
    r = torch.empty(a.n, dtype=torch.float64, device="cuda")
    s.residual(_dev(b), _dev(x), r)
    torch.cuda.synchronize()
    _eq(r.cpu().numpy(), oracle.residual64(a.rowptr, a.col, a.val, b, x))


TORCH_T = {P.FP64: torch.float64, P.FP32: torch.float32, P.FP16: torch.float16}


@pytest.mark.parametrize("uz", [P.FP64, P.FP32, P.FP16])
@pytest.mark.parametrize("ur", [P.FP64, P.FP32])
@pytest.mark.parametrize("omega", [2.0 ** -7, 1.0, 0.3, 2.0 ** 9])
def test_scale_precond_bitwise(case, uz, ur, omega):
    a, s = case
    rng = np.random.default_rng(3)
    r = rng.standard_normal(a.n) * np.exp2(rng.integers(-20, 3, a.n))
    if ur == P.FP32:
        r = oracle.round32(r)
    z = torch.empty(a.n, dtype=TORCH_T[uz], device="cuda")
    s.precond_apply(_dev(r, TORCH_T[ur]), z, uz, ur, omega)
    want = oracle.scale_precond(a.rowptr, a.col, a.val, oracle.M_JACOBI, uz, ur, omega, r)
    _eq(z.double().cpu().numpy(), want)


def _seqs():
    rng = np.random.default_rng(4)
    geo = 3.0 * 0.93 ** np.arange(400)
    osc = np.abs(2.0 * 0.95 ** np.arange(400) * (1 + 0.8 * np.sin(np.arange(400) * 0.7)))
    noisy = np.exp(np.cumsum(rng.normal(-0.05, 0.3, 400)))
    return {"geometric": geo, "oscillating": osc, "noisy": noisy}


@pytest.mark.parametrize("name", ["geometric", "oscillating", "noisy"])
@pytest.mark.parametrize("crit", [P.CRIT_WINDOW, P.CRIT_LINEAR])
@pytest.mark.parametrize("u0", [P.FP64, P.FP16])
@pytest.mark.parametrize("latch", [0, 1])
def test_selector_matches_oracle(name, crit, u0, latch):
    delta = _seqs()[name]
    nb, tol = 2.5, 1e-9
    gp = P.Policy(u0=u0, criterion=crit, latch=latch)
    op = oracle.Policy(u0=u0, criterion=crit, latch=latch)
    got = P.selector_trace(delta, nb, tol, gp)
    want = oracle.selector_trace(delta, nb, tol, op)
    assert np.array_equal(got, want)
    if name == "geometric":
        assert (got[-1] & 0xF) == P.FP32   # the u_r switch happened


@pytest.mark.parametrize("crit", [P.CRIT_WINDOW, P.CRIT_LINEAR])
@pytest.mark.parametrize("side", [-1, 0, 1])
@pytest.mark.parametrize("latch", [0, 1])
def test_selector_threshold_edges(crit, side, latch):
    # T = tol ||b|| placed exactly on (side 0) or one ulp either side of the
    # oracle's eta_40, and nu_k landing exactly on tau_zs and one ulp below it:
    # the device decides these comparisons as the binary64 evaluation does
    delta = 1e-4 * 0.95 ** (np.arange(120) - 25.0)
    delta[25] = 1e-4                      # nu_25 = tau_zs exactly (nb = 1)
    delta[26] = np.nextafter(1e-4, 0.0)
    eta = (oracle.eta_window(delta, 40, 10, 1.0) if crit == P.CRIT_WINDOW
           else oracle.eta_linear(delta, 40, 5, 1.0))
    tol = {0: eta, 1: np.nextafter(eta, np.inf), -1: np.nextafter(eta, 0.0)}[side]
    gp = P.Policy(u0=P.FP64, criterion=crit, latch=latch)
    op = oracle.Policy(u0=oracle.FP64, criterion=crit, latch=latch)
    got = P.selector_trace(delta, 1.0, tol, gp)
    want = oracle.selector_trace(delta, 1.0, tol, op)
    assert np.array_equal(got, want)
    assert (want[25] >> 4) == P.FP64 and (want[26] >> 4) == P.FP32


def test_uniform_slice_layout():
    # a 7-point stencil: nearly every slice holds its rows at one set of
    # offsets (the added entries are exact zeros, so the
    # products are unchanged); the staged SpMV of the solve reads those
    # offsets once per slice.  PCG(FP64) through that layout follows the
    # oracle's residual history.
    a = W.diffusion3d(24, 2.0, 11)
    s = P.Solver(a.rowptr, a.col, a.val)
    lay = s.layout()
    assert lay["idx16"] == 1 and lay["n"] == a.n and lay["nslices"] == (a.n + 31) // 32
    assert 0 < lay["stored_uniform"] < lay["stored"]
    # the rule, restated: 32 rows below n, the union of their offsets as large
    # as the longest row, every row plus every offset a column of the matrix
    want = 0
    for sl in range(lay["nslices"]):
        r0 = 32 * sl
        if r0 + 32 > a.n:
            continue
        offs = [set((a.col[a.rowptr[r]:a.rowptr[r + 1]] - r).tolist()) for r in range(r0, r0 + 32)]
        u = set().union(*offs)
        w = max(len(o) for o in offs)
        if len(u) == w and all(r0 + o >= 0 and r0 + 31 + o < a.n for o in u):
            want += 32 * w
    assert lay["stored_uniform"] == want
    assert lay["stored"] - lay["stored_uniform"] <= 2 * 32 * 7     # first and last slice
    b = np.random.default_rng(5).uniform(-1, 1, a.n)
    x, info = s.solve(_dev(b), tol=1e-10, maxit=2000, policy=P.Policy.pcg64(), history=True)
    ref = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=2000,
                       policy=oracle.Policy(criterion=oracle.FIXED, fixed_uz=oracle.FP64,
                                            fixed_ur=oracle.FP64, scale=oracle.SCALE_NONE))
    assert abs(info.iters - ref.iters) <= 1
    k = min(30, info.iters)
    assert np.allclose(info.relres_hist[:k], ref.relres_hist[:k], rtol=1e-9, atol=0)
    s.close()
    # rows of irregular lengths: no slice is uniform
    r = _varlen(200, 4)
    s2 = P.Solver(r.rowptr, r.col, r.val)
    assert s2.layout()["stored_uniform"] == 0
    s2.close()

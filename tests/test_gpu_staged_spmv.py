"""The persistent iteration kernel's matrix product (Alg. 3: q = A p in u_r,
gamma = q^T p) against the oracle, through ampcg_spmv_loop_step, which runs
that kernel's staged SpMV with the kernel's own grid, shared-memory stages and
per-warp slice runs.  The sizes are chosen so that there are more slices than
warps (from 151,553 rows up on a 148-SM B300): the runs hold floor or
ceil(slices / warps) slices, so runs of two or more occur (from 22% of the
warps at 57^3 to every warp at 128^3, 13-14 slices), the two-slice overlapped
trip and the stage refills run, and at 128^3 the matrix stream carries the L2
evict-first hint; a 20^3 system (250 slices) has warps with one slice and
warps with none.  q is compared bit for bit (one fma per stored entry in
ascending column order in both); gamma is a reduction in another order and
must agree to 1e-12 relative."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")

TT = {P.FP64: torch.float64, P.FP32: torch.float32, P.FP16: torch.float16}


def _random_narrow(n, seed, reach=2000):
    """Rows of 1..8 entries at random offsets within +-reach (int16 offsets,
    slices of unequal patterns), positive diagonal."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 8, n)
    rows, cols = [np.arange(n)], [np.arange(n)]
    for i in np.nonzero(k)[0]:
        c = np.unique(np.clip(i + rng.integers(-reach, reach + 1, k[i]), 0, n - 1))
        c = c[c != i]
        rows.append(np.full(c.size, i))
        cols.append(c)
    r, c = np.concatenate(rows), np.concatenate(cols)
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    val = np.where(r == c, 10.0, -rng.uniform(0.1, 1.0, r.size))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return W.CSR(n, np.cumsum(rowptr).astype(np.int32), c.astype(np.int32), val, {})


def _long_range(n):
    """1D Laplacian whose first and last rows couple to each other: column
    offsets beyond int16, so the matrix keeps int32 column indices."""
    mid = np.arange(1, n - 1)
    col = np.concatenate([[0, 1, n - 1], np.stack([mid - 1, mid, mid + 1], 1).ravel(), [0, n - 2, n - 1]])
    val = np.concatenate([[2.5, -1.0, -0.5], np.tile([-1.0, 2.0, -1.0], n - 2), [-0.5, -1.0, 2.5]])
    rowptr = (3 * np.arange(n + 1)).astype(np.int32)
    return W.CSR(n, rowptr, col.astype(np.int32), val.astype(np.float64), {})


CASES = {
    "diffusion_64cubed": lambda: W.diffusion3d(64, 2.0, 3),
    "diffusion_20cubed_few_slices": lambda: W.diffusion3d(20, 2.0, 6),
    "diffusion_57cubed_ragged": lambda: W.diffusion3d(57, 2.0, 4),
    "diffusion_128cubed": lambda: W.diffusion3d(128, 2.0, 0),
    "random_narrow_200003": lambda: _random_narrow(200003, 5),
    "long_range_int32_180001": lambda: _long_range(180001),
}

PAIRS = [(P.FP16, P.FP64), (P.FP16, P.FP32), (P.FP64, P.FP64), (P.FP32, P.FP32), (P.FP64, P.FP32),
         (P.FP32, P.FP64)]


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    a = CASES[request.param]()
    s = P.Solver(a.rowptr, a.col, a.val)
    yield request.param, a, s
    s.close()


def test_layout_takes_the_paths_under_test(case):
    name, a, s = case
    lay = s.layout()
    warps = 148 * 32
    if name.endswith("few_slices"):
        assert lay["nslices"] < warps      # runs of zero or one slice
    else:
        assert lay["nslices"] > warps, "runs of two or more slices need more slices than warps"
    assert lay["maxw"] <= 8
    assert lay["idx16"] == (0 if name.startswith("long_range") else 1)
    if name == "diffusion_128cubed":
        assert lay["stream_hint"] == 1


@pytest.mark.parametrize("uz,ur", PAIRS)
def test_loop_spmv_bitwise(case, uz, ur):
    name, a, s = case
    rng = np.random.default_rng(17 + 3 * uz + ur)
    p64 = oracle.round_to(uz, rng.standard_normal(a.n))
    p = torch.as_tensor(p64, device="cuda").to(TT[uz])
    q = torch.empty(a.n, dtype=TT[ur], device="cuda")
    g = s.spmv_loop_step(p, q, uz, ur)
    torch.cuda.synchronize()
    aval = a.val if ur == P.FP64 else oracle.round32(a.val)
    ref = oracle.spmv(a.rowptr, a.col, aval, oracle.FP64 if ur == P.FP64 else oracle.FP32, p64)
    got = q.double().cpu().numpy()
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, f"{bad.size} of {a.n} rows differ, first row {bad[0]}: {got[bad[0]]!r} vs {ref[bad[0]]!r}"
    gref = float(np.dot(ref, p64))
    terms = float(np.dot(np.abs(ref), np.abs(p64)))
    assert abs(g - gref) <= 1e-12 * terms

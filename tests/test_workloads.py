"""Invariants of the synthetic input generators (no solver arithmetic)."""
import numpy as np

import workloads as W


def test_poisson_and_diffusion_structure():
    a = W.poisson2d(64)
    assert (a.n, a.nnz) == (4096, 20224)
    d = W.diffusion3d(12, 2.0, 0)
    assert d.nnz == 7 * 12 ** 3 - 6 * 12 ** 2
    dense = d.to_dense()
    assert np.array_equal(dense, dense.T)
    assert np.all(np.diag(dense) > 0)
    off = dense - np.diag(np.diag(dense))
    assert np.all(np.diag(dense) >= -off.sum(axis=1) - 1e-12)   # weakly diagonally dominant
    assert np.all(np.linalg.eigvalsh(dense) > 0)
    assert np.array_equal(d.info["nbound"], 6 - (np.diff(d.rowptr) - 1))


def test_full_size_counts():
    a = W.diffusion3d(128, 2.0, 0)
    assert (a.n, a.nnz) == (2097152, 14581760)
    assert np.all(np.diff(a.col[a.rowptr[5]:a.rowptr[6]]) > 0)


def test_q1_element_rigid_body_modes():
    K = W.q1_element_stiffness(0.25, 0.3)
    ev = np.sort(np.linalg.eigvalsh(K))
    assert np.all(np.abs(ev[:6]) < 1e-12 * ev[-1]) and ev[6] > 1e-3 * ev[-1]
    corners = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    for i, j in [(0, 1), (1, 2), (0, 2)]:
        v = np.zeros(24)
        v[i::3] = -corners[:, j]
        v[j::3] = corners[:, i]
        assert np.abs(K @ v).max() < 1e-12 * ev[-1]


def test_elasticity_assembly_spd_and_blocks():
    B = W.elasticity_q1(6, seed=1)
    assert B.nb == 6 ** 3 - 6 ** 2 and B.bs == 3
    A = B.to_csr()
    dense = A.to_dense()
    assert np.allclose(dense, dense.T, rtol=0, atol=1e-12 * np.abs(dense).max())
    assert np.linalg.eigvalsh(dense).min() > 0
    assert np.diff(B.browptr).max() == 27


def test_batched_2d_cells_structure():
    a = W.diffusion2d_cells(6, 1000)
    A = a.to_dense()
    assert np.array_equal(A, A.T) and np.linalg.eigvalsh(A).min() > 0
    c = np.exp(np.random.default_rng(1000).standard_normal((6, 6))).reshape(-1)
    # interior face between cells 0 and 1: geometric mean; corner row sum: its 2 boundary faces
    assert A[0, 1] == -np.sqrt(c[0] * c[1])
    assert np.isclose(A[0].sum(), 2 * c[0])
    mats, rhs = W.batch_2d(16, seed=0)
    sides = [int(round(np.sqrt(m.n))) for m in mats]
    assert all(32 <= s <= 256 for s in sides) and len(set(sides)) > 8
    assert all(len(r) == m.n for m, r in zip(mats, rhs))

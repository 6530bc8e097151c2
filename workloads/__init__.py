"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only builds matrices and right-hand sides (NumPy, PCG64 seeds).  It
holds none of the solver's arithmetic, and neither the CPU oracle nor the CUDA
library imports it: callers generate a problem here and hand the same arrays to
both.

Matrices are CSR with int32 row pointers / column indices sorted ascending in
every row, FP64 values.  Grid node (x, y, z) has index x + nx*(y + ny*z).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]
    info: dict

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.col] = self.val
        return a


def _assemble(n: int, cols: list, vals: list) -> CSR:
    """Stack per-row candidate entries (already in ascending column order across
    the list) and drop the masked-out ones (col < 0)."""
    c = np.stack(cols, axis=1)          # [n, w]
    v = np.stack(vals, axis=1)
    keep = c >= 0
    counts = keep.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), c[keep].astype(np.int32), v[keep].astype(np.float64), {})


def poisson2d(nx: int, ny: int | None = None) -> CSR:
    """5-point Laplacian (4 / -1) on an nx*ny interior grid, Dirichlet, no h^2."""
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n)
    x, y = idx % nx, idx // nx
    neg = -np.ones(n, dtype=np.int64)
    cols = [np.where(y > 0, idx - nx, neg), np.where(x > 0, idx - 1, neg), idx,
            np.where(x < nx - 1, idx + 1, neg), np.where(y < ny - 1, idx + nx, neg)]
    m1 = -np.ones(n)
    vals = [m1, m1, 4.0 * np.ones(n), m1, m1]
    a = _assemble(n, cols, vals)
    a.info = {"kind": "poisson2d", "nx": nx, "ny": ny}
    return a


def smooth_gaussian_field(shape, sigma: float, seed: int, passes: int = 3) -> np.ndarray:
    """i.i.d. N(0,1) node field, separable 3-tap box filter along every axis
    repeated `passes` times with periodic wrap, normalised to mean 0, std sigma."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape)
    for _ in range(passes):
        for ax in range(g.ndim):
            g = (np.roll(g, 1, axis=ax) + g + np.roll(g, -1, axis=ax)) / 3.0
    g = (g - g.mean()) / g.std()
    return sigma * g


def diffusion3d_from_field(g: np.ndarray) -> CSR:
    """7-point variable-coefficient diffusion on the nodes of g[z, y, x],
    Dirichlet on all sides: face coefficient k_ij = exp((g_i + g_j)/2), boundary
    faces exp(g_i); a_ii = sum of the 6 face coefficients, a_ij = -k_ij."""
    nz, ny, nx = g.shape
    n = nx * ny * nz
    gf = g.reshape(-1)
    idx = np.arange(n)
    x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    sxy = nx * ny
    diag = np.zeros(n)
    cols, vals = [], []
    nbrs = [(z > 0, -sxy), (y > 0, -nx), (x > 0, -1), None, (x < nx - 1, 1), (y < ny - 1, nx),
            (z < nz - 1, sxy)]
    neg = -np.ones(n, dtype=np.int64)
    for nb in nbrs:
        if nb is None:
            cols.append(idx)
            vals.append(diag)  # filled below (same array object)
            continue
        inside, off = nb
        j = np.where(inside, idx + off, idx)
        k = np.where(inside, np.exp(0.5 * (gf + gf[j])), np.exp(gf))
        diag += k
        cols.append(np.where(inside, idx + off, neg))
        vals.append(-k)
    a = _assemble(n, cols, vals)
    kk = -a.val[a.val < 0]
    # boundary faces per node: the 6 faces minus the interior neighbours
    nbound = (6 - (np.diff(a.rowptr) - 1)).astype(np.int32)
    a.info = {"kind": "diffusion3d", "shape": (nx, ny, nz), "nbound": nbound,
              "coef_min": float(kk.min()) if kk.size else 1.0,
              "coef_max": float(kk.max()) if kk.size else 1.0}
    a.info["contrast"] = a.info["coef_max"] / a.info["coef_min"]
    return a


def diffusion3d(n: int, sigma: float = 2.0, seed: int = 0, passes: int = 3) -> CSR:
    """High-contrast 3D diffusion on n^3 nodes (field std sigma, seed)."""
    g = smooth_gaussian_field((n, n, n), sigma, seed, passes)
    a = diffusion3d_from_field(g)
    a.info.update({"n": n, "sigma": sigma, "seed": seed})
    return a


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """b ~ U[-1, 1] from default_rng(seed)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


# --- The paper's synthetic spectra (Sec. 2 and Sec. 5 examples) -------------

def random_orthonormal(n: int, seed: int) -> np.ndarray:
    """Q from the QR factorisation of an n*n standard normal matrix, with the
    signs fixed so that diag(R) > 0 (Haar-distributed)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def dense_spd_csr(eigs: np.ndarray, seed: int) -> CSR:
    """A = Q diag(eigs) Q^T (symmetrised) stored as a full CSR matrix."""
    n = eigs.size
    q = random_orthonormal(n, seed)
    a = (q * eigs) @ q.T
    a = 0.5 * (a + a.T)
    rowptr = (np.arange(n + 1) * n).astype(np.int32)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    out = CSR(n, rowptr, col, a.reshape(-1).copy(), {"kind": "dense_spectrum"})
    out.info["eigs"] = eigs
    return out


def eigs_motivating(n: int = 100) -> np.ndarray:
    """Motivating example (Sec. 2): five large outlying eigenvalues
    lambda_i = 1e-3 + (i-1)/99 (17/20)^(100-i), i = 95..99, lambda_100 = 1, and
    95 evenly spaced values linspace(1e-3, lambda_95, 95)."""
    lam = np.zeros(n)
    i = np.arange(1, n + 1)
    lam_big = 1e-3 + (i - 1) / 99.0 * (17.0 / 20.0) ** (100 - i)
    lam[94:99] = lam_big[94:99]
    lam[99] = 1.0
    lam[:95] = np.linspace(1e-3, lam[94], 95)
    return lam


def eigs_uniform(n: int = 100, lo_ratio: float = 10.0) -> np.ndarray:
    """lambda_i = i/(lo_ratio * n) + (n - i)/n, i = 0..n (n+1 values): the
    linear-convergence example uses lo_ratio = 10 (kappa = 10), the example
    without large outlying eigenvalues lo_ratio = 1000 (kappa = 1e3)."""
    i = np.arange(n + 1)
    return i / (lo_ratio * n) + (n - i) / n


def eigs_limitation(n: int, rho: float) -> np.ndarray:
    """Limitation examples (Sec. 5.6): lambda_i = 1e-3 + (i-1)/(n-1) rho^(n-i),
    i = 1..n-1, and lambda_n = 1."""
    i = np.arange(1, n + 1)
    lam = 1e-3 + (i - 1) / (n - 1) * rho ** (n - i)
    lam[-1] = 1.0
    return lam


def log_coeff_problem(n: int, sigma: float = 1.0, seed: int = 0, perturb: float = 0.1,
                      seed_perturb: int = 2, seed_rhs: int = 1):
    """Coefficient-field workload: theta a smoothed Gaussian node field (std
    sigma), a target field theta_t = theta + perturb * (same generator, other
    seed), the operator of diffusion3d_from_field and b ~ U[-1, 1]."""
    theta = smooth_gaussian_field((n, n, n), sigma, seed)
    theta_t = theta + perturb * smooth_gaussian_field((n, n, n), 1.0, seed_perturb)
    a = diffusion3d_from_field(theta)
    a_t = diffusion3d_from_field(theta_t)
    b = rhs_uniform(a.n, seed_rhs)
    return theta.reshape(-1), theta_t.reshape(-1), a, a_t, b


# --- Linear elasticity, trilinear hexahedra (Q1), block CSR 3x3 ------------

def q1_element_stiffness(h: float, nu: float) -> np.ndarray:
    """24x24 stiffness of a cube element of side h for E = 1, Poisson ratio nu,
    trilinear shape functions, 2x2x2 Gauss quadrature; dof order
    (node a, component c) -> 3a + c, nodes a = x + 2y + 4z over {0,1}^3."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = np.eye(3) * mu
    corners = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)]) * 2 - 1
    g = 1.0 / np.sqrt(3.0)
    K = np.zeros((24, 24))
    for gp in np.array(np.meshgrid([-g, g], [-g, g], [-g, g], indexing="ij")).reshape(3, -1).T:
        dN = np.zeros((8, 3))
        for a in range(8):
            xi = corners[a]
            f = 1 + xi * gp
            dN[a] = xi * np.array([f[1] * f[2], f[0] * f[2], f[0] * f[1]]) / 8.0
        dN *= 2.0 / h                      # d/dx = (2/h) d/dxi
        B = np.zeros((6, 24))
        for a in range(8):
            dx, dy, dz = dN[a]
            B[0, 3 * a] = dx
            B[1, 3 * a + 1] = dy
            B[2, 3 * a + 2] = dz
            B[3, 3 * a] = dy; B[3, 3 * a + 1] = dx
            B[4, 3 * a + 1] = dz; B[4, 3 * a + 2] = dy
            B[5, 3 * a] = dz; B[5, 3 * a + 2] = dx
        K += B.T @ D @ B * (h / 2) ** 3
    return 0.5 * (K + K.T)


@dataclass
class BSR:
    nb: int
    bs: int
    browptr: np.ndarray  # int32 [nb+1]
    bcol: np.ndarray     # int32 [nnzb]
    bval: np.ndarray     # float64 [nnzb, bs, bs]
    info: dict

    def to_csr(self) -> CSR:
        nb, bs = self.nb, self.bs
        nblk = np.diff(self.browptr)
        n = nb * bs
        rowlen = np.repeat(nblk * bs, bs)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(rowlen, out=rowptr[1:])
        col = np.empty(rowptr[-1], dtype=np.int32)
        val = np.empty(rowptr[-1])
        for I in range(nb):
            k0, k1 = self.browptr[I], self.browptr[I + 1]
            J = self.bcol[k0:k1]
            for r in range(bs):
                s = rowptr[I * bs + r]
                col[s:s + (k1 - k0) * bs] = (J[:, None] * bs + np.arange(bs)[None, :]).reshape(-1)
                val[s:s + (k1 - k0) * bs] = self.bval[k0:k1, r, :].reshape(-1)
        return CSR(n, rowptr.astype(np.int32), col, val, dict(self.info))


def elasticity_q1(n: int, seed: int = 0, nu: float = 0.3, e_lo: float = 1.0, e_hi: float = 1e3) -> BSR:
    """Q1 elasticity on n^3 nodes ((n-1)^3 cube elements, h = 1/(n-1)), Young's
    modulus log-uniform in [e_lo, e_hi] per element (seed), Poisson ratio nu,
    nodes on the x = 0 face clamped (removed).  Block CSR with 3x3 blocks."""
    ne = n - 1
    h = 1.0 / ne
    Kr = q1_element_stiffness(h, nu).reshape(8, 3, 8, 3).transpose(0, 2, 1, 3)  # [a, b, 3, 3]
    rng = np.random.default_rng(seed)
    E = np.exp(rng.uniform(np.log(e_lo), np.log(e_hi), ne ** 3))
    ex, ey, ez = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    eidx = ex + ne * (ey + ne * ez)
    E = E[eidx]
    node = lambda x, y, z: x + n * (y + n * z)
    enodes = np.stack([node(ex + ((a >> 0) & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)) for a in range(8)], 1)
    free = np.ones(n ** 3, dtype=bool)
    free[np.arange(n ** 3) % n == 0] = False               # x = 0 face
    newid = -np.ones(n ** 3, dtype=np.int64)
    newid[free] = np.arange(free.sum())
    nb = int(free.sum())
    keys, blocks = [], []
    for a in range(8):
        for b in range(8):
            I, J = newid[enodes[:, a]], newid[enodes[:, b]]
            ok = (I >= 0) & (J >= 0)
            keys.append(I[ok] * nb + J[ok])
            blocks.append(E[ok, None, None] * Kr[a, b][None])
    keys = np.concatenate(keys)
    blocks = np.concatenate(blocks)
    uk, inv = np.unique(keys, return_inverse=True)
    bval = np.zeros((uk.size, 3, 3))
    np.add.at(bval, inv, blocks)
    brow = (uk // nb).astype(np.int64)
    bcol = (uk % nb).astype(np.int32)
    browptr = np.zeros(nb + 1, dtype=np.int64)
    np.add.at(browptr, brow + 1, 1)
    browptr = np.cumsum(browptr).astype(np.int32)
    return BSR(nb, 3, browptr, bcol, bval, {"kind": "elasticity_q1", "n": n, "nu": nu, "dof": nb * 3})


def diffusion2d_cells(s: int, seed: int) -> CSR:
    """2D 5-point diffusion on an s x s grid of cells, Dirichlet: cell
    coefficients exp(N(0,1)) (seed), interior faces the geometric mean of the
    two cells, boundary faces the cell's coefficient; a_ii = sum of faces."""
    c = np.exp(np.random.default_rng(seed).standard_normal((s, s)))
    n = s * s
    idx = np.arange(n)
    x, y = idx % s, idx // s
    cf = c.reshape(-1)
    neg = -np.ones(n, dtype=np.int64)
    diag = np.zeros(n)
    cols, vals = [], []
    for nb in [(y > 0, -s), (x > 0, -1), None, (x < s - 1, 1), (y < s - 1, s)]:
        if nb is None:
            cols.append(idx)
            vals.append(diag)  # filled below (same array object)
            continue
        inside, off = nb
        j = np.where(inside, idx + off, idx)
        k = np.where(inside, np.sqrt(cf * cf[j]), cf)
        diag += k
        cols.append(np.where(inside, idx + off, neg))
        vals.append(-k)
    a = _assemble(n, cols, vals)
    a.info = {"kind": "diffusion2d_cells", "s": s, "seed": seed}
    return a


def batch_2d(nsys: int, seed: int = 0, smin: int = 32, smax: int = 256):
    """Batched workload: nsys systems with sides uniform in {smin..smax} (seed),
    system i from diffusion2d_cells(side_i, 1000 + i), b_i ~ U[-1,1] (seed i)."""
    sides = np.random.default_rng(seed).integers(smin, smax + 1, nsys)
    mats = [diffusion2d_cells(int(s), 1000 + i) for i, s in enumerate(sides)]
    rhs = [rhs_uniform(m.n, i) for i, m in enumerate(mats)]
    return mats, rhs

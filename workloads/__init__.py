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

"""Seeded synthetic inputs (sparse matrices and right-hand sides).

This module builds test systems only; it holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle take their inputs from
it.  Matrices are returned as CSR triples ``(rowptr int64, col int32,
val float64)`` with sorted column indices.

Workloads (stand-ins for the SuiteSparse matrices of the paper's Section 4,
which are not available here):

* ``conv_diff_2d``: -nu Lap(u) + w . grad(u) on the unit square, 5-point
  stencil, first-order upwind convection, Dirichlet boundary, rows scaled by
  h^2, plus a seeded U(0, shift) diagonal term.
* ``conv_diff_3d``: -div(kappa grad u) + w . grad(u) on the unit cube,
  7-point stencil, per-cell kappa ~ lognormal(0, 1), face coefficient the
  harmonic mean of the two cells, upwind convection, rows scaled by h^2.
* ``random_sparse``: nonsymmetric matrix with a fixed number of nonzeros per
  column, N(0, 1) values, a shifted diagonal, and optional log-uniform row /
  column scalings that raise its condition number.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _to_csr(M) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return (M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


def conv_diff_2d(N: int = 32, peclet: float = 10.0, nu: float = 1.0, diag_shift: float = 0.1,
                 seed: int = 1):
    """2D convection-diffusion, n = N*N, wind peclet*(1,1)/sqrt(2)."""
    h = 1.0 / (N + 1)
    w = peclet * nu / np.sqrt(2.0)
    wx = wy = w
    n = N * N
    idx = np.arange(n).reshape(N, N)  # idx[iy, ix]
    rows, cols, vals = [], [], []
    center = np.full((N, N), 4.0 * nu + h * (abs(wx) + abs(wy)))
    rng = np.random.default_rng(seed)
    center += rng.uniform(0.0, diag_shift, size=(N, N))
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(center.ravel())
    # west / east / south / north neighbours; upwind adds h*w to the upstream side
    for dy, dx, conv in ((0, -1, h * wx), (0, 1, 0.0), (-1, 0, h * wy), (1, 0, 0.0)):
        iy, ix = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        jy, jx = iy + dy, ix + dx
        ok = (jy >= 0) & (jy < N) & (jx >= 0) & (jx < N)
        rows.append(idx[iy[ok], ix[ok]])
        cols.append(idx[jy[ok], jx[ok]])
        vals.append(np.full(ok.sum(), -nu - conv))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _to_csr(A)


def conv_diff_3d(N=64, peclet: float = 50.0, seed: int = 3, lognormal_sigma: float = 1.0):
    """3D convection-diffusion with lognormal cell coefficients.

    ``N`` may be an int or a tuple (Nx, Ny, Nz); n = Nx*Ny*Nz.
    """
    if np.isscalar(N):
        Nx = Ny = Nz = int(N)
    else:
        Nx, Ny, Nz = (int(v) for v in N)
    h = 1.0 / (max(Nx, Ny, Nz) + 1)
    w = peclet / np.sqrt(3.0)
    rng = np.random.default_rng(seed)
    kap = np.exp(rng.normal(0.0, lognormal_sigma, size=(Nz, Ny, Nx)))
    n = Nx * Ny * Nz
    idx = np.arange(n).reshape(Nz, Ny, Nx)
    center = np.full((Nz, Ny, Nx), 3.0 * h * w)
    rows, cols, vals = [], [], []
    iz, iy, ix = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    for axis, (dz, dy, dx) in enumerate(((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0))):
        jz, jy, jx = iz + dz, iy + dy, ix + dx
        inside = (jz >= 0) & (jz < Nz) & (jy >= 0) & (jy < Ny) & (jx >= 0) & (jx < Nx)
        kf = kap.copy()  # boundary face: the cell's own coefficient
        kn = kap[np.clip(jz, 0, Nz - 1), np.clip(jy, 0, Ny - 1), np.clip(jx, 0, Nx - 1)]
        kf[inside] = 2.0 * kap[inside] * kn[inside] / (kap[inside] + kn[inside])
        center += kf
        upwind = (dz + dy + dx) < 0  # wind components are all positive
        conv = h * w if upwind else 0.0
        rows.append(idx[inside]); cols.append(idx[jz[inside], jy[inside], jx[inside]])
        vals.append(-kf[inside] - conv)
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(center.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _to_csr(A)


def random_sparse(n: int, nnz_per_col: int = 16, seed: int = 6, shift: float | None = None,
                  log10_scale: float = 0.0):
    """Nonsymmetric sparse matrix: nnz_per_col - 1 off-diagonal N(0,1) entries per
    column at random rows, plus a diagonal entry N(0,1) + shift*sign.  With
    ``log10_scale`` > 0 the result is D_r R D_c with D_r, D_c log-uniform on
    [1, 10^(log10_scale/2)]."""
    rng = np.random.default_rng(seed)
    k = nnz_per_col - 1
    if shift is None:
        shift = 2.0 * np.sqrt(max(k, 1))
    # k distinct off-diagonal rows per column: draw, then redraw the columns
    # that got a repeat until none is left
    rows = rng.integers(0, n - 1, size=(n, k), dtype=np.int64)
    while True:
        srt = np.sort(rows, axis=1)
        bad = np.nonzero(np.any(srt[:, 1:] == srt[:, :-1], axis=1))[0]
        if len(bad) == 0:
            break
        rows[bad] = rng.integers(0, n - 1, size=(len(bad), k), dtype=np.int64)
    rows[rows >= np.arange(n)[:, None]] += 1  # skip the diagonal
    colsj = np.repeat(np.arange(n), k)
    vals = rng.normal(0.0, 1.0, size=n * k)
    dg = rng.normal(0.0, 1.0, size=n)
    dg = dg + np.where(dg >= 0, shift, -shift)
    R = sp.coo_matrix((np.concatenate([vals, dg]),
                       (np.concatenate([rows.ravel(), np.arange(n)]), np.concatenate([colsj, np.arange(n)]))),
                      shape=(n, n))
    if log10_scale > 0:
        half = log10_scale / 2.0
        dr = 10.0 ** rng.uniform(0.0, half, size=n)
        dc = 10.0 ** rng.uniform(0.0, half, size=n)
        R = sp.diags(dr) @ sp.csr_matrix(R) @ sp.diags(dc)
    return _to_csr(R)


def rhs(A, seed: int = 2):
    """x_true ~ N(0, 1) and b = A x_true (double)."""
    rp, ci, va = A
    n = len(rp) - 1
    x = np.random.default_rng(seed).normal(0.0, 1.0, size=n)
    M = sp.csr_matrix((va, ci, rp), shape=(n, n))
    return M @ x, x


def to_scipy(A):
    rp, ci, va = A
    n = len(rp) - 1
    return sp.csr_matrix((va, ci, rp), shape=(n, n))


def cfg_small_2d(seed_mat: int = 1, seed_rhs: int = 2):
    """The n = 1024 system: 32x32 grid, Peclet 10, diagonal + U(0, 0.1)."""
    A = conv_diff_2d(32, 10.0, 1.0, 0.1, seed_mat)
    b, x = rhs(A, seed_rhs)
    return A, b, x


def cfg_large_3d(N=64, seed_mat: int = 3, seed_rhs: int = 2):
    """The 64^3 system (n = 262144): lognormal(0,1) cells, Peclet 50."""
    A = conv_diff_3d(N, 50.0, seed_mat)
    b, x = rhs(A, seed_rhs)
    return A, b, x

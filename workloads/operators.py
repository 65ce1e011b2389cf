"""Synthetic test operators (seeded).

The paper's own test matrices (its Table 1, from a public sparse-matrix
collection) are not available offline; these generators stand in for them
with the same kind of structure: nonsymmetric PDE stencils (convection-
diffusion, shifted Helmholtz, a heterogeneous 3D diffusion-convection field)
and an irregular power-law random matrix with a nonzero diagonal.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .csc import CSC


def _assemble(n, rows, cols, vals, dtype=np.float64) -> CSC:
    M = sp.coo_matrix((np.asarray(vals, dtype=dtype), (np.asarray(rows), np.asarray(cols))), shape=(n, n))
    return CSC.from_scipy(M.tocsc())


def convdiff2d(N: int, b=(10.0, 5.0)) -> CSC:
    """-Lap u + b . grad u on (0,1)^2 with homogeneous Dirichlet data.

    N x N interior grid, h = 1/(N+1), lexicographic order p = ix + N*iy
    (x fastest).  Diffusion: standard 5-point stencil.  Convection: first-
    order upwind (backward differences for b > 0).  No h^2 rescaling.
    Row p: diagonal 4/h^2 + b1/h + b2/h, west -1/h^2 - b1/h,
    south -1/h^2 - b2/h, east and north -1/h^2.
    """
    h = 1.0 / (N + 1)
    b1, b2 = b
    ix, iy = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    ix = ix.ravel(); iy = iy.ravel()
    p = ix + N * iy
    rows = [p]; cols = [p]; vals = [np.full(p.size, 4 / h**2 + b1 / h + b2 / h)]
    for dx, dy, c in ((-1, 0, -1 / h**2 - b1 / h), (0, -1, -1 / h**2 - b2 / h),
                      (1, 0, -1 / h**2), (0, 1, -1 / h**2)):
        m = (ix + dx >= 0) & (ix + dx < N) & (iy + dy >= 0) & (iy + dy < N)
        rows.append(p[m]); cols.append(p[m] + dx + N * dy); vals.append(np.full(m.sum(), c))
    return _assemble(N * N, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def helmholtz_wavenumber(N: int, points_per_wavelength: float = 10.0) -> float:
    h = 1.0 / (N + 1)
    return 2.0 * np.pi / (points_per_wavelength * h)


def helmholtz2d(N: int, k: float | None = None) -> CSC:
    """Complex shifted Helmholtz -Lap u - (k^2 + 0.5 i k^2) u, Dirichlet.

    Compact 9-point Laplacian (1/(6h^2)) [-1 -4 -1; -4 20 -4; -1 -4 -1] on an
    N x N interior grid, h = 1/(N+1), lexicographic order.  The default k
    gives 10 grid points per wavelength (k = 2 pi / (10 h)).
    """
    h = 1.0 / (N + 1)
    if k is None:
        k = helmholtz_wavenumber(N)
    shift = -(k * k + 0.5j * k * k)
    ix, iy = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    ix = ix.ravel(); iy = iy.ravel()
    p = ix + N * iy
    s = 1.0 / (6.0 * h * h)
    rows = [p]; cols = [p]; vals = [np.full(p.size, 20.0 * s + shift, dtype=np.complex128)]
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            if dx == 0 and dy == 0:
                continue
            c = -4.0 * s if (dx == 0 or dy == 0) else -1.0 * s
            m = (ix + dx >= 0) & (ix + dx < N) & (iy + dy >= 0) & (iy + dy < N)
            rows.append(p[m]); cols.append(p[m] + dx + N * dy)
            vals.append(np.full(m.sum(), c, dtype=np.complex128))
    return _assemble(N * N, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), np.complex128)


def powerlaw_degrees(n: int, rng: np.random.Generator, dmin=3, dmax=60, gamma=2.2) -> np.ndarray:
    d = np.arange(dmin, dmax + 1)
    p = d.astype(np.float64) ** (-gamma)
    p /= p.sum()
    return rng.choice(d, size=n, p=p).astype(np.int64)


def powerlaw_random(n: int = 200_000, seed: int = 0, dmin=3, dmax=60, gamma=2.2, diag_factor=1.2) -> CSC:
    """Random sparse nonsymmetric matrix with power-law column degrees.

    Column degree d_j ~ P(d) proportional to d^-gamma on {dmin..dmax},
    counting the diagonal.  The d_j - 1 off-diagonal rows are uniform without
    replacement from {0..n-1} minus {j}; their values are N(0,1).  The
    diagonal is diag_factor times the column's off-diagonal absolute sum.
    numpy PCG64 (default_rng) with the given seed.
    """
    rng = np.random.default_rng(seed)
    deg = powerlaw_degrees(n, rng, dmin, dmax, gamma)
    off = deg - 1
    col = np.repeat(np.arange(n, dtype=np.int64), off)
    # Draw from {0..n-2} and skip the diagonal; redraw duplicates within a column.
    row = rng.integers(0, n - 1, size=col.size)
    row = row + (row >= col)
    while True:
        order = np.lexsort((row, col))
        row = row[order]; col = col[order]
        dup = np.zeros(row.size, dtype=bool)
        dup[1:] = (row[1:] == row[:-1]) & (col[1:] == col[:-1])
        nd = int(dup.sum())
        if nd == 0:
            break
        r = rng.integers(0, n - 1, size=nd)
        row[dup] = r + (r >= col[dup])
    v = rng.standard_normal(row.size)
    colsum = np.bincount(col, weights=np.abs(v), minlength=n)
    diag = diag_factor * colsum
    rows = np.concatenate([row, np.arange(n)])
    cols = np.concatenate([col, np.arange(n)])
    vals = np.concatenate([v, diag])
    return _assemble(n, rows, cols, vals)


def lognormal_field(N: int, sigma: float = 1.5, corr: float = 8.0, seed: int = 0) -> np.ndarray:
    """kappa = exp(sigma g) on an N^3 grid; g is seeded white noise smoothed by
    a Gaussian kernel of standard deviation `corr` cells (periodic), then
    normalised to zero mean and unit variance.  Array index [iz, iy, ix]."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((N, N, N))
    g = gaussian_filter(g, sigma=corr, mode="wrap")
    g = (g - g.mean()) / g.std()
    return np.exp(sigma * g)


def lognormal3d(N: int = 64, sigma: float = 1.5, corr: float = 8.0, conv=(20.0, 0.0, 0.0), seed: int = 0) -> CSC:
    """-div(kappa grad u) + c . grad u on (0,1)^3, Dirichlet, 7-point stencil.

    kappa from lognormal_field; face coefficients are harmonic means of the
    two cell values (the cell value itself on boundary faces).  Convection
    first-order upwind.  h = 1/(N+1), order p = ix + N*iy + N^2*iz.
    """
    h = 1.0 / (N + 1)
    kap = lognormal_field(N, sigma, corr, seed)
    iz, iy, ix = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    ix = ix.ravel(); iy = iy.ravel(); iz = iz.ravel()
    kp = kap.ravel()
    p = ix + N * iy + N * N * iz
    diag = np.zeros(p.size)
    rows = []; cols = []; vals = []
    for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        for sgn in (-1, 1):
            jx, jy, jz = ix + sgn * dx, iy + sgn * dy, iz + sgn * dz
            inside = (jx >= 0) & (jx < N) & (jy >= 0) & (jy < N) & (jz >= 0) & (jz < N)
            q = np.where(inside, jx + N * jy + N * N * jz, 0)
            kq = np.where(inside, kp[q], kp)
            kf = 2.0 * kp * kq / (kp + kq)
            diag += kf / h**2
            c = conv[d]
            upwind = (sgn == -1 and c > 0) or (sgn == 1 and c < 0)
            if upwind:
                diag += abs(c) / h
            off = -kf / h**2 - (abs(c) / h if upwind else 0.0)
            rows.append(p[inside]); cols.append(q[inside]); vals.append(off[inside])
    rows.append(p); cols.append(p); vals.append(diag)
    return _assemble(N**3, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))

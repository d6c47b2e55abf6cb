"""Seeded Inverse-Poisson least-squares matrices A = J^T (paper, Appendices A
and B), generated from the formulas printed there.

This module only *generates* problems; it holds none of the spaQR arithmetic.

The variable-coefficient Poisson equation -div(z grad u) = h on an n x n
(x n) grid with u = 0 on the boundary is discretised on a staggered grid: u at
the n^d interior grid points, z at the (n+1)^d cell centres around them.  The
residual of the equation at grid point g is f_g(u, z) (Appendix A eq. for 2D,
Appendix B for 3D; the constant q_g does not enter the Jacobian).  J =
d f / d(u, z) has one row per equation and one column per variable; the
least-squares matrix is A = J^T: one row per variable (all u, then all z, in
lexicographic order), one column per equation, so that the columns are the grid
points v = i + n*(j + n*k) of the geometric nested dissection.

Readings (the paper leaves them open):

* u and z are drawn at random: u ~ U[-1, 1) on the interior points, z ~ U[1, 2)
  on the cells (a positive diffusion coefficient), from
  numpy.random.default_rng(seed) in this order (u, then z), then b ~ N(0, 1).
* "flat" = f in (0, 1): u = 1 and z = 1 on the central box that covers the
  fraction f of the grid points in every axis (the paper's way of creating zero
  rows to lower the aspect ratio M/N); the z rows inside it vanish.
* Rows that are identically zero are dropped (the paper removes them).
* Row matching (Section 2.2 matches rows to columns before the max-norm rule;
  every row of J^T touches several columns): u row g <-> column g, whose entry
  -a_0 never vanishes.
* 3D: the printed coefficients make a_1..a_6 = -1/4 (sum of four z) and
  a_0 = 3/4 (sum of eight z), so the row sum of the stencil is -2 a_0, unlike
  the 2D stencil (row sum 0).  Reading: a_1..a_6 = +1/4 (sum of four z), the
  3D analogue of the 2D operator (sum_k a_k = a_0).
"""
from __future__ import annotations

import numpy as np

from inputs.grid_ls import GridProblem


def _box_mask(shape, flat):
    """Central box covering the fraction `flat` of the points in every axis."""
    mask = np.zeros(shape, dtype=bool)
    if not flat:
        return mask
    sl = []
    for s in shape:
        w = int(round(flat * s))
        lo = (s - w) // 2
        sl.append(slice(lo, lo + w))
    mask[tuple(sl)] = True
    return mask


def _coeffs_2d(z):
    """a0..a4 at every interior point (arrays n x n, axis order (i, j)) from z
    ((n+1) x (n+1)); z[p, q] is the cell between points p..p+1 and q..q+1 of
    the padded grid (interior points are 1..n)."""
    zc = z[1:, 1:]    # z_{i,j}
    zw = z[:-1, 1:]   # z_{i-1,j}
    zs = z[1:, :-1]   # z_{i,j-1}
    zsw = z[:-1, :-1]  # z_{i-1,j-1}
    a0 = zc + zw + zs + zsw
    a1 = 0.5 * (zc + zs)
    a2 = 0.5 * (zw + zc)
    a3 = 0.5 * (zsw + zw)
    a4 = 0.5 * (zs + zsw)
    return a0, a1, a2, a3, a4


def residual_2d(u, z):
    """f(u, z) without q at every interior point (n x n): the formula of
    Appendix A written out directly (used to pin the Jacobian assembly)."""
    n = u.shape[0]
    up = np.zeros((n + 2, n + 2))
    up[1:-1, 1:-1] = u
    a0, a1, a2, a3, a4 = _coeffs_2d(z)
    c = up[1:-1, 1:-1]
    return (-a0 * c + a1 * up[2:, 1:-1] + a2 * up[1:-1, 2:] + a3 * up[:-2, 1:-1] + a4 * up[1:-1, :-2])


def _coeffs_3d(z):
    """a0..a6 at every interior point (n x n x n, axes (i, j, k)) from z
    ((n+1)^3, z[p, q, r] = cell between points p..p+1, q..q+1, r..r+1)."""
    def Z(di, dj, dk):  # z_{i+di, j+dj, k+dk} for di, dj, dk in {0, -1}
        return z[1 + di: z.shape[0] + di if di else None, 1 + dj: z.shape[1] + dj if dj else None,
                 1 + dk: z.shape[2] + dk if dk else None]
    z000, z100, z010, z001 = Z(0, 0, 0), Z(-1, 0, 0), Z(0, -1, 0), Z(0, 0, -1)
    z110, z011, z101, z111 = Z(-1, -1, 0), Z(0, -1, -1), Z(-1, 0, -1), Z(-1, -1, -1)
    a0 = 0.75 * (z000 + z100 + z010 + z001 + z110 + z011 + z101 + z111)
    a1 = 0.25 * (z000 + z001 + z010 + z011)
    a2 = 0.25 * (z100 + z000 + z101 + z001)
    a3 = 0.25 * (z100 + z000 + z110 + z010)
    a4 = 0.25 * (z100 + z101 + z110 + z111)
    a5 = 0.25 * (z110 + z010 + z111 + z011)
    a6 = 0.25 * (z101 + z001 + z111 + z011)
    return a0, a1, a2, a3, a4, a5, a6


def residual_3d(u, z):
    """f(u, z) without q at every interior point (n^3): Appendix B written out
    directly, with the sign reading of the module docstring."""
    n = u.shape[0]
    up = np.zeros((n + 2, n + 2, n + 2))
    up[1:-1, 1:-1, 1:-1] = u
    a0, a1, a2, a3, a4, a5, a6 = _coeffs_3d(z)
    c = up[1:-1, 1:-1, 1:-1]
    return (-a0 * c + a1 * up[2:, 1:-1, 1:-1] + a2 * up[1:-1, 2:, 1:-1] + a3 * up[1:-1, 1:-1, 2:]
            + a4 * up[:-2, 1:-1, 1:-1] + a5 * up[1:-1, :-2, 1:-1] + a6 * up[1:-1, 1:-1, :-2])


def _assemble(rows_cols_vals, m_rows, n_cols):
    """CSR (columns ascending in a row, duplicates summed) without zero rows;
    returns (rowptr, colidx, vals, kept row ids)."""
    r, c, v = (np.concatenate(x) for x in zip(*rows_cols_vals))
    import scipy.sparse as sp

    A = sp.coo_matrix((v, (r, c)), shape=(m_rows, n_cols)).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    A.sort_indices()
    keep = np.flatnonzero(np.diff(A.indptr) > 0)
    A = A[keep]
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64), keep


def jacobian_rows_2d(u, z):
    """Triplets (row, column, value) of J^T: u rows 0..n^2-1 (point (i, j) ->
    i + n j, 0-based), z rows n^2 + p + (n+1) q; column = equation point."""
    n = u.shape[0]
    a0, a1, a2, a3, a4 = _coeffs_2d(z)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")  # 0-based interior point
    eq = ii + n * jj
    out = []
    # d f_g / d u_{g'}: u_{g'} is the centre (-a0), east (a1), north (a2), west (a3), south (a4) of g
    out.append((eq.ravel(), eq.ravel(), (-a0).ravel()))
    for (di, dj, a) in ((1, 0, a1), (0, 1, a2), (-1, 0, a3), (0, -1, a4)):
        ok = (ii + di >= 0) & (ii + di < n) & (jj + dj >= 0) & (jj + dj < n)
        urow = (ii + di) + n * (jj + dj)
        out.append((urow[ok], eq[ok], a[ok]))
    # d f_g / d z: the four cells around g, with u = 0 outside the interior
    up = np.zeros((n + 2, n + 2))
    up[1:-1, 1:-1] = u
    c, e, w = up[1:-1, 1:-1], up[2:, 1:-1], up[:-2, 1:-1]
    nn, s = up[1:-1, 2:], up[1:-1, :-2]
    zrow = lambda p, q: n * n + p + (n + 1) * q  # noqa: E731  cell (p, q), 0..n
    for (dp, dq, val) in ((1, 1, -c + 0.5 * e + 0.5 * nn),   # z_{i,j}
                          (0, 1, -c + 0.5 * nn + 0.5 * w),   # z_{i-1,j}
                          (1, 0, -c + 0.5 * e + 0.5 * s),    # z_{i,j-1}
                          (0, 0, -c + 0.5 * w + 0.5 * s)):   # z_{i-1,j-1}
        out.append((zrow(ii + dp, jj + dq).ravel(), eq.ravel(), val.ravel()))
    return out, n * n + (n + 1) ** 2, n * n


def jacobian_rows_3d(u, z):
    """Triplets of J^T for the 3D problem: u rows i + n (j + n k), z rows
    n^3 + p + (n+1)(q + (n+1) r); column = equation point."""
    n = u.shape[0]
    a0, a1, a2, a3, a4, a5, a6 = _coeffs_3d(z)
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    eq = ii + n * (jj + n * kk)
    out = [(eq.ravel(), eq.ravel(), (-a0).ravel())]
    for (d, a) in (((1, 0, 0), a1), ((0, 1, 0), a2), ((0, 0, 1), a3), ((-1, 0, 0), a4), ((0, -1, 0), a5),
                   ((0, 0, -1), a6)):
        ok = ((ii + d[0] >= 0) & (ii + d[0] < n) & (jj + d[1] >= 0) & (jj + d[1] < n) & (kk + d[2] >= 0)
              & (kk + d[2] < n))
        urow = (ii + d[0]) + n * ((jj + d[1]) + n * (kk + d[2]))
        out.append((urow[ok], eq[ok], a[ok]))
    up = np.zeros((n + 2, n + 2, n + 2))
    up[1:-1, 1:-1, 1:-1] = u
    c = up[1:-1, 1:-1, 1:-1]
    nb = {(1, 0, 0): up[2:, 1:-1, 1:-1], (0, 1, 0): up[1:-1, 2:, 1:-1], (0, 0, 1): up[1:-1, 1:-1, 2:],
          (-1, 0, 0): up[:-2, 1:-1, 1:-1], (0, -1, 0): up[1:-1, :-2, 1:-1], (0, 0, -1): up[1:-1, 1:-1, :-2]}
    # the cell z_{i+di, j+dj, k+dk} (di, dj, dk in {0, -1}) enters a_0 with 3/4 and the three
    # face coefficients whose four cells contain it with 1/4: on the +x face iff di = 0, on the
    # -x face iff di = -1 (likewise y, z)
    n1 = n + 1
    for di in (0, -1):
        for dj in (0, -1):
            for dk in (0, -1):
                val = -0.75 * c
                val = val + 0.25 * (nb[(1, 0, 0)] if di == 0 else nb[(-1, 0, 0)])
                val = val + 0.25 * (nb[(0, 1, 0)] if dj == 0 else nb[(0, -1, 0)])
                val = val + 0.25 * (nb[(0, 0, 1)] if dk == 0 else nb[(0, 0, -1)])
                p, q, r = ii + 1 + di, jj + 1 + dj, kk + 1 + dk
                out.append(((n ** 3 + p + n1 * (q + n1 * r)).ravel(), eq.ravel(), val.ravel()))
    return out, n ** 3 + n1 ** 3, n ** 3


def inverse_poisson(n: int, dim: int = 2, flat: float = 0.0, seed: int = 0) -> GridProblem:
    """The seeded J^T least-squares problem on an n^dim grid (module docstring)."""
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    u = rng.uniform(-1.0, 1.0, size=shape)
    z = rng.uniform(1.0, 2.0, size=(n + 1,) * dim)
    if flat:
        u[_box_mask(shape, flat)] = 1.0
        # the cells whose corners all lie in the flat box of points
        zmask = np.zeros((n + 1,) * dim, dtype=bool)
        pm = np.pad(_box_mask(shape, flat), 1)
        if dim == 2:
            zmask = pm[:-1, :-1] & pm[1:, :-1] & pm[:-1, 1:] & pm[1:, 1:]
        else:
            zmask = (pm[:-1, :-1, :-1] & pm[1:, :-1, :-1] & pm[:-1, 1:, :-1] & pm[:-1, :-1, 1:]
                     & pm[1:, 1:, :-1] & pm[1:, :-1, 1:] & pm[:-1, 1:, 1:] & pm[1:, 1:, 1:])
        z[zmask] = 1.0
    trip, m_rows, n_cols = (jacobian_rows_2d if dim == 2 else jacobian_rows_3d)(u, z)
    rowptr, colidx, vals, _ = _assemble(trip, m_rows, n_cols)
    m = rowptr.size - 1
    b = rng.standard_normal(m)
    dims = (n, n, 1) if dim == 2 else (n, n, n)
    # the u rows come first and never vanish (their centre entry is -a_0 < 0): u row g <-> column g
    # is a perfect matching with nonzero entries
    return GridProblem(dims[0], dims[1], dims[2], m, n_cols, rowptr, colidx, vals, b, "ip", seed,
                       match=np.arange(n_cols, dtype=np.int32))

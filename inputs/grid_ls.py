"""Seeded synthetic grid least-squares problems min ||A x - b||_2.

This module only *generates* problems; it contains none of the spaQR
arithmetic.  Both the CPU oracle and the GPU library are fed from here.

Problem family (a PDE-grid least-squares class like the paper's Section 4
benchmarks, whose graph(A^T A) is the 5-point (2D) or 7-point (3D) stencil):

* vertices v = i + nx*(j + ny*k) (lexicographic); one unknown per vertex,
  so N = nx*ny*nz;
* rows, in this order: every x-edge (i,j,k)-(i+1,j,k) in lexicographic order
  of its lower endpoint, then every y-edge, then every z-edge, then one
  vertex row per v;
* an edge row holds +w at the lower-index vertex and -w at the higher one;
  a vertex row holds d at its vertex;
* random draws from numpy.random.default_rng(seed) in this order: all w
  (edge-row order), all d, then b ~ N(0, 1) of length M.

Weight laws: "u12" w ~ U[1, 2); "c3" w = 10^U[-3, 3]; "c2" w = 10^U[-2, 2];
d ~ U[0.1, 1] always.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

WEIGHT_LAWS = ("u12", "c3", "c2")


@dataclass
class GridProblem:
    nx: int
    ny: int
    nz: int
    m: int
    n: int
    rowptr: np.ndarray  # int64, length m + 1
    colidx: np.ndarray  # int32, length nnz, ascending within a row
    vals: np.ndarray  # float64, length nnz
    b: np.ndarray  # float64, length m
    law: str
    seed: int
    match: np.ndarray | None = None  # optional row matching: match[j] = the row matched to column j

    @property
    def dims(self):
        return (self.nx, self.ny, self.nz)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.m, self.n))


def _draw_weights(rng, law: str, count: int) -> np.ndarray:
    if law == "u12":
        return rng.uniform(1.0, 2.0, size=count)
    if law == "c3":
        return 10.0 ** rng.uniform(-3.0, 3.0, size=count)
    if law == "c2":
        return 10.0 ** rng.uniform(-2.0, 2.0, size=count)
    raise ValueError(f"unknown weight law {law!r}")


def _edges(nx: int, ny: int, nz: int):
    """Lower/upper endpoints of all x-, then y-, then z-edges (lexicographic)."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    lows, highs = [], []
    if nx > 1:
        lows.append(idx[:, :, :-1].ravel())
        highs.append(idx[:, :, 1:].ravel())
    if ny > 1:
        lows.append(idx[:, :-1, :].ravel())
        highs.append(idx[:, 1:, :].ravel())
    if nz > 1:
        lows.append(idx[:-1, :, :].ravel())
        highs.append(idx[1:, :, :].ravel())
    if lows:
        return np.concatenate(lows), np.concatenate(highs)
    return np.zeros(0, np.int64), np.zeros(0, np.int64)


def grid_problem(nx: int, ny: int, nz: int = 1, law: str = "u12", seed: int = 0) -> GridProblem:
    """Build the seeded grid problem described in the module docstring."""
    n = nx * ny * nz
    lo, hi = _edges(nx, ny, nz)
    ne = lo.size
    m = ne + n
    rng = np.random.default_rng(seed)
    w = _draw_weights(rng, law, ne)
    d = rng.uniform(0.1, 1.0, size=n)
    b = rng.standard_normal(m)

    rowptr = np.empty(m + 1, dtype=np.int64)
    rowptr[0] = 0
    rowptr[1 : ne + 1] = 2 * np.arange(1, ne + 1, dtype=np.int64)
    rowptr[ne + 1 :] = 2 * ne + np.arange(1, n + 1, dtype=np.int64)
    colidx = np.empty(2 * ne + n, dtype=np.int32)
    vals = np.empty(2 * ne + n, dtype=np.float64)
    colidx[0 : 2 * ne : 2] = lo
    colidx[1 : 2 * ne : 2] = hi
    vals[0 : 2 * ne : 2] = w
    vals[1 : 2 * ne : 2] = -w
    colidx[2 * ne :] = np.arange(n, dtype=np.int32)
    vals[2 * ne :] = d
    return GridProblem(nx, ny, nz, m, n, rowptr, colidx, vals, b, law, seed)


# The workloads used by the tests and the benchmark, named by what they are.
WORKLOADS = {
    # 2D 64x64, w ~ U[1,2), nested dissection depth 6.
    "grid2d_64": dict(dims=(64, 64, 1), law="u12", depth=6),
    # 2D 1024x1024, high-contrast w = 10^U[-3,3], depth 16.
    "grid2d_1024": dict(dims=(1024, 1024, 1), law="c3", depth=16),
    # 3D 64^3, w ~ U[1,2), depth 15.
    "grid3d_64": dict(dims=(64, 64, 64), law="u12", depth=15),
    # 2D 128x128 batch member, w = 10^U[-2,2].
    "grid2d_128_c2": dict(dims=(128, 128, 1), law="c2", depth=8),
    # 3D 128^3, w = 10^U[-3,3], depth 18.
    "grid3d_128": dict(dims=(128, 128, 128), law="c3", depth=18),
    # 2D 256x256 of the 1024x1024 family (same leaf size), for kernel profiles.
    "grid2d_256_c3": dict(dims=(256, 256, 1), law="c3", depth=12),
    # The paper's Inverse-Poisson J^T (inputs/inverse_poisson.py): 2D 1024^2 and 3D 64^3 grids of
    # equations, random u and z, aspect ratio about 2.
    "invpoisson2d_1024": dict(dims=(1024, 1024, 1), law="ip", depth=16),
    "invpoisson3d_64": dict(dims=(64, 64, 64), law="ip", depth=15),
}


def workload(name: str, seed: int = 0) -> tuple[GridProblem, int]:
    """Return (problem, nested-dissection depth) for a named workload."""
    spec = WORKLOADS[name]
    nx, ny, nz = spec["dims"]
    if spec["law"] == "ip":
        from inputs.inverse_poisson import inverse_poisson

        return inverse_poisson(nx, 2 if nz == 1 else 3, seed=seed), spec["depth"]
    return grid_problem(nx, ny, nz, spec["law"], seed), spec["depth"]


def tile_problem(prob: GridProblem, t: int) -> GridProblem:
    """The corner tile [0, t)^d of a grid problem as a problem of its own: the
    rows of `prob` whose entries all lie in the tile (edges with both
    endpoints inside, vertex rows inside), in the generator's row order, with
    the values and right-hand side of `prob` (a sample of the same matrix)."""
    nx, ny, nz = prob.dims
    tx, ty = min(t, nx), min(t, ny)
    tz = min(t, nz) if nz > 1 else 1
    sub = grid_problem(tx, ty, tz, "u12", 0)  # the tile's structure; values replaced below
    nex = (nx - 1) * ny * nz
    ney = nx * (ny - 1) * nz
    nez = nx * ny * (nz - 1) if nz > 1 else 0
    rows = []
    if tx > 1:
        I, J, K = np.meshgrid(np.arange(tx - 1), np.arange(ty), np.arange(tz), indexing="ij")
        o = np.lexsort((I.ravel(), J.ravel(), K.ravel()))
        I, J, K = I.ravel()[o], J.ravel()[o], K.ravel()[o]
        rows.append(K * ny * (nx - 1) + J * (nx - 1) + I)
    if ty > 1:
        I, J, K = np.meshgrid(np.arange(tx), np.arange(ty - 1), np.arange(tz), indexing="ij")
        o = np.lexsort((I.ravel(), J.ravel(), K.ravel()))
        I, J, K = I.ravel()[o], J.ravel()[o], K.ravel()[o]
        rows.append(nex + K * (ny - 1) * nx + J * nx + I)
    if tz > 1:
        I, J, K = np.meshgrid(np.arange(tx), np.arange(ty), np.arange(tz - 1), indexing="ij")
        o = np.lexsort((I.ravel(), J.ravel(), K.ravel()))
        I, J, K = I.ravel()[o], J.ravel()[o], K.ravel()[o]
        rows.append(nex + ney + K * ny * nx + J * nx + I)
    V = np.arange(tx * ty * tz)
    vi, vj, vk = V % tx, (V // tx) % ty, V // (tx * ty)
    rows.append(nex + ney + nez + vk * nx * ny + vj * nx + vi)
    rows = np.concatenate(rows)
    assert rows.size == sub.m
    vals = np.empty_like(sub.vals)
    # gather the values row by row: every row of the tile has the same number
    # of entries (2 for an edge, 1 for a vertex) as its row in prob
    src_start = prob.rowptr[rows]
    cnt = sub.rowptr[1:] - sub.rowptr[:-1]
    assert np.array_equal(cnt, prob.rowptr[rows + 1] - src_start)
    idx = np.repeat(src_start - sub.rowptr[:-1], cnt) + np.arange(sub.nnz)
    vals[:] = prob.vals[idx]
    return GridProblem(tx, ty, tz, sub.m, sub.n, sub.rowptr, sub.colidx, vals, prob.b[rows].copy(), prob.law,
                       prob.seed)

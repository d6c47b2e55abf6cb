"""Seeded irregular (non-grid) sparse least-squares problems min ||A x - b||_2.

This module only *generates* problems; it contains none of the spaQR
arithmetic.  The family stands in for matrices without a geometric ordering
(the paper's SuiteSparse set is not available here): graph(A^T A) is an
irregular k-nearest-neighbour graph of random points.

* N points uniform in the unit square, one unknown each (vertex ids in draw
  order, so the numbering carries no geometry);
* one edge row per unordered pair {i, j} where j is among the k nearest
  neighbours of i or i among those of j; +w at the lower id, -w at the higher;
  rows sorted by (lower id, higher id);
* one vertex row (single entry d) for a random subset of the vertices: every
  connected component gets at least one, so that A has full column rank, and
  about `vertex_frac` of all vertices get one; these rows follow the edge rows
  in ascending vertex order.  Columns without a vertex row must be matched to
  an edge row, so the row-column matching is not the trivial one.
* random draws from numpy.random.default_rng(seed) in this order: the points,
  one weight w per edge row (law "u12": U[1,2); "c2": 10^U[-2,2]), the vertex
  row subset, one d ~ U[0.1, 1] per vertex row, then b ~ N(0, 1).
"""
from __future__ import annotations

import numpy as np

from inputs.grid_ls import GridProblem


def knn_problem(n: int, k: int = 4, vertex_frac: float = 0.1, law: str = "u12", seed: int = 0) -> GridProblem:
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    _, nb = cKDTree(pts).query(pts, k=k + 1)
    lo = np.minimum(np.repeat(np.arange(n), k), nb[:, 1:].ravel())
    hi = np.maximum(np.repeat(np.arange(n), k), nb[:, 1:].ravel())
    pairs = np.unique(np.stack([lo, hi], axis=1), axis=0)  # sorted by (lower, higher)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    ne = pairs.shape[0]
    if law == "u12":
        w = rng.uniform(1.0, 2.0, size=ne)
    elif law == "c2":
        w = 10.0 ** rng.uniform(-2.0, 2.0, size=ne)
    else:
        raise ValueError(f"unknown weight law {law!r}")
    G = csr_matrix((np.ones(ne), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    ncomp, comp = connected_components(G, directed=False)
    pick = rng.random(n) < vertex_frac
    for c in range(ncomp):  # every component gets a vertex row (its lowest-id vertex)
        members = np.nonzero(comp == c)[0]
        if not pick[members].any():
            pick[members[0]] = True
    vrows = np.nonzero(pick)[0]
    d = rng.uniform(0.1, 1.0, size=vrows.size)
    m = ne + vrows.size
    b = rng.standard_normal(m)
    rowptr = np.empty(m + 1, dtype=np.int64)
    rowptr[0] = 0
    rowptr[1 : ne + 1] = 2 * np.arange(1, ne + 1, dtype=np.int64)
    rowptr[ne + 1 :] = 2 * ne + np.arange(1, vrows.size + 1, dtype=np.int64)
    colidx = np.empty(2 * ne + vrows.size, dtype=np.int32)
    vals = np.empty(2 * ne + vrows.size, dtype=np.float64)
    colidx[0 : 2 * ne : 2] = pairs[:, 0]
    colidx[1 : 2 * ne : 2] = pairs[:, 1]
    vals[0 : 2 * ne : 2] = w
    vals[1 : 2 * ne : 2] = -w
    colidx[2 * ne :] = vrows
    vals[2 * ne :] = d
    # nx = n, ny = nz = 1: no geometry; the algebraic analysis orders it
    return GridProblem(n, 1, 1, m, n, rowptr, colidx, vals, b, law, seed)

"""The Inverse-Poisson J^T workload (paper, Appendices A and B) and the oracle
on it, without a GPU.

Pins of the generator: J^T equals the central differences of the residual
f(u, z) written out directly from the appendix formulas (f is bilinear in
(u, z), so the differences are exact up to rounding); with u = z = 1 on the
whole grid every z row of a cell with all four (eight) corners inside the grid
vanishes, which leaves n^d + (n+1)^d - (n-1)^d rows; the u rows give a perfect
matching.  The oracle (with that matching, Section 2.2) then factors and
solves: at eps = 0 in at most 2 CGLS iterations with x equal to the
normal-equation solution, at eps > 0 to ||A^T r|| / ||A^T b|| < 1e-10.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from inputs import inverse_poisson as ip
from oracle.spaqr import OracleSpaQR


@pytest.mark.parametrize("dim,n", [(2, 4), (2, 5), (3, 3)])
def test_jacobian_is_the_derivative_of_the_residual(dim, n):
    rng = np.random.default_rng(11 + n)
    u = rng.uniform(-1, 1, size=(n,) * dim)
    z = rng.uniform(1, 2, size=(n + 1,) * dim)
    trip, M, N = (ip.jacobian_rows_2d if dim == 2 else ip.jacobian_rows_3d)(u, z)
    r, c, v = (np.concatenate(x) for x in zip(*trip))
    JT = sp.coo_matrix((v, (r, c)), shape=(M, N)).toarray()
    res = ip.residual_2d if dim == 2 else ip.residual_3d
    f = lambda uu, zz: np.ravel(res(uu, zz), order="F")  # noqa: E731  point i + n j (+ n^2 k)
    J = np.zeros((N, M))
    for t in range(M):
        du, dz = np.zeros_like(u), np.zeros_like(z)
        if t < u.size:
            du[np.unravel_index(t, u.shape, order="F")] = 1.0
        else:
            dz[np.unravel_index(t - u.size, z.shape, order="F")] = 1.0
        J[:, t] = (f(u + du, z + dz) - f(u - du, z - dz)) / 2.0
    assert np.abs(JT - J.T).max() <= 1e-14 * np.abs(JT).max()


@pytest.mark.parametrize("dim,n", [(2, 8), (2, 13), (3, 5)])
def test_flat_grid_keeps_only_boundary_cells(dim, n):
    p = ip.inverse_poisson(n, dim, flat=1.0, seed=0)
    assert p.n == n ** dim
    assert p.m == n ** dim + (n + 1) ** dim - (n - 1) ** dim
    q = ip.inverse_poisson(n, dim, flat=0.0, seed=0)
    assert q.m == n ** dim + (n + 1) ** dim  # random u, z: no zero row


def test_u_rows_match_the_columns():
    p = ip.inverse_poisson(9, 2, seed=3)
    A = p.to_scipy().tocsr()
    assert np.array_equal(np.sort(p.match), np.arange(p.n))
    diag = np.array([A[p.match[j], j] for j in range(p.n)])
    assert np.all(diag < 0)  # -a_0 with z > 0
    assert np.linalg.matrix_rank(A.toarray()) == p.n


def _rel_normal(p, x):
    A = p.to_scipy()
    return np.linalg.norm(A.T @ (A @ x - p.b)) / np.linalg.norm(A.T @ p.b)


def test_oracle_exact_at_eps0():
    p = ip.inverse_poisson(32, 2, seed=1)
    o = OracleSpaQR(p, 5, 0.0).factor()
    x, info = o.solve(p.b)
    assert info["iters"] <= 2
    A = p.to_scipy().tocsc()
    xr = spla.spsolve((A.T @ A).tocsc(), A.T @ p.b)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-10


@pytest.mark.parametrize("n,dim,flat,depth,eps", [(32, 2, 0.0, 5, 1e-4), (32, 2, 0.9, 5, 1e-3),
                                                  (8, 3, 0.0, 4, 1e-3)])
def test_oracle_converges(n, dim, flat, depth, eps):
    p = ip.inverse_poisson(n, dim, flat, seed=1)
    o = OracleSpaQR(p, depth, eps).factor()
    x, info = o.solve(p.b)
    assert _rel_normal(p, x) < 1e-10
    assert info["iters"] <= 10

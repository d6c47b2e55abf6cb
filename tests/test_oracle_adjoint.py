"""Pins of the reference gradient (oracle/adjoint.py) that do not use it to check itself."""
import numpy as np
import scipy.sparse as sp

from inputs.grid_ls import grid_problem
from oracle import adjoint


def _loss(A, b, c):
    # L = c . x with x the dense least-squares solution (LAPACK), independent of the oracle
    x = np.linalg.lstsq(A.toarray(), b, rcond=None)[0]
    return float(c @ x)


def test_grad_matches_central_differences():
    p = grid_problem(5, 4, 1, "c2", 3)
    A = p.to_scipy().tocsr()
    rng = np.random.default_rng(7)
    c = rng.standard_normal(p.n)
    x, lam, gb, gv = adjoint.lstsq_grad(A, p.b, c)
    h = 1e-6
    for e in rng.choice(A.nnz, 12, replace=False):
        Ap, Am = A.copy(), A.copy()
        Ap.data[e] += h
        Am.data[e] -= h
        fd = (_loss(Ap, p.b, c) - _loss(Am, p.b, c)) / (2 * h)
        assert abs(fd - gv[e]) <= 1e-6 * max(1.0, abs(fd)), (e, fd, gv[e])
    for i in rng.choice(p.m, 8, replace=False):
        bp, bm = p.b.copy(), p.b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (_loss(A, bp, c) - _loss(A, bm, c)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gb[i])


def test_square_case_closed_form():
    # M = N: x = A^{-1} b, r = 0, dL/db = A^{-T} g, dL/dA = -(A^{-T} g) x^T
    rng = np.random.default_rng(1)
    n = 9
    D = sp.random(n, n, density=0.4, random_state=2, format="csr") + sp.eye(n) * 3.0
    A = sp.csr_matrix(D)
    b = rng.standard_normal(n)
    g = rng.standard_normal(n)
    x, lam, gb, gv = adjoint.lstsq_grad(A, b, g)
    Ad = A.toarray()
    xs = np.linalg.solve(Ad, b)
    y = np.linalg.solve(Ad.T, g)
    np.testing.assert_allclose(x, xs, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gb, y, rtol=1e-11, atol=1e-12)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    np.testing.assert_allclose(gv, -y[rows] * xs[A.indices], rtol=1e-10, atol=1e-12)


def test_normal_solve_residual():
    p = grid_problem(12, 10, 1, "c3", 0)
    A = p.to_scipy().tocsr()
    g = np.random.default_rng(0).standard_normal(p.n)
    lam = adjoint.normal_solve(A, g)
    res = A.T @ (A @ lam) - g
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(g)

"""The oracle's other solve formulations, pinned without a GPU.

* CSNE (Section 1, after Bjorck): W^T W x~ = A~^T b with refinement.  At
  eps = 0 (W^T W = A~^T A~ up to rounding) it is exact after one solve (the
  refinement finds nothing to correct); at eps > 0 the refinement converges.
  Both must equal the normal-equation solution (scipy's sparse direct solve of
  A^T A x = A^T b).
* "Diag." (Section 4): CGLS preconditioned by diag(A^T A) only; it reaches the
  same solution, in far more iterations than the spaQR-preconditioned CGLS.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from inputs.grid_ls import grid_problem
from oracle.spaqr import OracleSpaQR, solve_diag_cgls


@pytest.fixture(scope="module")
def grid64():
    p = grid_problem(64, 64, 1, "u12", 0)
    A = p.to_scipy().tocsc()
    return p, spla.spsolve((A.T @ A).tocsc(), A.T @ p.b)


def _err(x, xr):
    return np.linalg.norm(x - xr) / np.linalg.norm(xr)


def test_csne_exact_at_eps0(grid64):
    p, xr = grid64
    x, info = OracleSpaQR(p, 6, 0.0).factor().solve_csne(p.b)
    assert info["iters"] <= 2 and info["converged"]
    assert _err(x, xr) < 1e-12


@pytest.mark.parametrize("eps", [1e-4, 1e-2])
def test_csne_refinement_converges(grid64, eps):
    p, xr = grid64
    o = OracleSpaQR(p, 6, eps).factor()
    x, info = o.solve_csne(p.b)
    assert info["converged"] and info["iters"] <= 20
    assert _err(x, xr) < 1e-8
    # each refinement step contracts the normal-equation residual
    h = info["hist"]
    assert all(b < a for a, b in zip(h, h[1:]))


def test_diag_cgls_reaches_the_solution_slowly(grid64):
    p, xr = grid64
    x, info = solve_diag_cgls(p, p.b)
    assert info["converged"]
    assert _err(x, xr) < 1e-7
    _, spaqr_info = OracleSpaQR(p, 6, 1e-4).factor().solve(p.b)
    assert info["iters"] >= 10 * spaqr_info["iters"]

"""The paper's other solve formulations on the GPU, against the oracle (C ABI).

* CSNE (Section 1): the corrected seminormal equations with refinement,
  x~ <- x~ + W^{-1} W^{-T} A~^T (b - A~ x~), from spaqr_solve_csne, against
  OracleSpaQR.solve_csne on the same inputs: the same number of refinement
  steps (within max(1, ceil(0.1 it))), the same stopping residual and the same
  solution.  At eps = 0 one step is exact.
* "Diag." (Section 4): a handle in SPAQR_MODE_DIAG (no factorization, W = I)
  runs CGLS with the column scaling alone; its iteration count and solution
  are compared with oracle.spaqr.solve_diag_cgls.
* "Direct" (Section 4): SPAQR_MODE_DIRECT (no compression) solves exactly:
  at most two CGLS iterations and the normal-equation solution.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from inputs.grid_ls import grid_problem
from oracle.spaqr import OracleSpaQR, solve_diag_cgls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid64():
    p = grid_problem(64, 64, 1, "u12", 0)
    A = p.to_scipy().tocsc()
    return p, spla.spsolve((A.T @ A).tocsc(), A.T @ p.b)


def _err(x, xr):
    return np.linalg.norm(x - xr) / np.linalg.norm(xr)


def _rel(p, x):
    A = p.to_scipy()
    return np.linalg.norm(A.T @ (A @ x - p.b)) / np.linalg.norm(A.T @ p.b)


def _within(it, it_o):
    return abs(it - it_o) <= max(1, math.ceil(0.1 * it_o))


@pytest.mark.parametrize("eps", [0.0, 1e-4, 1e-2])
def test_csne_matches_oracle(grid64, eps):
    import paper_2102_09878_gb300 as sq

    p, xr = grid64
    xo, io = OracleSpaQR(p, 6, eps).factor().solve_csne(p.b)
    g = sq.SpaQR(p, sq.Analysis(p.dims, 6), eps=eps)
    x = g.solve_csne(p.b)
    info = g.last_info
    assert info["converged"] and _rel(p, x) < 1e-10
    assert _within(info["iters"], io["iters"]), (info["iters"], io["iters"])
    if eps == 0.0:
        assert info["iters"] <= 2
    assert _err(x, xo) < 1e-8 and _err(x, xr) < 1e-8


def test_csne_on_device_and_mixed(grid64):
    import torch

    import paper_2102_09878_gb300 as sq

    p, xr = grid64
    an = sq.Analysis(p.dims, 6)
    g = sq.SpaQR(p, an, eps=1e-4)
    x = g.solve_csne(torch.from_numpy(p.b).cuda()).cpu().numpy()
    assert _err(x, xr) < 1e-8
    gm = sq.SpaQR(p, an, eps=1e-4, precision="mixed")
    xm = gm.solve_csne(p.b)
    assert gm.last_info["converged"] and _rel(p, xm) < 1e-10


@pytest.mark.parametrize("dims,law", [((32, 32, 1), "u12"), ((64, 64, 1), "u12"), ((8, 8, 8), "c2")])
def test_diag_cgls_matches_oracle(dims, law):
    import paper_2102_09878_gb300 as sq

    p = grid_problem(*dims, law, 0)
    xo, io = solve_diag_cgls(p, p.b, maxit=20000)
    g = sq.SpaQR(p, sq.Analysis(p.dims, 3), mode="diag", maxit=20000)
    assert g.stats()["n_ops"] == 0
    x = g.solve(p.b)
    it = g.last_info["iters"]
    assert g.last_info["converged"] and _rel(p, x) < 1e-10
    assert _within(it, io["iters"]), (it, io["iters"])
    assert _err(x, xo) < 1e-7


def test_direct_mode_solves_exactly(grid64):
    import paper_2102_09878_gb300 as sq

    p, xr = grid64
    g = sq.SpaQR(p, sq.Analysis(p.dims, 6), mode="direct")
    x = g.solve(p.b)
    assert g.last_info["iters"] <= 2 and _err(x, xr) < 1e-10

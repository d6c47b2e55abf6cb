"""GPU factorization and solve parity with the oracle (2D 64x64, depth 6, and
smaller 2D/3D cases), through the C ABI.

* Direct mode: every stored R_s = [R_ss R_sn] equals the oracle's to 1e-11
  relative (multifrontal QR; R is unique with a non-negative diagonal).
* Full pipeline at eps = 0: every stored factor equals the oracle's (same
  readings, same order) to 1e-10, A D W^{-1} preserves norms (Q^T A W^{-1} = I,
  Section 2.7) and CGLS converges at once.
* eps > 0: ||A^T r|| / ||A^T b|| < 1e-10 and the CGLS iteration count within
  max(1, ceil(0.1 * it_oracle)) of the oracle's.
"""
import math

import numpy as np
import pytest

from inputs.grid_ls import grid_problem
from oracle.spaqr import OracleSpaQR

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def grid64():
    return grid_problem(64, 64, 1, "u12", 0)


def _gpu(prob, depth, **kw):
    import paper_2102_09878_gb300 as sq

    an = sq.Analysis(prob.dims, depth)
    return sq.SpaQR(prob, an, **kw)


def _compare_ops(gops, oops, tol):
    assert len(gops) == len(oops), (len(gops), len(oops))
    for g, o in zip(gops, oops):
        assert g["kind"] == o.kind and g["stage"] == o.stage
        np.testing.assert_array_equal(g["slots"], o.slots)
        if o.kind == "Rs":
            np.testing.assert_array_equal(g["nslots"], o.nslots)
            assert _rel(np.hstack([g["R"], g["Rn"]]), np.hstack([o.R, o.Rn])) < tol
        elif o.kind == "Rp":
            assert _rel(g["R"], o.R) < tol
        else:
            assert g["V"].shape == o.V.shape
            assert _rel(g["V"], o.V) < tol and _rel(g["taus"], o.taus) < tol


def test_direct_mode_fronts_match_oracle(grid64):
    o = OracleSpaQR(grid64, 6, 0.0, mode="direct").factor()
    g = _gpu(grid64, 6, eps=0.0, mode="direct")
    _compare_ops(g.ops(), o.ops, 1e-11)


@pytest.mark.parametrize("rows,qrw", [("tree", 1280), ("maxnorm", 1280), ("tree", 32)])
def test_full_pipeline_eps0_matches_oracle(grid64, rows, qrw):
    """qrw = 32 routes every tall step-1 block of width >= 32 (here up to
    2048 x 64) through the Householder QR before its pivoted QR."""
    import torch

    o = OracleSpaQR(grid64, 6, 0.0, rows=rows).factor()
    g = _gpu(grid64, 6, eps=0.0, rows=rows, step1_qr_width=qrw)
    _compare_ops(g.ops(), o.ops, 1e-10)
    rng = np.random.default_rng(0)
    for _ in range(3):
        z = torch.from_numpy(rng.standard_normal(grid64.n)).cuda()
        t = g.apply_Winv(z.clone())
        q = g.apply_A(t)
        assert abs(q.norm().item() / z.norm().item() - 1.0) < 1e-10
        # the GPU apply agrees with the oracle's apply
        ref = o.apply_Winv(z.cpu().numpy())
        assert _rel(t.cpu().numpy(), ref) < 1e-10
        refT = o.apply_WinvT(z.cpu().numpy())
        assert _rel(g.apply_Winv(z.clone(), transpose=True).cpu().numpy(), refT) < 1e-10
    x = g.solve(grid64.b)
    assert g.last_info["iters"] <= 2
    xo, _ = o.solve(grid64.b)
    assert _rel(x, xo) < 1e-9


@pytest.mark.parametrize("eps,rows", [(1e-4, "tree"), (1e-2, "tree"), (1e-4, "maxnorm")])
def test_eps_solve_matches_oracle(grid64, eps, rows):
    o = OracleSpaQR(grid64, 6, eps, rows=rows).factor()
    xo, io = o.solve(grid64.b)
    g = _gpu(grid64, 6, eps=eps, rows=rows)
    x = g.solve(grid64.b)
    A = grid64.to_scipy()
    rel = np.linalg.norm(A.T @ (A @ x - grid64.b)) / np.linalg.norm(A.T @ grid64.b)
    assert rel < 1e-10, rel
    it, ito = g.last_info["iters"], io["iters"]
    assert abs(it - ito) <= max(1, math.ceil(0.1 * ito)), (it, ito)
    assert _rel(x, xo) < 1e-7


@pytest.mark.parametrize("dims,depth,law,eps", [((32, 32, 1), 5, "c3", 1e-3), ((12, 12, 12), 7, "u12", 1e-3),
                                                 ((40, 24, 1), 6, "c2", 1e-5)])
def test_small_grids_match_oracle(dims, depth, law, eps):
    prob = grid_problem(*dims, law=law, seed=3)
    o = OracleSpaQR(prob, depth, eps).factor()
    xo, io = o.solve(prob.b)
    g = _gpu(prob, depth, eps=eps)
    x = g.solve(prob.b)
    A = prob.to_scipy()
    rel = np.linalg.norm(A.T @ (A @ x - prob.b)) / np.linalg.norm(A.T @ prob.b)
    assert rel < 1e-10
    it, ito = g.last_info["iters"], io["iters"]
    assert abs(it - ito) <= max(1, math.ceil(0.1 * ito)), (it, ito)


def test_mixed_precision_converges(grid64):
    g = _gpu(grid64, 6, eps=1e-4, precision="mixed")
    x = g.solve(grid64.b)
    A = grid64.to_scipy()
    rel = np.linalg.norm(A.T @ (A @ x - grid64.b)) / np.linalg.norm(A.T @ grid64.b)
    assert rel < 1e-10
    assert g.last_info["iters"] < 30


def test_device_solve_and_graphs_off(grid64):
    import torch

    g = _gpu(grid64, 6, eps=1e-4, use_graphs=False)
    x1 = g.solve(grid64.b)
    b = torch.from_numpy(grid64.b).cuda()
    g2 = _gpu(grid64, 6, eps=1e-4, use_graphs=True)
    x2 = g2.solve(b).cpu().numpy()
    assert _rel(x1, x2) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dims,depth,law,eps", [((64, 64, 1), 6, "u12", 1e-4), ((12, 12, 12), 7, "u12", 1e-3)])
def test_step1_qr_route_matches_direct_route(dims, depth, law, eps, precision):
    """Section 2.5.1 step 1 through a Householder QR first (tall blocks of width
    >= 32: up to 2048 x 64 in 2D, 648 x 108 in 3D) or directly.  FP64: same
    ranks and the same stored factors (the pivoted QR of the triangle takes the
    pivots of the block itself; both routes write the kept rows with R_ii >= 0).
    FP32 factor: rank decisions at eps may differ in the last bits, so both
    preconditioners are checked through the solve."""
    prob = grid_problem(*dims, law=law, seed=3)
    a = _gpu(prob, depth, eps=eps, precision=precision, step1_qr_width=32)
    b = _gpu(prob, depth, eps=eps, precision=precision, step1_qr_width=0)
    if precision == "fp64":
        oa, ob = a.ops(), b.ops()
        assert len(oa) == len(ob)
        for x, y in zip(oa, ob):
            assert x["kind"] == y["kind"] and x["stage"] == y["stage"]
            np.testing.assert_array_equal(x["slots"], y["slots"])
            if "nslots" in x:
                np.testing.assert_array_equal(x["nslots"], y["nslots"])
            for key in ("R", "Rn", "V", "taus"):
                if key in x and np.size(x[key]):
                    assert x[key].shape == y[key].shape, key
                    assert _rel(x[key], y[key]) < 1e-9, (key, _rel(x[key], y[key]))
    xa, xb = a.solve(prob.b), b.solve(prob.b)
    A = prob.to_scipy()
    for x in (xa, xb):
        assert np.linalg.norm(A.T @ (A @ x - prob.b)) / np.linalg.norm(A.T @ prob.b) < 1e-10
    assert abs(a.last_info["iters"] - b.last_info["iters"]) <= 1


def test_block_cache_reuse_and_release():
    """Freed working blocks are kept for the next factorization (the same
    sizes come back), reuse changes no result, and release empties the cache."""
    import gc

    import paper_2102_09878_gb300 as sq

    p = grid_problem(64, 64, 1, "u12", 3)
    an = sq.Analysis(p.dims, 6)
    s1 = sq.SpaQR(p, an, eps=1e-2, precision="mixed")
    x1 = s1.solve(p.b)
    ops1 = s1.ops()
    del s1
    gc.collect()
    lib = sq.capi.load()
    assert lib.spaqr_cached_bytes() > 0
    s2 = sq.SpaQR(p, an, eps=1e-2, precision="mixed")
    x2 = s2.solve(p.b)
    ops2 = s2.ops()
    assert len(ops1) == len(ops2)
    for a, b in zip(ops1, ops2):
        for key in ("R", "Rn", "V", "taus"):
            if a.get(key) is not None and np.size(a[key]):
                np.testing.assert_allclose(a[key], b[key], rtol=1e-6, atol=1e-6 * np.abs(a[key]).max())
    np.testing.assert_allclose(x1, x2, rtol=1e-8, atol=1e-8 * np.abs(x1).max())
    del s2
    gc.collect()
    assert sq.release_cached_memory() > 0
    assert lib.spaqr_cached_bytes() == 0

"""Failure paths of the C ABI (status codes of include/spaqr.h), on the GPU.

Every failure here is made on the host or by a bounded device wait that is
made to expire; nothing faults or traps the GPU, and every case checks that
the process can go on working afterwards.

* A zero column: A D with unit column norms (Section 2.7) does not exist and
  A has no full column rank (Section 1) -> SPAQR_ERR_RANK_DEFICIENT.
* maxit reached -> SPAQR_ERR_NOT_CONVERGED with x and the solve info still
  written (the iterate after maxit CGLS steps, Section 4).
* A non-finite right-hand side -> SPAQR_ERR_INVALID_ARG; the handle stays usable.
* The CTA-group exchange of the column-pivoted QR (Section 2.5 kernels) with
  a short wait limit and one arrival that never comes: every wait expires, the
  kernel writes rank -1 and returns, the call reports SPAQR_ERR_TIMEOUT; with
  the limit restored the same call succeeds and matches the cluster route.
"""
import ctypes as C

import numpy as np
import pytest

from inputs.grid_ls import grid_problem

pytestmark = pytest.mark.gpu


def _sq():
    import paper_2102_09878_gb300 as sq

    return sq


def test_zero_column_is_rank_deficient():
    sq = _sq()
    p = grid_problem(16, 16, 1, "u12", 0)
    A = p.to_scipy().tolil()
    A[:, 37] = 0.0  # column 37 (its vertex row and its four edge entries) becomes empty
    A = A.tocsr()
    A.eliminate_zeros()
    p.rowptr = A.indptr.astype(np.int64)
    p.colidx = A.indices.astype(np.int32)
    p.vals = A.data.astype(np.float64)
    an = sq.Analysis(p.dims, 4)
    with pytest.raises(sq.SpaqrError) as ei:
        sq.SpaQR(p, an, eps=1e-3)
    assert ei.value.code == sq.capi.SPAQR_ERR_RANK_DEFICIENT
    assert "zero column 37" in str(ei.value)
    # the process goes on: the intact problem factors and solves
    q = grid_problem(16, 16, 1, "u12", 0)
    x = sq.SpaQR(q, an, eps=1e-3).solve(q.b)
    Aq = q.to_scipy()
    assert np.linalg.norm(Aq.T @ (Aq @ x - q.b)) / np.linalg.norm(Aq.T @ q.b) < 1e-10


def test_maxit_not_converged_writes_x_and_info():
    sq = _sq()
    p = grid_problem(32, 32, 1, "c3", 0)
    an = sq.Analysis(p.dims, 5)
    s = sq.SpaQR(p, an, eps=1e-1, maxit=1)
    lib = sq.capi.load()
    info = sq.capi.SolveInfo()
    x = np.full(p.n, np.nan)
    b = np.ascontiguousarray(p.b)
    rc = lib.spaqr_solve(s._h, sq.capi.ptr(b), sq.capi.ptr(x), 0, C.byref(info))
    assert rc == sq.capi.SPAQR_ERR_NOT_CONVERGED
    assert info.iters == 1 and info.converged == 0
    assert np.all(np.isfinite(x)) and np.linalg.norm(x) > 0
    A = p.to_scipy()
    rel = np.linalg.norm(A.T @ (A @ x - p.b)) / np.linalg.norm(A.T @ p.b)
    assert abs(rel - info.rel_resid) <= 1e-8 * max(rel, 1e-300) + 1e-14
    assert 1e-10 < rel < 1.0
    # one CGLS step from x = 0 is the step along the preconditioned steepest-descent
    # direction; the library's iterate reduces ||A x - b|| below ||b||
    assert np.linalg.norm(A @ x - p.b) < np.linalg.norm(p.b)


def test_nonfinite_rhs_is_rejected_and_handle_survives():
    sq = _sq()
    p = grid_problem(16, 16, 1, "u12", 0)
    s = sq.SpaQR(p, sq.Analysis(p.dims, 4), eps=1e-3)
    for bad in (np.nan, np.inf):
        b = p.b.copy()
        b[5] = bad
        with pytest.raises(sq.SpaqrError) as ei:
            s.solve(b)
        assert ei.value.code == sq.capi.SPAQR_ERR_INVALID_ARG
    x = s.solve(p.b)
    A = p.to_scipy()
    assert np.linalg.norm(A.T @ (A @ x - p.b)) / np.linalg.norm(A.T @ p.b) < 1e-10


def test_qrcp_group_wait_expiry_reports_timeout_then_recovers():
    sq = _sq()
    lib = sq.capi.load()
    rng = np.random.default_rng(3)
    mats = [rng.standard_normal((300, 260)), rng.standard_normal((200, 90))]
    eps = 1e-8
    try:
        # about 0.5 ms per wait at the maximum SM clock, one arrival that never comes
        assert lib.spaqr_debug_set_qrcp_wait(1 << 20, 1) == sq.capi.SPAQR_OK
        with pytest.raises(sq.SpaqrError) as ei:
            sq.dense_qrcp(mats, eps, route="grid")
        assert ei.value.code == sq.capi.SPAQR_ERR_TIMEOUT
    finally:
        lib.spaqr_debug_set_qrcp_wait(0, 0)
    ranks, rows, V, T = sq.dense_qrcp(mats, eps, route="grid")
    ranks_c, rows_c, _, _ = sq.dense_qrcp(mats, eps, route="cluster")
    assert list(ranks) == list(ranks_c) == [260, 90]
    for a, b in zip(rows, rows_c):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
    # a factorization in the same process still works
    p = grid_problem(16, 16, 1, "u12", 0)
    x = sq.SpaQR(p, sq.Analysis(p.dims, 4), eps=1e-3).solve(p.b)
    A = p.to_scipy()
    assert np.linalg.norm(A.T @ (A @ x - p.b)) / np.linalg.norm(A.T @ p.b) < 1e-10

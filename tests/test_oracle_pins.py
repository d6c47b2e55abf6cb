"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

* Householder QR vs LAPACK (numpy.linalg.qr, complete mode): the same
  reflector convention, so the whole transformed front must agree.
* Column-pivoted QR vs LAPACK dgeqp3 (scipy.linalg.qr(pivoting=True)) and vs
  planted singular spectra.
* Direct mode (no scaling/sparsification) is multifrontal QR, whose R is the
  Cholesky factor of the permuted A~^T A (the paper's Section 1 remark that R
  equals the Cholesky factor of A^T A).
* Full pipeline at eps = 0 drops nothing: W^T W = A~^T A~ (Q^T A W^{-1} = I,
  Section 2.7) and CGLS converges in one step to the least-squares solution.
* eps > 0: W^T W - A~^T A~ = O(eps), CGLS reaches ||A^T r|| / ||A^T b|| < 1e-10.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from inputs.grid_ls import grid_problem
from oracle import dense as dn
from oracle.spaqr import OracleSpaQR


# ---------------------------------------------------------------- dense
@pytest.mark.parametrize("m,n,c", [(9, 6, 6), (12, 10, 4), (30, 7, 7), (5, 8, 5), (1, 3, 1)])
def test_householder_matches_lapack_complete_q(m, n, c):
    rng = np.random.default_rng(m * 100 + n)
    F0 = rng.standard_normal((m, n))
    F = F0.copy()
    dn.householder_qr(F, c)
    # LAPACK's reflectors on the first c columns give the same Q_1 ... Q_c
    Q, _ = np.linalg.qr(F0[:, :c], mode="complete")
    np.testing.assert_allclose(F, Q.T @ F0, atol=1e-13 * np.abs(F0).max() * m)


def test_householder_sign_fix_gives_unique_r():
    rng = np.random.default_rng(3)
    F0 = rng.standard_normal((20, 8))
    F = F0.copy()
    dn.householder_qr(F, 8)
    dn.sign_fix_rows(F, 8)
    R_chol = np.linalg.cholesky(F0.T @ F0).T
    assert np.all(np.diag(F[:8, :8]) > 0)
    np.testing.assert_allclose(F[:8, :8], R_chol, rtol=0, atol=1e-12 * np.abs(R_chol).max())
    np.testing.assert_allclose(F[8:], 0.0, atol=1e-14 * 20)


def test_householder_zero_column_is_identity():
    F = np.zeros((4, 3))
    F[:, 1] = [1.0, 2.0, 3.0, 4.0]
    G = F.copy()
    V, taus = dn.householder_qr(G, 1)
    assert taus[0] == 0.0
    np.testing.assert_array_equal(G, F)


@pytest.mark.parametrize("m,n", [(7, 10), (12, 5), (8, 8), (3, 30)])
def test_qrcp_matches_dgeqp3(m, n):
    rng = np.random.default_rng(m + 7 * n)
    X = rng.standard_normal((m, n))
    k, Xf, perm, V, taus = dn.qrcp(X, 0.0)
    Q2, R2, P2 = sla.qr(X, pivoting=True)
    assert k == min(m, n)
    np.testing.assert_array_equal(perm[:k], P2[:k])
    np.testing.assert_allclose(np.abs(np.diag(Xf[:k, :k])), np.abs(np.diag(R2)[:k]), rtol=1e-12)
    # Q^T X from the stored reflectors reproduces the factor rows
    QtX = dn.apply_qt_left(X[:, perm], V, taus)
    np.testing.assert_allclose(QtX[:k], Xf[:k], atol=1e-12)


@pytest.mark.parametrize("eps,expect", [(1e-2, 3), (1e-5, 5), (1e-9, 7), (0.0, 8)])
def test_qrcp_rank_planted_spectrum(eps, expect):
    rng = np.random.default_rng(11)
    m, n = 12, 8
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vt, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.array([1.0, 0.5, 0.2, 1e-4, 5e-5, 1e-7, 5e-8, 1e-12])
    X = (U * sig) @ Vt.T
    k, _, _, _, _ = dn.qrcp(X, eps)
    assert k == expect


def test_qrcp_zero_and_empty():
    assert dn.qrcp(np.zeros((4, 5)), 1e-3)[0] == 0
    assert dn.qrcp(np.zeros((0, 5)), 1e-3)[0] == 0
    assert dn.qrcp(np.zeros((3, 0)), 0.0)[0] == 0
    k, rows = dn.qrcp_rows(np.zeros((4, 5)), 0.0)
    assert k == 0 and rows.shape == (0, 5)


def test_qrcp_rows_preserve_gram_when_nothing_dropped():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((9, 4))  # more rows than columns: rank 4 keeps X^T X
    k, rows = dn.qrcp_rows(X, 0.0)
    assert k == 4
    np.testing.assert_allclose(rows.T @ rows, X.T @ X, atol=1e-12)


def test_q_apply_variants_are_consistent():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((6, 9))
    k, _, _, V, taus = dn.qrcp(X, 0.0)
    Q = dn.apply_q_left(np.eye(6), V, taus)
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-14)
    Y = rng.standard_normal((3, 6))
    np.testing.assert_allclose(dn.apply_q_right(Y, V, taus), Y @ Q, atol=1e-14)
    np.testing.assert_allclose(dn.apply_qt_left(Y.T, V, taus), Q.T @ Y.T, atol=1e-14)


# ---------------------------------------------------------------- factor
@pytest.fixture(scope="module")
def grid64():
    return grid_problem(64, 64, 1, "u12", 0)


def _dense_W(o, n):
    return o.apply_W(np.eye(n))


def test_direct_mode_is_cholesky_of_normal_matrix(grid64):
    o = OracleSpaQR(grid64, 6, 0.0, mode="direct").factor()
    n = grid64.n
    order = np.concatenate([op.slots for op in o.ops if op.kind == "Rs"])
    assert np.array_equal(np.sort(order), np.arange(n))
    W = np.zeros((n, n))
    for op in o.ops:
        assert op.kind == "Rs"
        W[np.ix_(op.slots, op.slots)] = op.R
        W[np.ix_(op.slots, op.nslots)] = op.Rn
    Wp = W[np.ix_(order, order)]
    np.testing.assert_allclose(np.tril(Wp, -1), 0.0)
    AtA = (o.At.T @ o.At).toarray()[np.ix_(order, order)]
    C = np.linalg.cholesky(AtA).T
    rel = np.linalg.norm(Wp - C) / np.linalg.norm(C)
    assert rel < 1e-12, rel


def test_full_pipeline_eps0_is_exact(grid64):
    o = OracleSpaQR(grid64, 6, 0.0).factor()
    kinds = {op.kind for op in o.ops}
    assert "Rp" in kinds  # scaling ran
    n = grid64.n
    W = _dense_W(o, n)
    AtA = (o.At.T @ o.At).toarray()
    rel = np.linalg.norm(W.T @ W - AtA) / np.linalg.norm(AtA)
    assert rel < 1e-12, rel
    # the three applies agree with the dense W
    Winv = o.apply_Winv(np.eye(n))
    np.testing.assert_allclose(Winv @ W, np.eye(n), atol=1e-9)
    np.testing.assert_allclose(o.apply_WinvT(np.eye(n)), Winv.T, atol=1e-9)
    # A~ W^{-1} has orthonormal columns (Q^T A W^{-1} = I)
    AW = o.At @ Winv
    np.testing.assert_allclose(AW.T @ AW, np.eye(n), atol=1e-10)


def test_solve_eps0_matches_normal_equations(grid64):
    o = OracleSpaQR(grid64, 6, 0.0).factor()
    x, info = o.solve(grid64.b, tol=1e-10)
    assert info["iters"] <= 2
    A = grid64.to_scipy()
    xs = spla.spsolve((A.T @ A).tocsc(), A.T @ grid64.b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10
    r = A.T @ (A @ x - grid64.b)
    assert np.linalg.norm(r) / np.linalg.norm(A.T @ grid64.b) < 1e-10


@pytest.mark.parametrize("eps", [1e-4, 1e-2])
def test_eps_positive_is_order_eps_and_converges(grid64, eps):
    o = OracleSpaQR(grid64, 6, eps).factor()
    assert any(op.kind == "Qp" for op in o.ops)  # something was sparsified
    n = grid64.n
    W = _dense_W(o, n)
    AtA = (o.At.T @ o.At).toarray()
    rel = np.linalg.norm(W.T @ W - AtA) / np.linalg.norm(AtA)
    assert rel < 10 * eps, rel
    for op in o.ops:
        if op.kind == "Qp":
            Q = dn.apply_q_left(np.eye(op.slots.size), op.V, op.taus)
            np.testing.assert_allclose(Q.T @ Q, np.eye(op.slots.size), atol=1e-13)
    x, info = o.solve(grid64.b, tol=1e-10)
    assert info["converged"] and info["iters"] < 20
    A = grid64.to_scipy()
    r = A.T @ (A @ x - grid64.b)
    assert np.linalg.norm(r) / np.linalg.norm(A.T @ grid64.b) < 1e-10


def test_smaller_eps_needs_no_more_iterations():
    prob = grid_problem(48, 48, 1, "c3", 2)
    its = []
    for eps in (1e-1, 1e-3, 1e-6):
        o = OracleSpaQR(prob, 6, eps).factor()
        its.append(o.solve(prob.b)[1]["iters"])
    assert its[0] >= its[1] >= its[2], its


def test_3d_small_exact_and_converges():
    prob = grid_problem(8, 8, 8, "u12", 0)
    o = OracleSpaQR(prob, 6, 0.0).factor()
    W = _dense_W(o, prob.n)
    AtA = (o.At.T @ o.At).toarray()
    assert np.linalg.norm(W.T @ W - AtA) / np.linalg.norm(AtA) < 1e-12
    o = OracleSpaQR(prob, 6, 1e-3).factor()
    x, info = o.solve(prob.b)
    assert info["converged"]


def test_step1_rows_sign_fixed_are_unique():
    """Step 1 keeps the first k rows of the pivoted R with R_ii >= 0: for a
    full-rank tall block these rows are the Cholesky factor of the pivoted
    normal matrix, so a QR of the block followed by the pivoted QR of its
    triangle gives the same rows (the route the GPU takes for tall blocks)."""
    import numpy as np

    from oracle import dense as dn

    rng = np.random.default_rng(17)
    X = rng.standard_normal((60, 25)) * np.logspace(0, -3, 25)
    k, rows = dn.qrcp_rows(X, 0.0, sign_fix=True)
    _, Xf, perm, _, _ = dn.qrcp(X, 0.0)
    L = np.linalg.cholesky(X[:, perm].T @ X[:, perm])
    np.testing.assert_allclose(rows[:, perm], L.T, rtol=1e-9, atol=1e-12 * np.abs(L).max())
    R0 = np.linalg.qr(X, mode="r")
    k2, rows2 = dn.qrcp_rows(R0, 0.0, sign_fix=True)
    assert k2 == k
    np.testing.assert_allclose(rows2, rows, rtol=1e-9, atol=1e-12 * np.abs(rows).max())

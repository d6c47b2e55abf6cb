"""GPU parity of the batched dense kernels (through the C ABI) against the oracle.

Front QR (Section 2.3): the oracle's textbook Householder QR of the same
front, then its sign fix; both take the same reflector convention, so the
whole transformed front must agree (rows below c are the rows returned to the
owners or reassigned, so they matter too).  Column-pivoted QR (Section 2.5 /
Section 4 rank rule): ranks and leading rows of Q^T A against the oracle.
Batches are uneven and include empty, 1x1, wide, tall and large fronts (the
last ones take the blocked multi-CTA path).
"""
import numpy as np
import pytest

from oracle import dense as dn

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _oracle_front(A, c):
    F = A.copy()
    dn.householder_qr(F, c)
    dn.sign_fix_rows(F, c)
    return F


def _rel(a, b):
    den = max(np.linalg.norm(b), 1e-300)
    return np.linalg.norm(a - b) / den


def test_front_qr_uneven_batch():
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(0)
    shapes = [(1, 1, 1), (5, 3, 3), (40, 25, 10), (64, 64, 32), (70, 40, 20), (33, 90, 7), (200, 150, 31),
              (128, 17, 17), (3, 9, 2), (250, 300, 64), (8, 5, 0)]
    mats = [rng.standard_normal((m, n)) for (m, n, _) in shapes]
    cs = [c for (_, _, c) in shapes]
    out = sq.dense_front_qr(mats, cs)
    for A, c, F in zip(mats, cs, out):
        ref = _oracle_front(A, c) if c else A
        assert _rel(F, ref) < TOL, (A.shape, c, _rel(F, ref))


def test_front_qr_large_blocked_path():
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(1)
    shapes = [(1200, 400, 70), (3000, 200, 33), (900, 900, 130), (2500, 64, 64)]
    mats = [rng.standard_normal((m, n)) for (m, n, _) in shapes]
    cs = [c for (_, _, c) in shapes]
    out = sq.dense_front_qr(mats, cs)
    for A, c, F in zip(mats, cs, out):
        ref = _oracle_front(A, c)
        assert _rel(F, ref) < TOL, (A.shape, c, _rel(F, ref))
        assert np.all(np.diag(F[:c, :c]) >= 0)
        assert np.all(np.tril(F[:, :c], -1) == 0)


def test_front_qr_zero_column_and_rank_one():
    import paper_2102_09878_gb300 as sq

    A = np.zeros((6, 4))
    A[:, 1] = np.arange(1, 7)
    B = np.outer(np.arange(1.0, 9.0), np.ones(5))
    out = sq.dense_front_qr([A, B], [2, 3])
    for M, c, F in zip([A, B], [2, 3], out):
        ref = _oracle_front(M, c)
        np.testing.assert_allclose(F, ref, atol=1e-12 * max(1.0, np.abs(M).max()))


@pytest.mark.parametrize("route", ["cluster", "grid"])
@pytest.mark.parametrize("eps", [0.0, 1e-3, 1e-8])
def test_qrcp_batch_matches_oracle(eps, route):
    """route "grid": every matrix taller than 64 rows runs on a group of >= 17
    CTAs exchanging through global memory (9 columns over 17 CTAs leaves most
    of them empty; the batch spans several launches)."""
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(2)
    mats = []
    for (m, n, r) in [(12, 30, 12), (40, 25, 25), (20, 20, 8), (7, 100, 7), (60, 9, 9), (1, 1, 1), (30, 30, 4),
                      (150, 400, 60), (80, 30, 30), (100, 9, 9), (65, 200, 40), (300, 70, 70), (257, 257, 100)]:
        U = rng.standard_normal((m, r))
        Vt = rng.standard_normal((r, n))
        s = np.logspace(0, -10, r)
        mats.append((U * s) @ Vt)
    mats.append(np.zeros((5, 6)))
    mats.append(np.zeros((90, 40)))
    ranks, rows, V, T = sq.dense_qrcp(mats, eps, route=route)
    for i, A in enumerate(mats):
        k, Xf, perm, Vo, To = dn.qrcp(A, eps)
        assert ranks[i] == k, (i, ranks[i], k)
        if k < A.shape[0]:
            ref = np.zeros((k, A.shape[1]))
            ref[:, perm] = Xf[:k]
            assert _rel(rows[i], ref) < 1e-10, (i, _rel(rows[i], ref))
        # reflectors of pivots far above the noise are well determined: reflector j
        # carries an error of about u |R_11| / |R_jj| (u = 1.1e-16), below 1e-10 for
        # |R_jj| > 1e-5 |R_11|
        good = np.abs(np.diag(Xf[:k, :k])) > 1e-5 * abs(Xf[0, 0]) if k else []
        if k and good.any():
            j = int(np.argmin(good)) if not good.all() else k
            assert _rel(V[i][:, :j], Vo[:, :j]) < 1e-10 and _rel(T[i][:j], To[:j]) < 1e-10, i


def test_qrcp_large_matrix_global_path():
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(3)
    A = rng.standard_normal((160, 900)) * np.logspace(0, -6, 900)
    ranks, rows, V, T = sq.dense_qrcp([A], 1e-4)
    k, Xf, perm, Vo, To = dn.qrcp(A, 1e-4)
    assert ranks[0] == k
    ref = np.zeros((k, A.shape[1]))
    ref[:, perm] = Xf[:k]
    if k < A.shape[0]:
        assert _rel(rows[0], ref) < 1e-10
    assert _rel(V[0], Vo) < 1e-10


@pytest.mark.parametrize("m,n", [(50, 500), (100, 500), (100, 1000), (100, 2000), (100, 4000), (200, 4000),
                                 (33, 7000), (300, 70)])
def test_qrcp_every_cluster_size(m, n):
    """Shapes chosen so that the planner uses 1, 2, 4, 8 and 16 CTAs per matrix
    with the column slabs in shared memory, and 16 CTAs over a global copy.  The
    matrix is repeated so that the batch fills the GPU (the planner then keeps
    the smallest cluster that fits)."""
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(m * 7 + n)
    r = min(m, n)
    A = (rng.standard_normal((m, r)) * np.logspace(0, -9, r)) @ rng.standard_normal((r, n))
    for eps in (0.0, 1e-6):
        k, Xf, perm, Vo, To = dn.qrcp(A, eps)
        good = np.abs(np.diag(Xf[:k, :k])) > 1e-6 * abs(Xf[0, 0])
        j = k if good.all() else int(np.argmin(good))
        for reps in (1, 160):
            ranks, rows, V, T = sq.dense_qrcp([A] * reps, eps)
            for q in (0, reps - 1):
                assert ranks[q] == k, (ranks[q], k)
                assert _rel(V[q][:, :j], Vo[:, :j]) < 1e-10 and _rel(T[q][:j], To[:j]) < 1e-10
                if k < m:
                    ref = np.zeros((k, n))
                    ref[:, perm] = Xf[:k]
                    assert _rel(rows[q], ref) < 1e-9


@pytest.mark.parametrize("route", ["cluster", "auto"])
@pytest.mark.parametrize("m,n,eps", [(2000, 600, 0.0), (2000, 600, 1e-3), (1500, 1400, 1e-6), (600, 3000, 1e-8),
                                     (700, 2500, 0.0)])
def test_qrcp_delayed_update_global_path(m, n, eps, route):
    """Matrices too large for the slabs of 16 CTAs.  route "cluster": the
    delayed-update kernel (panels of reflectors applied as one block update),
    including ranks that stop in the middle of a panel; route "auto": slabs in
    shared memory over CTA groups of up to one CTA per SM (55 to 88 CTAs per
    matrix here), exchanging through global memory."""
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(m + 3 * n)
    r = min(m, n)
    A = (rng.standard_normal((m, r)) * np.logspace(0, -12, r)) @ rng.standard_normal((r, n))
    ranks, rows, V, T = sq.dense_qrcp([A, A[:, ::-1].copy()], eps, route=route)
    for q, B in enumerate((A, A[:, ::-1].copy())):
        k, Xf, perm, Vo, To = dn.qrcp(B, eps)
        assert ranks[q] == k, (ranks[q], k)
        good = np.abs(np.diag(Xf[:k, :k])) > 1e-6 * abs(Xf[0, 0])
        j = k if good.all() else int(np.argmin(good))
        assert _rel(V[q][:, :j], Vo[:, :j]) < 1e-9 and _rel(T[q][:j], To[:j]) < 1e-9
        if k < m:
            ref = np.zeros((k, n))
            ref[:, perm] = Xf[:k]
            assert _rel(rows[q], ref) < 1e-8


def test_qrcp_wide_fp64_shallow_panels():
    """A wide FP64 matrix whose delayed-update coefficients for 16-step panels
    exceed shared memory: the planner takes shallower panels (same results)."""
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(21)
    m, n, r = 2048, 20000, 120
    A = (rng.standard_normal((m, r)) * np.logspace(0, -8, r)) @ rng.standard_normal((r, n))
    ranks, rows, V, T = sq.dense_qrcp([A], 1e-5)
    k, Xf, perm, Vo, To = dn.qrcp(A, 1e-5)
    assert ranks[0] == k
    good = np.abs(np.diag(Xf[:k, :k])) > 1e-6 * abs(Xf[0, 0])
    j = k if good.all() else int(np.argmin(good))
    assert _rel(V[0][:, :j], Vo[:, :j]) < 1e-9 and _rel(T[0][:j], To[:j]) < 1e-9
    ref = np.zeros((k, n))
    ref[:, perm] = Xf[:k]
    assert _rel(rows[0], ref) < 1e-8


@pytest.mark.parametrize("route", ["cluster", "grid", "auto"])
def test_qrcp_f32_matches_oracle(route):
    """The FP32 pivoted QR of the mixed-precision factorization (FP32 data and
    pivot norms as in single-precision LAPACK, R_ii and the rank test to FP64 accuracy in
    double-float arithmetic) against the
    FP64 oracle on matrices whose spectrum leaves no doubt about the rank at
    eps = 1e-4 (singular values in [1e-2, 1] above a gap to 1e-7): same rank,
    same pivots, rows and reflectors within FP32 accuracy (5e-4 relative: FP32
    rounding, 6e-8 per operation, grown by the 1e2 condition of the kept block
    and by sums of up to 1650 terms).  Shapes cover one warp, clusters, and
    (route "auto") CTA groups over global memory (1650 x 879)."""
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(31)
    mats = []
    for (m, n, r) in [(60, 40, 25), (300, 200, 120), (257, 700, 150), (800, 300, 200), (1650, 879, 300)]:
        s = np.concatenate([np.logspace(0, -2, r), 1e-7 * np.ones(min(m, n) - r)])
        U, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
        W, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
        mats.append((U * s) @ W.T)
    ranks, rows, V, T = sq.dense_qrcp_f32(mats, 1e-4, route=route)
    for i, A in enumerate(mats):
        k, Xf, perm, Vo, To = dn.qrcp(A, 1e-4)
        assert ranks[i] == k, (i, ranks[i], k)
        ref = np.zeros((k, A.shape[1]))
        ref[:, perm] = Xf[:k]
        assert _rel(rows[i], ref) < 5e-4, (i, _rel(rows[i], ref))
        assert _rel(V[i], Vo) < 5e-4 and _rel(T[i], To) < 5e-4, i


@pytest.mark.parametrize("f32", [False, True])
def test_qrcp_work_copy_groups(f32):
    """Matrices larger than the shared memory of every SM (FP64 3000 x 1600,
    FP32 4000 x 2300, two each), route "grid": CTA groups over a global work
    copy (all SMs shared between the two), rank 200 at eps 1e-8 (FP64, noise 1e-13) or at
    eps 1e-4 (FP32: singular values down to 1e-2, then only the FP32 rounding
    of the data)."""
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(41)
    m, n, r = (4000, 2300, 200) if f32 else (3000, 1600, 200)
    s = np.logspace(0, -2, r) if f32 else np.logspace(0, -6, r)
    mats = []
    for _ in range(2):
        U, _ = np.linalg.qr(rng.standard_normal((m, r)))
        W, _ = np.linalg.qr(rng.standard_normal((n, r)))
        mats.append((U * s) @ W.T + (0.0 if f32 else 1e-13) * rng.standard_normal((m, n)))
    eps = 1e-4 if f32 else 1e-8
    fn = sq.dense_qrcp_f32 if f32 else sq.dense_qrcp
    tol = 1e-9
    ranks, rows, V, T = fn(mats, eps, route="grid")
    for i, A in enumerate(mats):
        if f32:
            # 2300 columns of nearly equal norms: FP32 and FP64 norms may order
            # near-ties differently, so check what any valid answer satisfies:
            # the rank, and A = Q [rows; 0] to FP32 accuracy, 1e-4 (the dropped part
            # is the FP32 rounding of the data)
            assert ranks[i] == r, ranks[i]
            Y = np.zeros((m, n))
            Y[:r] = rows[i]
            assert _rel(dn.apply_q_left(Y, V[i], T[i]), A) < 1e-4
            continue
        k, Xf, perm, Vo, To = dn.qrcp(A, eps)
        assert ranks[i] == k == r, (ranks[i], k)
        ref = np.zeros((k, n))
        ref[:, perm] = Xf[:k]
        assert _rel(rows[i], ref) < tol, _rel(rows[i], ref)
        assert _rel(V[i], Vo) < tol and _rel(T[i], To) < tol

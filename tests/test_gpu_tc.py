"""Tensor-core (tcgen05, 3xTF32) products of the FP32 factorization.

* The GEMM C - A B matches the FP64 product to FP32 accuracy: the 3xTF32
  split (hi = tf32(x), lo = x - hi; hi.hi + hi.lo + lo.hi) must do better than
  one TF32 product, whose 10-bit mantissa gives errors near 1e-3.
* The FP32 blocked front QR (tensor-core trailing updates) matches the FP64
  oracle's Householder QR to FP32 accuracy, including uneven tiles, trailing
  blocks narrower than a tile and fronts whose panel count differs in one batch.
"""
import numpy as np
import pytest

from oracle import dense as dn

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_front(A, c):
    F = A.copy()
    dn.householder_qr(F, c)
    dn.sign_fix_rows(F, c)
    return F


@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (5, 3, 32), (300, 200, 64), (1000, 517, 32), (129, 257, 96),
                                   (40, 1000, 8)])
def test_tc_gemm_matches_fp64(m, n, k):
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(m + 7 * n + 31 * k)
    A = rng.standard_normal((m, k)).astype(np.float32)
    B = rng.standard_normal((k, n)).astype(np.float32)
    Cm = rng.standard_normal((m, n)).astype(np.float32)
    out = sq.dense_tc_gemm(A, B, Cm)
    ref = Cm.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64)
    err = np.abs(out - ref).max() / (np.abs(A).max() * np.abs(B).max() * k)
    assert err < 2e-6, err


@pytest.mark.parametrize("shape", [(1200, 400, 70), (3000, 200, 33), (900, 900, 130), (2500, 64, 64), (700, 650, 600)])
def test_front_qr_f32_tensor_core_path(shape):
    import paper_2102_09878_gb300 as sq

    m, n, c = shape
    rng = np.random.default_rng(m + n + c)
    A = rng.standard_normal((m, n))
    F = sq.dense_front_qr_f32([A], [c])[0]
    ref = _oracle_front(A, c)
    assert _rel(F.astype(np.float64), ref) < 1e-4, _rel(F.astype(np.float64), ref)


def test_front_qr_f32_uneven_batch():
    import paper_2102_09878_gb300 as sq

    rng = np.random.default_rng(5)
    shapes = [(1500, 300, 290), (800, 700, 64), (2000, 100, 40), (600, 600, 1)]
    mats = [rng.standard_normal((m, n)) for (m, n, _) in shapes]
    outs = sq.dense_front_qr_f32(mats, [c for (_, _, c) in shapes])
    for A, (m, n, c), F in zip(mats, shapes, outs):
        ref = _oracle_front(A, c)
        assert _rel(F.astype(np.float64), ref) < 1e-4, (m, n, c)

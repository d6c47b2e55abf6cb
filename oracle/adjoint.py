"""Reference gradient of the least-squares solution (test infrastructure only).

The solution map of the problem statement, x(A, b) = argmin ||A x - b||_2 =
(A^T A)^{-1} A^T b (Section 1, M >= N, full column rank), differentiated by
hand: for a scalar loss L with g = dL/dx, put lambda = (A^T A)^{-1} g and
r = b - A x.  Then

    dx = (A^T A)^{-1} (dA^T r - A^T dA x)
    dL = g^T dx = r^T dA lambda - (A lambda)^T dA x + (A lambda)^T db

so dL/db = A lambda and dL/dA = r lambda^T - (A lambda) x^T, taken on the
nonzeros of A.  Every step below is that definition written out, with a sparse
direct solve (SuperLU) of the normal equations as the linear-algebra
primitive.  Pinned in tests by central finite differences and by the square
case, where x = A^{-1} b gives dL/db = A^{-T} g and dL/dA = -A^{-T} g x^T.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def normal_solve(A: sp.csr_matrix, rhs: np.ndarray) -> np.ndarray:
    """(A^T A)^{-1} rhs by a sparse direct factorization of the normal matrix."""
    N = (A.T @ A).tocsc()
    return spla.spsolve(N, rhs)


def lstsq(A: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """x = (A^T A)^{-1} A^T b."""
    return normal_solve(A, A.T @ b)


def lstsq_grad(A: sp.csr_matrix, b: np.ndarray, g: np.ndarray, x: np.ndarray | None = None):
    """(x, lambda, dL/db, dL/dvals) for dL/dx = g; dL/dvals in the CSR order of A."""
    A = sp.csr_matrix(A)
    if x is None:
        x = lstsq(A, b)
    lam = normal_solve(A, g)
    r = b - A @ x
    al = A @ lam
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    cols = A.indices
    gvals = r[rows] * lam[cols] - al[rows] * x[cols]
    return x, lam, al, gvals

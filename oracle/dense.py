"""Oracle: dense Householder QR and column-pivoted (rank-revealing) QR in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``house`` / ``householder_qr``: the textbook Householder reflector
  H = I - tau v v^T with v[0] = 1 and beta = -sign(alpha) ||x|| (sign(0) = +1),
  H x = beta e_1; tau = 0 (H = I) when x[1:] is zero.  Used for the block
  Householder QR of a front (Section 2.3) and of A_pp in the interface
  scaling (Section 2.4).  ``sign_fix_rows`` then makes diag(R) >= 0.
* ``qrcp``: column-pivoted Householder QR (pivot = largest remaining column
  norm, ties to the lowest original column index) stopped at the numerical rank: r is the
  largest prefix with |R_ii| >= eps |R_11| and R_ii != 0 (Section 4, the
  paper's use of a column-pivoted QR with that stopping rule).  Column norms
  are downdated after every step and recomputed exactly when the downdated
  squared norm falls below 1e-8 of its last exact value.
"""
from __future__ import annotations

import math

import numpy as np

RECOMPUTE_FRACTION = 1e-8


def house(x: np.ndarray):
    """Reflector for x: returns (v, tau, beta) with (I - tau v v^T) x = beta e_1."""
    alpha = float(x[0])
    sigma = float(x[1:] @ x[1:])
    v = np.zeros_like(x)
    v[0] = 1.0
    if sigma == 0.0:
        return v, 0.0, alpha
    norm = math.sqrt(alpha * alpha + sigma)
    beta = -norm if alpha >= 0.0 else norm
    v[1:] = x[1:] / (alpha - beta)
    tau = (beta - alpha) / beta
    return v, tau, beta


def householder_qr(F: np.ndarray, c: int):
    """In-place Householder QR of the first c columns of F, applying every
    reflector to the remaining columns as well.  Returns (V, taus): column j of
    V holds reflector j in rows j..m-1 (V[j, j] = 1)."""
    m, n = F.shape
    steps = min(c, m)
    V = np.zeros((m, steps))
    taus = np.zeros(steps)
    for j in range(steps):
        v, tau, beta = house(F[j:, j].copy())
        V[j:, j] = v
        taus[j] = tau
        F[j, j] = beta
        F[j + 1 :, j] = 0.0
        if tau != 0.0 and j + 1 < n:
            w = v @ F[j:, j + 1 :]
            F[j:, j + 1 :] -= tau * np.outer(v, w)
    return V, taus


def sign_fix_rows(F: np.ndarray, c: int) -> None:
    """Flip rows i < c of R (the leading c rows of F) so that R_ii >= 0."""
    for i in range(min(c, F.shape[0])):
        if F[i, i] < 0.0:
            F[i, :] *= -1.0


def qrcp(X: np.ndarray, eps: float):
    """Column-pivoted Householder QR of X, stopped at the numerical rank.

    Returns (k, Xf, perm, V, taus): k is the rank; Xf is X after the k
    reflectors with its columns permuted by perm (rows 0..k-1 hold [R11 R12]);
    V (m x k) and taus hold the reflectors, Q = H_1 ... H_k.
    """
    X = np.array(X, dtype=np.float64, copy=True)
    m, n = X.shape
    perm = np.arange(n)
    nu = np.einsum("ij,ij->j", X, X) if m and n else np.zeros(n)
    nu_ref = nu.copy()
    kmax = min(m, n)
    V = np.zeros((m, kmax))
    taus = np.zeros(kmax)
    r11 = 0.0
    k = 0
    for i in range(kmax):
        sub = nu[i:]
        cand = np.flatnonzero(sub == sub.max()) + i
        j = int(cand[np.argmin(perm[cand])])  # ties to the lowest original column index
        if j != i:
            X[:, [i, j]] = X[:, [j, i]]
            nu[[i, j]] = nu[[j, i]]
            nu_ref[[i, j]] = nu_ref[[j, i]]
            perm[[i, j]] = perm[[j, i]]
        v, tau, beta = house(X[i:, i].copy())
        if i == 0:
            r11 = abs(beta)
        if beta == 0.0 or abs(beta) < eps * r11:
            break
        V[i:, i] = v
        taus[i] = tau
        X[i, i] = beta
        X[i + 1 :, i] = 0.0
        if tau != 0.0 and i + 1 < n:
            w = v @ X[i:, i + 1 :]
            X[i:, i + 1 :] -= tau * np.outer(v, w)
        k = i + 1
        for jj in range(i + 1, n):
            nu[jj] -= X[i, jj] * X[i, jj]
            if nu[jj] < RECOMPUTE_FRACTION * nu_ref[jj]:
                nu[jj] = float(X[i + 1 :, jj] @ X[i + 1 :, jj])
                nu_ref[jj] = nu[jj]
    return k, X, perm, V[:, :k], taus[:k]


def qrcp_rows(X: np.ndarray, eps: float, sign_fix: bool = False):
    """Rank k and the first k rows of Q^T X (columns in their original order).
    sign_fix: flip each row i whose diagonal entry R_ii (column perm[i]) is
    negative, so that the rows no longer depend on the reflector signs."""
    k, Xf, perm, _, _ = qrcp(X, eps)
    out = np.zeros((k, X.shape[1]))
    out[:, perm] = Xf[:k, :]
    if sign_fix:
        for i in range(k):
            if Xf[i, i] < 0.0:
                out[i, :] *= -1.0
    return k, out


def apply_q_right(Y: np.ndarray, V: np.ndarray, taus: np.ndarray) -> np.ndarray:
    """Y Q with Q = H_1 ... H_k (each row y^T -> y^T H_1 ... H_k)."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    for i in range(V.shape[1]):
        v = V[:, i]
        Y -= taus[i] * np.outer(Y @ v, v)
    return Y


def apply_qt_left(Y: np.ndarray, V: np.ndarray, taus: np.ndarray) -> np.ndarray:
    """Q^T Y = H_k ... H_1 Y."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    for i in range(V.shape[1]):
        v = V[:, i]
        Y -= taus[i] * np.outer(v, v @ Y)
    return Y


def apply_q_left(Y: np.ndarray, V: np.ndarray, taus: np.ndarray) -> np.ndarray:
    """Q Y = H_1 ... H_k Y."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    for i in reversed(range(V.shape[1])):
        v = V[:, i]
        Y -= taus[i] * np.outer(v, v @ Y)
    return Y

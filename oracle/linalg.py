"""Dense FP64 building blocks of the oracle (test infrastructure).

Alg. 1 needs a QR decomposition (fourth step, and the re-orthonormalisation
of the subspace iterations) and an SVD of the small matrix T (sixth step).  The
oracle writes both out by hand, with numpy's matrix-vector products as the only
library primitive:

  householder_qr  -- Householder reflections, thin Q and upper-triangular R
                     (Golub & Van Loan, Matrix Computations, Alg. 5.2.1).
  jacobi_svd      -- one-sided (Hestenes 1958) Jacobi SVD: rotate column pairs
                     of A until all are mutually orthogonal; cyclic-by-rows
                     pair order; stop when |a_i.a_j| <= tol ||a_i|| ||a_j|| for
                     every pair, at most `max_sweeps` sweeps.
  sign_fix        -- the column sign convention used for U.
"""
from __future__ import annotations

import numpy as np


class NoConvergence(RuntimeError):
    pass


def householder_qr(A: np.ndarray):
    """Thin QR of A (n x l, n >= l): Q (n x l) with orthonormal columns and R
    (l x l) upper triangular, A = Q R.  A zero column below the diagonal gives
    an identity reflector, so Q stays orthonormal when A is rank deficient."""
    A = np.array(A, dtype=np.float64, copy=True)
    n, l = A.shape
    if n < l:
        raise ValueError("householder_qr needs n >= l")
    V = []
    for j in range(l):
        x = A[j:, j]
        nx = np.sqrt(x @ x)
        v = x.copy()
        if nx == 0.0:
            V.append(None)
            continue
        alpha = -nx if x[0] >= 0 else nx
        v[0] -= alpha
        vn = np.sqrt(v @ v)
        v /= vn
        A[j:, j:] -= 2.0 * np.outer(v, v @ A[j:, j:])
        V.append(v)
    R = np.triu(A[:l, :l])
    Q = np.zeros((n, l))
    Q[np.arange(l), np.arange(l)] = 1.0
    for j in reversed(range(l)):
        v = V[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q, R


def jacobi_svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """One-sided Jacobi SVD of A (m x l, m >= l).

    Finds an orthogonal J (product of plane rotations) such that A J = W has
    mutually orthogonal columns.  Then A = (W diag(1/s)) diag(s) J^T with
    s = column norms of W.  Returns (Ul, s, Vr): Ul (m x l) left singular
    vectors, s (l,) singular values in descending order (stable for ties), Vr
    (l x l) right singular vectors (= J, permuted), so A = Ul diag(s) Vr^T.
    Columns of Ul for s == 0 are zero."""
    W = np.array(A, dtype=np.float64, copy=True)
    m, l = W.shape
    J = np.eye(l)
    for _sweep in range(max_sweeps):
        rotated = False
        for i in range(l - 1):
            for j in range(i + 1, l):
                wi, wj = W[:, i], W[:, j]
                alpha = wi @ wi
                beta = wj @ wj
                gamma = wi @ wj
                if gamma == 0.0 or abs(gamma) <= tol * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                wi_old = wi.copy()
                W[:, i] = c * wi_old - s * wj
                W[:, j] = s * wi_old + c * wj
                ji_old = J[:, i].copy()
                J[:, i] = c * ji_old - s * J[:, j]
                J[:, j] = s * ji_old + c * J[:, j]
        if not rotated:
            break
    else:
        raise NoConvergence(f"one-sided Jacobi did not converge in {max_sweeps} sweeps")
    s = np.sqrt(np.einsum("ij,ij->j", W, W))
    order = np.argsort(-s, kind="stable")
    s = s[order]
    W = W[:, order]
    J = J[:, order]
    Ul = np.zeros_like(W)
    nz = s > 0
    Ul[:, nz] = W[:, nz] / s[nz]
    return Ul, s, J


def sign_fix(U: np.ndarray) -> np.ndarray:
    """Signs (+1/-1 per column) that make each column's largest-magnitude
    entry positive; exact ties go to the lowest row index.  Zero columns
    keep +1."""
    idx = np.argmax(np.abs(U), axis=0)
    piv = U[idx, np.arange(U.shape[1])]
    return np.where(piv < 0, -1.0, 1.0)

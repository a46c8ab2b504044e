"""Randomized POD of a snapshot matrix partitioned by rows across ranks, in
FP64 (oracle; test infrastructure).

The algebra of Alg. 1 (Sec. 4.2) when each of R ranks holds a contiguous block
S_r of the rows of S (grid cells r0 .. r0 + n_r - 1) and all m snapshots:

    Lambda (m x l)            drawn by every rank from the same counters
    P_r = S_r Lambda          local
    QR of P (rows spread)     CholeskyQR2: G = sum_r P_r^T P_r (one sum over
                              ranks of an l x l matrix), R = chol(G),
                              Q_r = P_r R^-1; twice
    subspace iterations       Z = sum_r S_r^T Q_r (one sum of m x l), its QR
                              replicated on every rank, P_r = S_r Z, then the
                              distributed CholeskyQR2 again
    T = sum_r Q_r^T S_r       one sum of l x m
    SVD of T                  replicated (one-sided Jacobi)
    U_r = Q_r Uhat            local rows of U
    signs                     the largest-magnitude entry of every column of
                              the whole U (ties to the lowest global row) is
                              made positive: each rank offers its own
                              candidate, all ranks pick the same one
    C = sum_r U_r,k^T S_r     one sum of k x m (Sec. 4.3)

so a pass over S costs one reduction of its small result, as the GPU
library's single-device passes produce exactly these per-block partial
sums.  The QR of the subspace iterations is CholeskyQR2 where the
single-process oracle uses Householder QR: both give the same orthonormal
basis of the same span, up to the signs that the final sign rule removes.

Communication is passed in: allreduce(a) returns the elementwise sum over
ranks of the numpy array a (the same result on every rank) and
allgather(obj) returns the list of every rank's obj in rank order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .linalg import householder_qr, jacobi_svd
from .philox import gaussian_sketch


@dataclass
class ShardedResult:
    U: np.ndarray        # n_r x l: this rank's rows of U^r
    sigma: np.ndarray    # l singular values (replicated)
    V: np.ndarray        # m x l (replicated)
    Uhat: np.ndarray     # l x l (replicated)
    C: np.ndarray        # k x m modal coefficients (replicated)


def cholesky_qr2(P_r: np.ndarray, allreduce):
    """Orthonormal basis of the row-distributed P (this rank's rows P_r):
    two rounds of G = sum_r P_r^T P_r, R = chol(G) (upper), P_r <- P_r R^-1."""
    Q = np.asarray(P_r, dtype=np.float64)
    for _ in range(2):
        G = allreduce(Q.T @ Q)
        Rt = np.linalg.cholesky(G)                 # G = Rt Rt^T, R = Rt^T
        # Q <- Q R^-1, i.e. solve R^T X^T = Q^T
        Q = np.linalg.solve(Rt, Q.T).T
    return Q


def rpod_rows(S_r: np.ndarray, row0: int, k: int, p: int, q: int, seed: int,
              allreduce, allgather, stream: int = 0) -> ShardedResult:
    """Alg. 1 on the row block S_r (rows row0 .. row0 + n_r - 1 of S) of a
    matrix whose blocks are spread over the ranks of allreduce/allgather."""
    S_r = np.asarray(S_r, dtype=np.float64)
    n_r, m = S_r.shape
    l = k + p
    # Alg. 1, the sketch: the same counters on every rank
    Lam = gaussian_sketch(seed, m, l, stream)
    # Alg. 1, P = S Lambda (local rows) and its orthonormal basis
    Q = cholesky_qr2(S_r @ Lam, allreduce)
    # Alg. 1, subspace iterations with re-orthonormalisation
    for _ in range(q):
        Z, _ = householder_qr(allreduce(S_r.T @ Q))
        Q = cholesky_qr2(S_r @ Z, allreduce)
    # Alg. 1, T = Q^T S and its SVD (replicated)
    T = allreduce(Q.T @ S_r)
    V, sigma, Uhat = jacobi_svd(T.T)
    # Alg. 1, lift: this rank's rows of U
    U = Q @ Uhat
    # signs: per column the entry of largest magnitude over all ranks (ties
    # to the lowest global row) becomes positive
    cand = []
    for c in range(l):
        if n_r:
            i = int(np.argmax(np.abs(U[:, c])))
            cand.append((float(abs(U[i, c])), row0 + i, 1.0 if U[i, c] >= 0 else -1.0))
        else:
            cand.append((-1.0, 0, 1.0))
    offers = allgather(cand)
    sg = np.empty(l)
    for c in range(l):
        best = max((o[c] for o in offers), key=lambda t: (t[0], -t[1]))
        sg[c] = best[2]
    U = U * sg
    Uhat = Uhat * sg
    V = V * sg
    # Sec. 4.3: C = U_k^T S, one sum over the row blocks
    C = allreduce(U[:, :k].T @ S_r)
    return ShardedResult(U=U, sigma=sigma, V=V, Uhat=Uhat, C=C)

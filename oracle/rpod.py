"""Randomized POD, step by step in FP64 (oracle; test infrastructure).

Follows Alg. 1 of Sec. 4.2 (randomized POD with subspace iterations) in the
paper's notation: S is the N_C x N^s snapshot matrix (n x m here), N^r the
target rank (k), p the oversampling, q the number of subspace iterations,
l = N^r + p.

Readings of the paper (each listed in the design notes):
  * Lambda is N^s x (N^r + p) (the second definition in Sec. 4.2; the first one
    omits the oversampling).
  * The subspace iterations P <- (S S^T)^q P are carried out with an
    orthonormalisation after every product with S or S^T.  The span is the same
    in exact arithmetic; without it the columns of P collapse onto the leading
    singular vector in floating point.  Sec. 4.2 calls these subspace
    iterations and points to Gu (2015), where they are written this way.
  * The output dimension "N_h" of Alg. 1 is N_C, the number of grid cells.
  * Modal coefficients are C = U_{N^r}^T S (Sec. 4.3, the matrix below
    Eq. (psi_approx_snap_mu)), computed here literally from S.
  * Signs: column c of U is flipped so that its largest-magnitude entry is
    positive (exact ties to the lowest row); Uhat, V and C follow the flip.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .linalg import householder_qr, jacobi_svd, sign_fix
from .philox import gaussian_sketch


@dataclass
class RPODResult:
    U: np.ndarray        # n x l (all columns of U^r; the basis is U[:, :k])
    sigma: np.ndarray    # l singular values, descending
    V: np.ndarray        # m x l right singular vectors of T
    Uhat: np.ndarray     # l x l left singular vectors of T
    Q: np.ndarray        # n x l orthonormal basis of the sampled space
    T: np.ndarray        # l x m, T = Q^T S
    C: np.ndarray        # k x m modal coefficients U_k^T S
    Lam: np.ndarray      # m x l sketch
    k: int


def round_to(x: np.ndarray, dtype: str | None) -> np.ndarray:
    """Round FP64 values to bf16/fp16/fp32 and back (storage precision of a
    reduced-precision input); None leaves x unchanged."""
    if dtype is None or dtype == "f64":
        return x
    if dtype == "f32":
        return x.astype(np.float32).astype(np.float64)
    if dtype == "f16":
        return x.astype(np.float16).astype(np.float64)
    if dtype == "bf16":
        import torch
        return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).to(torch.float64).numpy()
    raise ValueError(dtype)


def rpod(S: np.ndarray, k: int, p: int, q: int, seed: int, stream: int = 0,
         Lam: np.ndarray | None = None, sketch_dtype: str | None = None,
         S_passes: np.ndarray | None = None) -> RPODResult:
    """Alg. 1 on S (n x m).  Returns U^r (n x l), Sigma^r, V^r and the modal
    coefficients.

    Lam: optional explicit sketch (default: the Philox sketch of `seed`,
    `stream`), rounded to `sketch_dtype` when given.  S_passes: the matrix
    read by the sketch and subspace-iteration products (default S); the
    precision forms pass a rounded copy here while T = Q^T S reads S itself."""
    S = np.asarray(S, dtype=np.float64)
    n, m = S.shape
    l = k + p
    if not (1 <= k and p >= 0 and q >= 0 and l <= min(n, m)):
        raise ValueError("need 1 <= k, p >= 0, q >= 0, k + p <= min(n, m)")
    Sp = S if S_passes is None else np.asarray(S_passes, dtype=np.float64)
    # Alg. 1, draw the Gaussian sketching matrix
    if Lam is None:
        Lam = gaussian_sketch(seed, m, l, stream)
    Lam = round_to(Lam, sketch_dtype)
    # Alg. 1, sampled matrix P = S Lambda, with an orthonormal basis of it
    P = Sp @ Lam
    Q, _ = householder_qr(P)
    # Alg. 1, q subspace iterations P <- (S S^T) P, orthonormalised after
    # each product
    for _ in range(q):
        Z, _ = householder_qr(Sp.T @ Q)
        Q, _ = householder_qr(Sp @ Z)
    # Alg. 1, T = Q^T S
    T = Q.T @ S
    # Alg. 1, SVD of T: one-sided Jacobi on T^T = V diag(sigma) Uhat^T
    V, sigma, Uhat = jacobi_svd(T.T)
    # Alg. 1, lift U^r = Q Uhat
    U = Q @ Uhat
    sg = sign_fix(U)
    U = U * sg
    Uhat = Uhat * sg
    V = V * sg
    # Sec. 4.3: modal coefficients C = U_{N^r}^T S
    C = U[:, :k].T @ S
    return RPODResult(U=U, sigma=sigma, V=V, Uhat=Uhat, Q=Q, T=T, C=C,
                      Lam=Lam, k=k)


def project(U: np.ndarray, S_new: np.ndarray) -> np.ndarray:
    """Galerkin projection of new snapshots on the basis: C' = U^T S'
    (Sec. 4.3, the coefficient matrix applied to held-out snapshots)."""
    return np.asarray(U, np.float64).T @ np.asarray(S_new, np.float64)


def pod(S: np.ndarray, N: int):
    """Deterministic POD, Eq. (svd): the first N left singular vectors and all
    singular values of S, by the one-sided Jacobi SVD (for small S only)."""
    S = np.asarray(S, dtype=np.float64)
    n, m = S.shape
    if n >= m:
        Ul, s, _ = jacobi_svd(S)
    else:
        _, s, Ul = jacobi_svd(S.T)
    Ul = Ul * sign_fix(Ul)
    return Ul[:, :N], s


def energy_rank(sigma: np.ndarray, delta: float) -> int:
    """Eq. (energy): the smallest N^r with sum_{i<=N} sigma_i / sum_i sigma_i
    >= delta, over the singular values given (descending).  The denominator
    is the last of the same sequential partial sums, so the ratio reaches
    exactly 1 at the end; a spectrum with no positive sum retains nothing and
    gives 0.  0 < delta <= 1 (the paper asks 0 < delta < 1)."""
    s = np.asarray(sigma, dtype=np.float64)
    if not 0.0 < delta <= 1.0:
        raise ValueError("delta must lie in (0, 1]")
    if s.size == 0:
        return 0
    c = np.cumsum(s)
    total = c[-1]
    if not total > 0.0:
        return 0
    for N in range(1, s.size + 1):
        if c[N - 1] / total >= delta:
            return N
    return s.size


def time_average(S: np.ndarray, nt: int) -> np.ndarray:
    """Time-averaged fields of Eq. (time_av), one per parameter sample.  The
    snapshot matrix holds M = m / nt samples of nt consecutive snapshots
    (the column order of the matrix after Eq. (fluct_psi): by sample, then
    time); column g of the n x M result is the mean of columns g*nt ..
    g*nt + nt - 1."""
    S = np.asarray(S, dtype=np.float64)
    n, m = S.shape
    if nt < 1 or m % nt != 0:
        raise ValueError("nt must divide the number of snapshots")
    M = m // nt
    out = np.empty((n, M))
    for g in range(M):
        out[:, g] = S[:, g * nt:(g + 1) * nt].sum(axis=1) / nt
    return out


def fluctuations(S: np.ndarray, nt: int):
    """Fluctuation snapshots of Eqs. (fluct_q), (fluct_psi): every snapshot
    minus the time average of its own parameter sample.  Returns (F, Sbar)
    with F n x m and Sbar the n x M time averages of Eq. (time_av)."""
    S = np.asarray(S, dtype=np.float64)
    Sbar = time_average(S, nt)
    return S - np.repeat(Sbar, nt, axis=1), Sbar


def max_principal_angle(A: np.ndarray, B: np.ndarray) -> float:
    """Largest principal angle between span(A) and span(B) (orthonormal
    columns, same count), as asin(||(I - A A^T) B||_2): accurate near zero."""
    R = B - A @ (A.T @ B)
    s = np.linalg.norm(R, 2) if R.size else 0.0
    return float(np.arcsin(min(1.0, s)))

"""Comparison helpers for GPU-vs-oracle rPOD tests (pure numpy)."""
import numpy as np


def sigma_close(sg, so, rel, abs_frac, floor=1e-3):
    """sigma_i agree to `rel` where sigma_i >= floor * sigma_1, else to
    abs_frac * sigma_1 (rounding in a Gram-based small SVD is absolute
    relative to sigma_1 there)."""
    sg = np.asarray(sg, np.float64)
    so = np.asarray(so, np.float64)
    s1 = so[0]
    big = so >= floor * s1
    err_rel = np.abs(sg[big] - so[big]) / so[big]
    err_abs = np.abs(sg[~big] - so[~big])
    ok = np.all(err_rel <= rel) and np.all(err_abs <= abs_frac * s1)
    return ok, (err_rel.max() if err_rel.size else 0.0), (err_abs.max() / s1 if err_abs.size else 0.0)


def max_angle(A, B):
    """Largest principal angle between the column spans of A and B (both
    with orthonormal columns), asin of ||(I - A A^T) B||_2."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    R = B - A @ (A.T @ B)
    return float(np.arcsin(min(1.0, np.linalg.norm(R, 2))))


def orth_err(U):
    U = np.asarray(U, np.float64)
    return float(np.abs(U.T @ U - np.eye(U.shape[1])).max())

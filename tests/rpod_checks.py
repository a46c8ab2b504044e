"""Comparison helpers for GPU-vs-oracle rPOD tests (pure numpy)."""
import numpy as np


# Below this fraction of sigma_1 the FP64 forms compare sigma_i absolutely:
# values there sit at the rounding level of S itself (a sampled direction
# of S below about u ||S|| is noise on both sides).
F64_FLOOR = 1e-9


def sigma_close(sg, so, rel, abs_frac, floor=1e-3):
    """sigma_i agree to `rel` where sigma_i >= floor * sigma_1, else to
    abs_frac * sigma_1.  The FP64 form is relatively accurate down to
    F64_FLOOR (Jacobi small SVD); the FP32 and 16-bit forms take their
    small SVD from eigenpairs of the Gram T T^T, whose rounding is absolute
    relative to sigma_1^2, so their tests keep the default floor."""
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

"""GPU tests of the small SVD's eigensolver on spectra with exact multiple
singular values (Alg. 1, SVD of T): the tridiagonal start must keep the
vectors of a multiple eigenvalue independent (clustered Gram-Schmidt, vector
replacement) and the Ogita-Aishima refinement must treat the cluster as one.

S = U0 diag(sigma) V0^T with random orthonormal U0, V0 and sigma made of
groups of equal values plus a distinct tail, exact rank J <= l, so Alg. 1
recovers the spectrum exactly (up to rounding).  Left singular vectors of a
multiple singular value are unique only as a subspace: the test compares
the span of every group, and the spans at the k boundary (which falls
between groups)."""
import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from tests.rpod_checks import max_angle, orth_err

pytestmark = pytest.mark.gpu

GROUPS = [(8.0, 3), (4.0, 4), (2.0, 5)]          # (value, multiplicity)
TAIL = [1.0, 0.5, 0.25, 0.125, 0.0625, 0.03125]  # distinct values


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def spectrum():
    s = []
    for v, mult in GROUPS:
        s += [v] * mult
    return np.array(s + TAIL)


def repeated_matrix(n, m, seed):
    rng = np.random.default_rng(seed)
    s = spectrum()
    J = s.size
    U0, _ = np.linalg.qr(rng.standard_normal((n, J)))
    V0, _ = np.linalg.qr(rng.standard_normal((m, J)))
    S = (U0 * s) @ V0.T
    return torch.from_numpy(S).t().contiguous().t(), U0, s


@pytest.mark.parametrize("compute,dtype,srel,ang", [
    ("f64", torch.float64, 1e-10, 1e-8),
    ("f32", torch.float32, 1e-5, 1e-4),
    ("bf16", torch.float32, 1e-3, 1e-2),
])
def test_multiple_singular_values(compute, dtype, srel, ang):
    n, m = 2048, 600
    S, U0, s = repeated_matrix(n, m, seed=5)
    J = s.size                     # 18
    k, p, q = 12, 8, 1             # k ends after the three groups; l = 20 > J
    flags = R.RPOD_FLAG_RETURN_ALL_L | (R.RPOD_FLAG_REFINE_FP32 if compute == "bf16" else 0)
    plan = R.Plan(n, m, k, p, q, seed=3, compute=compute, flags=flags)
    Sd = S.t().contiguous().to(dtype).cuda().t()
    U, sig, C = plan.basis(Sd)
    rc, _ = plan.status()
    assert rc == R.RPOD_OK, R.rpod_strerror(rc)
    sig = sig.cpu().numpy()
    Ug = U.double().cpu().numpy()
    # the spectrum, groups included; the l - J values beyond the rank vanish
    assert np.all(np.abs(sig[:J] - s) <= srel * s), np.abs(sig[:J] - s) / s
    assert np.all(sig[J:] <= max(srel, 1e-6) * s[0])
    # every group spans the right subspace, and so does U_k
    c = 0
    for v, mult in GROUPS:
        assert max_angle(U0[:, c:c + mult], Ug[:, c:c + mult]) <= ang, (v, mult)
        c += mult
    assert max_angle(U0[:, :k], Ug[:, :k]) <= ang
    # the distinct tail one vector at a time (FP64 and FP32 forms)
    if compute != "bf16":
        for i in range(c, J):
            assert max_angle(U0[:, i:i + 1], Ug[:, i:i + 1]) <= 10 * ang, i
    assert orth_err(Ug[:, :J]) <= (1e-12 if compute == "f64" else 1e-5)
    # coefficients C = U_k^T S
    Ck = C.double().cpu().numpy()
    ref = Ug[:, :k].T @ S.numpy()
    assert np.abs(Ck - ref).max() <= max(srel, 1e-6) * 10 * s[0]

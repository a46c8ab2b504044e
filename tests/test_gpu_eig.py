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


@pytest.mark.parametrize("compute,dtype,srel,ang", [
    ("f32", torch.float32, 1e-5, 1e-4),
    ("bf16", torch.float32, 1e-3, 1e-2),
])
@pytest.mark.parametrize("data_seed,sketch_seed", [(6, 1), (8, 2), (9, 3), (11, 5)])
def test_multiple_singular_values_orthonormal_over_seeds(compute, dtype, srel, ang, data_seed,
                                                         sketch_seed):
    """The small SVD of the FP32 and 16-bit forms on exactly multiple
    singular values, over several data and sketch seeds: the FP32 Gram
    splits each group by rounding alone (gaps near u_32 ||T||^2), where the
    eigenvector refinement must keep every pair of a group on its
    orthonormalizing update -- a pass that took such a pair as separated
    divides by a rounding-level gap.  Every group's span, the spectrum and
    the orthonormality of U are checked: 1e-5 for the FP32 form (two
    refinement passes); the 16-bit forms take one pass, which leaves an
    eigenvector error of about (u_32 ||A|| / gap)^2 -- here ||A||_F = 116
    and the smallest gap of the distinct tail 2.9e-3, about 6e-6 before the
    pass's constant -- so 5e-5 for them."""
    n, m = 2048, 600
    S, U0, s = repeated_matrix(n, m, seed=data_seed)
    J = s.size
    k, p, q = 12, 8, 1
    flags = R.RPOD_FLAG_RETURN_ALL_L | (R.RPOD_FLAG_REFINE_FP32 if compute == "bf16" else 0)
    plan = R.Plan(n, m, k, p, q, seed=sketch_seed, compute=compute, flags=flags)
    Sd = S.t().contiguous().to(dtype).cuda().t()
    U, sig, C = plan.basis(Sd)
    rc, _ = plan.status()
    assert rc == R.RPOD_OK, R.rpod_strerror(rc)
    sig = sig.cpu().numpy()
    Ug = U.double().cpu().numpy()
    assert np.all(np.abs(sig[:J] - s) <= srel * s)
    c = 0
    for v, mult in GROUPS:
        assert max_angle(U0[:, c:c + mult], Ug[:, c:c + mult]) <= ang, (v, mult)
        c += mult
    assert orth_err(Ug[:, :J]) <= (1e-5 if compute == "f32" else 5e-5)

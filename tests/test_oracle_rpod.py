"""Pins for the FP64 rPOD oracle (Alg. 1) against exact-rank recovery, brute
force, the closed-form spectrum of the synthetic recipe, orthonormality and
the randomized range-finder bound."""
import numpy as np
import pytest

from oracle.linalg import jacobi_svd
from oracle.rpod import energy_rank, max_principal_angle, pod, project, rpod
from synth import make_recipe, mode_matrix, snapshot_matrix, time_matrix


def _lowrank(n, m, J, seed, decay=0.5):
    rng = np.random.default_rng(seed)
    Uq, _ = np.linalg.qr(rng.standard_normal((n, J)))
    Vq, _ = np.linalg.qr(rng.standard_normal((m, J)))
    s = decay ** np.arange(J) * 10.0
    return Uq @ np.diag(s) @ Vq.T, Uq, s


@pytest.mark.parametrize("J,k,p,q", [(5, 5, 3, 1), (3, 6, 2, 0), (8, 8, 0, 2)])
def test_exact_rank_recovery(J, k, p, q):
    S, Uq, s = _lowrank(120, 90, J, seed=J + k)
    r = rpod(S, k, p, q, seed=3)
    assert np.allclose(r.sigma[:J], s, rtol=1e-12)
    assert np.all(r.sigma[J:] <= 1e-12 * s[0])
    assert max_principal_angle(r.U[:, :J], Uq) < 1e-12


@pytest.mark.parametrize("n,m", [(64, 48), (30, 45), (17, 17)])
def test_brute_force_full_rank(n, m):
    rng = np.random.default_rng(n * m)
    S = rng.standard_normal((n, m)) * np.logspace(0, -3, m)[None, :]
    l = min(n, m)
    r = rpod(S, l - 2, 2, 1, seed=1)
    Un, sn, _ = np.linalg.svd(S, full_matrices=False)
    assert np.allclose(r.sigma, sn, rtol=1e-11, atol=1e-14 * sn[0])
    # distinct singular values: each column equals numpy's up to sign
    for c in range(l):
        assert min(np.abs(r.U[:, c] - Un[:, c]).max(),
                   np.abs(r.U[:, c] + Un[:, c]).max()) < 1e-9


def test_closed_form_spectrum_exact_rank():
    # J = 15 modes <= l: rPOD is exact; the DST-II orthogonality of the modes
    # gives sv(S) = sqrt(n)/2 * sv(diag(amp) A^T)
    rec = make_recipe(16, 16, 200, 15, ("power", 1.5), seed=4, noise=0.0)
    S = snapshot_matrix(rec, noise=False).numpy()
    closed = np.sqrt(rec.n) / 2 * np.linalg.svd(
        (time_matrix(rec) * rec.amp[None, :]).T, compute_uv=False)
    r = rpod(S, 10, 10, 1, seed=0)
    assert np.allclose(r.sigma[:15], closed, rtol=1e-11)
    assert np.all(r.sigma[15:] < 1e-12 * closed[0])


def test_modes_discretely_orthogonal():
    rec = make_recipe(12, 20, 10, 60, seed=0, noise=0.0)
    phi = mode_matrix(rec)
    G = phi.T @ phi
    assert np.abs(G - np.eye(rec.J) * rec.n / 4).max() < 1e-11


def test_project_recovers_recipe_coefficients():
    """Galerkin projection against the recipe's closed form: the sine modes
    satisfy Phi^T Phi = (n/4) I, so with U = (2/sqrt(n)) Phi and the
    noise-free S = Phi (amp * A)^T the projection U^T S is
    (sqrt(n)/2) amp_j cos(omega_j t_p + theta_j); a transposed operand or a
    missing scale fails it."""
    rec = make_recipe(16, 24, 37, 30, ("power", 1.0), seed=3, noise=0.0)
    S = snapshot_matrix(rec, noise=False).numpy()
    U = mode_matrix(rec) * (2.0 / np.sqrt(rec.n))
    t = rec.times()
    closed = (np.sqrt(rec.n) / 2) * rec.amp[:, None] * np.cos(
        np.outer(rec.omega, t) + rec.theta[:, None])
    C = project(U, S)
    assert C.shape == (rec.J, rec.m)
    assert np.abs(C - closed).max() <= 1e-12 * np.abs(closed).max()
    # a subset of snapshots projects to the same columns
    assert np.abs(project(U, S[:, 5:9]) - closed[:, 5:9]).max() <= 1e-12 * np.abs(closed).max()


def test_closed_form_spectrum_with_truncation():
    # more modes than l: the leading sigma still converge to the closed form
    rec = make_recipe(32, 32, 400, 200, ("exp", 10.0), seed=1, noise=1e-6)
    S = snapshot_matrix(rec).numpy()
    closed = np.sqrt(rec.n) / 2 * np.linalg.svd(
        (time_matrix(rec) * rec.amp[None, :]).T, compute_uv=False)
    r = rpod(S, 10, 10, 2, seed=0)
    noise_bound = 1e-6 * (np.sqrt(rec.n) + np.sqrt(rec.m)) * 3   # Weyl + slack
    assert np.all(np.abs(r.sigma[:10] - closed[:10]) <= 1e-6 * closed[:10] + noise_bound)


def test_orthonormality_and_coefficients():
    rec = make_recipe(20, 20, 150, 100, ("power", 1.5), seed=2)
    S = snapshot_matrix(rec).numpy()
    r = rpod(S, 8, 6, 1, seed=5)
    l = 14
    assert np.abs(r.U.T @ r.U - np.eye(l)).max() < 1e-13
    assert np.abs(r.Uhat.T @ r.Uhat - np.eye(l)).max() < 1e-13
    # literal C = U_k^T S equals Sigma_k V_k^T from the SVD of T
    C2 = np.diag(r.sigma[:8]) @ r.V[:, :8].T
    assert np.abs(r.C - C2).max() < 1e-12 * r.sigma[0]
    # U Sigma V^T reproduces Q Q^T S
    assert np.abs(r.U @ np.diag(r.sigma) @ r.V.T - r.Q @ (r.Q.T @ S)).max() < 1e-12 * r.sigma[0]
    assert np.allclose(project(r.U[:, :8], S), r.C, atol=1e-12 * r.sigma[0])
    # sign convention: largest-magnitude entry of each column is positive
    idx = np.argmax(np.abs(r.U), axis=0)
    assert np.all(r.U[idx, np.arange(l)] > 0)


def test_range_finder_bound():
    # Halko, Martinsson & Tropp (2011) Thm 10.5, q = 0:
    # E ||(I - QQ^T) S||_F <= (1 + k/(p-1))^(1/2) (sum_{j>k} sigma_j^2)^(1/2)
    rng = np.random.default_rng(0)
    n, m, k, p = 150, 120, 6, 4
    Uq, _ = np.linalg.qr(rng.standard_normal((n, m)))
    Vq, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = 0.7 ** np.arange(m)
    S = Uq @ np.diag(s) @ Vq.T
    tail = np.sqrt(np.sum(s[k:] ** 2))
    bound = np.sqrt(1 + k / (p - 1)) * tail
    errs = {0: [], 1: [], 2: []}
    for seed in range(50):
        for q in errs:
            r = rpod(S, k, p, q, seed=seed)
            E = S - r.Q @ (r.Q.T @ S)
            errs[q].append(np.linalg.norm(E))
    for q in errs:
        # Q has l = k + p columns: the optimal rank-l error is a floor
        assert np.all(np.array(errs[q]) >= np.sqrt(np.sum(s[k + p:] ** 2)) * (1 - 1e-12))
        assert max(errs[q]) <= 10 * bound
    assert np.mean(errs[0]) <= bound
    assert np.mean(errs[1]) <= np.mean(errs[0]) and np.mean(errs[2]) <= np.mean(errs[1])


def test_error_falls_with_oversampling():
    rec = make_recipe(24, 24, 300, 200, ("exp", 20.0), seed=3)
    S = snapshot_matrix(rec).numpy()
    sn = np.linalg.svd(S, compute_uv=False)
    errs = []
    for p in (0, 5, 20, 50):
        e = np.mean([np.abs(rpod(S, 10, p, 0, seed=s).sigma[:10] - sn[:10]).max()
                     for s in range(5)])
        errs.append(e)
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_reduced_precision_passes_hook():
    rng = np.random.default_rng(8)
    S = rng.standard_normal((40, 30))
    a = rpod(S, 4, 3, 1, seed=2)
    b = rpod(S, 4, 3, 1, seed=2, S_passes=S.copy())
    assert np.array_equal(a.sigma, b.sigma)


def test_pod_matches_numpy_and_energy_rank():
    rng = np.random.default_rng(9)
    S = rng.standard_normal((30, 50))
    U, s = pod(S, 5)
    sn = np.linalg.svd(S, compute_uv=False)
    assert np.allclose(s, sn, rtol=1e-13)
    assert np.abs(U.T @ U - np.eye(5)).max() < 1e-13
    assert energy_rank(np.array([4.0, 3.0, 2.0, 1.0]), 0.7) == 2
    assert energy_rank(np.array([4.0, 3.0, 2.0, 1.0]), 0.75) == 3
    assert energy_rank(np.array([4.0, 3.0, 2.0, 1.0]), 0.4) == 1


def test_argument_checks():
    with pytest.raises(ValueError):
        rpod(np.zeros((10, 5)), 4, 2, 1, seed=0)


def test_error_falls_with_faster_decay():
    # Sec. 5: modes of a field with faster-decaying singular values are
    # reproduced more accurately (the stream function against the vorticity);
    # as a property of Alg. 1: with geometric spectra decay^j (plus a flat
    # tail) and q = 0, the subspace error of U_k falls as the decay steepens,
    # on average over seeds
    n, m, k, p = 160, 120, 6, 4
    means = []
    for decay in (0.95, 0.8, 0.6):
        errs = []
        for seed in range(8):
            rng = np.random.default_rng(100 + seed)
            Uq, _ = np.linalg.qr(rng.standard_normal((n, m)))
            Vq, _ = np.linalg.qr(rng.standard_normal((m, m)))
            s = decay ** np.arange(m) + 1e-3
            S = (Uq * s) @ Vq.T
            r = rpod(S, k, p, 0, seed=seed)
            errs.append(max_principal_angle(Uq[:, :k], r.U[:, :k]))
        means.append(float(np.mean(errs)))
    assert means[0] > means[1] > means[2], means

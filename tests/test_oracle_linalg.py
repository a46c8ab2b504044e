"""Pins for the oracle's Householder QR and one-sided Jacobi SVD (Alg. 1,
fourth and sixth steps) against numpy.linalg and exact identities."""
import numpy as np
import pytest

from oracle.linalg import NoConvergence, householder_qr, jacobi_svd, sign_fix

SHAPES = [(1, 1), (5, 1), (6, 6), (40, 13), (64, 64), (300, 30)]


@pytest.mark.parametrize("shape", SHAPES)
def test_householder_qr(shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    Q, R = householder_qr(A)
    n, l = shape
    assert np.allclose(R, np.triu(R))
    assert np.abs(Q.T @ Q - np.eye(l)).max() < 1e-14
    assert np.abs(Q @ R - A).max() < 1e-14 * np.abs(A).max() * np.sqrt(n)
    Rn = np.linalg.qr(A)[1]
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rn)), rtol=1e-12)


def test_householder_qr_rank_deficient():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((50, 4))
    A = np.concatenate([B, B[:, :2] * 2.0, np.zeros((50, 2))], axis=1)
    Q, R = householder_qr(A)
    assert np.abs(Q.T @ Q - np.eye(8)).max() < 1e-14
    assert np.abs(Q @ R - A).max() < 1e-13


@pytest.mark.parametrize("shape", SHAPES)
def test_jacobi_svd_matches_numpy(shape):
    rng = np.random.default_rng(7 + sum(shape))
    A = rng.standard_normal(shape)
    Ul, s, V = jacobi_svd(A)
    sn = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, sn, rtol=1e-13, atol=1e-14 * sn[0])
    assert np.all(np.diff(s) <= 0)
    l = shape[1]
    tol = max(1e-14, 2e-15 * l)   # rounding grows with the number of rotations
    assert np.abs(V.T @ V - np.eye(l)).max() < tol
    assert np.abs(Ul.T @ Ul - np.eye(l)).max() < 10 * tol
    assert np.abs(Ul @ np.diag(s) @ V.T - A).max() < 1e-14 * np.sqrt(l) * s[0] * 10


def test_jacobi_svd_graded_relative_accuracy():
    # A = X D with well-conditioned X: one-sided Jacobi gets every singular
    # value to high relative accuracy (Demmel & Veselic 1992)
    rng = np.random.default_rng(11)
    X, _ = np.linalg.qr(rng.standard_normal((60, 20)))
    d = np.logspace(0, -12, 20)
    A = X @ np.diag(d)
    _, s, _ = jacobi_svd(A)
    assert np.allclose(s, d, rtol=1e-12, atol=0)


def test_jacobi_svd_known_2x2():
    # [[3, 0], [4, 5]] has singular values sqrt(45) and sqrt(5)
    _, s, _ = jacobi_svd(np.array([[3.0, 0.0], [4.0, 5.0]]))
    assert s == pytest.approx([np.sqrt(45.0), np.sqrt(5.0)], rel=1e-15)


def test_jacobi_svd_rank_deficient_and_zero():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((30, 3))
    A = np.concatenate([B, B @ rng.standard_normal((3, 2)), np.zeros((30, 1))], axis=1)
    Ul, s, V = jacobi_svd(A)
    sn = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:3], sn[:3], rtol=1e-13)
    assert np.all(s[3:] < 1e-13 * s[0])
    assert np.abs(V.T @ V - np.eye(6)).max() < 1e-14
    assert np.abs(Ul @ np.diag(s) @ V.T - A).max() < 1e-13 * s[0]


def test_jacobi_svd_sweep_cap():
    rng = np.random.default_rng(2)
    with pytest.raises(NoConvergence):
        jacobi_svd(rng.standard_normal((20, 10)), max_sweeps=1)


def test_sign_fix():
    U = np.array([[0.1, -0.9, 0.0], [-0.8, 0.2, 0.0], [0.3, 0.9, 0.0]])
    assert sign_fix(U).tolist() == [-1.0, -1.0, 1.0]

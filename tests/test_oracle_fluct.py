"""Pins for the oracle's time averages and fluctuations (Eqs. (time_av),
(fluct_q)) and energy-based rank (Eq. (energy)): an exactly representable
construction with known means, the special cases that reduce to numpy's mean
or to the identity, the invariants of the decomposition, and closed-form
ranks."""
import numpy as np
import pytest

from oracle.rpod import energy_rank, fluctuations, time_average


def exact_construction(n, nt, M, seed):
    """S = A E^T + F0 with integer A and integer F0 whose columns sum to zero
    within every group of nt snapshots (nt a power of two: every mean exact)."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-50, 50, (n, M)).astype(np.float64)
    F0 = np.empty((n, nt * M))
    for g in range(M):
        v = rng.integers(-20, 20, (n, nt)).astype(np.float64)
        v[:, -1] = -v[:, :-1].sum(axis=1)
        F0[:, g * nt:(g + 1) * nt] = v
    return np.repeat(A, nt, axis=1) + F0, A, F0


@pytest.mark.parametrize("n,nt,M", [(7, 8, 5), (3, 1, 4), (16, 32, 2), (1, 4, 1)])
def test_exact_means_and_fluctuations(n, nt, M):
    S, A, F0 = exact_construction(n, nt, M, seed=n * nt + M)
    F, Sbar = fluctuations(S, nt)
    assert np.array_equal(time_average(S, nt), A)
    assert np.array_equal(Sbar, A)
    assert np.array_equal(F, F0)


def test_one_sample_is_numpy_mean_and_nt_one_is_identity():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((40, 33)) * 3.0 + 1.0
    Sbar = time_average(S, 33)
    assert Sbar.shape == (40, 1)
    assert np.allclose(Sbar[:, 0], np.mean(S, axis=1), rtol=1e-15, atol=1e-15)
    F, Sbar1 = fluctuations(S, 1)
    assert np.array_equal(Sbar1, S)
    assert np.array_equal(F, np.zeros_like(S))


def test_invariants_random():
    rng = np.random.default_rng(2)
    nt, M = 7, 6
    S = rng.standard_normal((25, nt * M)) + rng.standard_normal((25, 1)) * 10
    F, Sbar = fluctuations(S, nt)
    # every sample's fluctuations average to zero, and S = F + Sbar E^T
    for g in range(M):
        assert np.abs(F[:, g * nt:(g + 1) * nt].sum(axis=1)).max() < 1e-12
        # the mean of a sample lies within that sample's range
        blk = S[:, g * nt:(g + 1) * nt]
        assert np.all(Sbar[:, g] >= blk.min(axis=1)) and np.all(Sbar[:, g] <= blk.max(axis=1))
    assert np.abs(F + np.repeat(Sbar, nt, axis=1) - S).max() < 1e-13


def test_argument_checks():
    with pytest.raises(ValueError):
        time_average(np.zeros((3, 10)), 3)
    with pytest.raises(ValueError):
        time_average(np.zeros((3, 10)), 0)
    with pytest.raises(ValueError):
        energy_rank(np.ones(3), 0.0)


def test_energy_rank_closed_forms():
    # equal singular values: the ratio after N of l values is N / l
    l = 10
    for delta, want in [(0.5, 5), (0.55, 6), (0.05, 1), (1.0, 10), (0.91, 10)]:
        assert energy_rank(np.ones(l), delta) == want
    # geometric spectrum 2^-i: partial sums 2 - 2^(1-N) over the total
    s = 0.5 ** np.arange(8)
    total = 2 - 2.0 ** -7
    for N in range(1, 9):
        ratio = (2 - 2.0 ** (1 - N)) / total
        assert energy_rank(s, ratio) == N
    # trailing zeros are never needed; a zero spectrum retains nothing
    assert energy_rank(np.array([3.0, 1.0, 0.0, 0.0]), 1.0) == 2
    assert energy_rank(np.zeros(5), 0.9) == 0
    assert energy_rank(np.array([4.0, 3.0, 2.0, 1.0]), 0.7) == 2

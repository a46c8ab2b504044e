"""Pins for the oracle's Philox4x64-10 and Gaussian sketch (Alg. 1, first step)."""
import numpy as np
import pytest

from oracle.philox import box_muller, gaussian_sketch, mulhilo64, philox4x64


def test_mulhilo64_matches_python_bigints():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**63, 500, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    b = rng.integers(0, 2**63, 500, dtype=np.uint64) * np.uint64(2)
    a[:3] = [2**64 - 1, 0, 1]
    b[:3] = [2**64 - 1, 2**64 - 1, 2**64 - 1]
    hi, lo = mulhilo64(a, b)
    for x, y, h, l in zip(a.tolist(), b.tolist(), hi.tolist(), lo.tolist()):
        p = x * y
        assert h == p >> 64 and l == p & (2**64 - 1)


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (2**64 - 1,) * 4),                 # wraps to the all-zero counter
    ((5, 7), (3, 1, 0, 0)),
    ((0xDEADBEEF, 2**63 + 11), (17, 2**40 + 3, 9, 2**64 - 5)),
    ((123456789, 0), (0, 16, 0, 0)),
])
def test_raw_words_match_numpy_philox(key, ctr):
    # numpy's Philox is Philox4x64-10; it increments word 0 of the counter
    # (with carry) before each block, so its first block is f(ctr + 1).
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    ref = bg.random_raw(12).reshape(3, 4)
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    for blk in range(3):
        cc = (c + 1 + blk) % 2**256
        words = [(cc >> (64 * i)) & (2**64 - 1) for i in range(4)]
        out = philox4x64(np.array(words, dtype=np.uint64), np.array(key, dtype=np.uint64))
        assert out.tolist() == ref[blk].tolist()


def test_round_count_matters():
    k = np.array([1, 2], dtype=np.uint64)
    c = np.array([3, 4, 5, 6], dtype=np.uint64)
    assert philox4x64(c, k, 10).tolist() != philox4x64(c, k, 7).tolist()


def test_box_muller_extremes():
    z0, z1 = box_muller(np.array([2**64 - 1], np.uint64), np.array([0], np.uint64))
    # u1 = 1 -> radius 0
    assert z0[0] == 0.0 and z1[0] == 0.0
    z0, z1 = box_muller(np.array([0], np.uint64), np.array([0], np.uint64))
    # u1 = 2^-53, angle 0: z0 = sqrt(2*53*ln 2), z1 = 0
    assert z0[0] == pytest.approx(np.sqrt(2 * 53 * np.log(2.0)), rel=1e-15)
    assert z1[0] == 0.0


def test_sketch_moments():
    lam = gaussian_sketch(seed=42, m=5003, l=200, stream=0)
    z = lam.ravel()
    N = z.size
    assert abs(z.mean()) < 5 / np.sqrt(N)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / N)
    assert abs(np.mean(z**3)) < 5 * np.sqrt(15.0 / N)
    assert abs(np.mean(z**4) - 3.0) < 5 * np.sqrt(96.0 / N)
    # tail mass beyond 3 sigma
    assert abs(np.mean(np.abs(z) > 3.0) - 0.0026998) < 5 * np.sqrt(0.0027 / N)


def test_sketch_element_counter_layout():
    m, l, seed, stream = 7, 3, 9, 5
    lam = gaussian_sketch(seed, m, l, stream)
    assert lam.shape == (m, l)
    for j in range(l):
        for i in range(m):
            e = i + j * m
            w = philox4x64(np.array([e // 2, stream, 0, 0], np.uint64),
                           np.array([seed, 0], np.uint64))
            z0, z1 = box_muller(w[0:1], w[1:2])
            assert lam[i, j] == (z0[0] if e % 2 == 0 else z1[0])


def test_streams_and_seeds_are_independent():
    a = gaussian_sketch(1, 100, 10, 0)
    b = gaussian_sketch(1, 100, 10, 1)
    c = gaussian_sketch(2, 100, 10, 0)
    assert abs(np.corrcoef(a.ravel(), b.ravel())[0, 1]) < 0.15
    assert abs(np.corrcoef(a.ravel(), c.ravel())[0, 1]) < 0.15

"""Philox4x64-10 and the Gaussian sketch matrix Lambda (oracle; test infrastructure).

Alg. 1 (first step) draws Lambda in R^{N^s x (N^r + p)} with i.i.d. N(0, 1)
entries; the paper fixes nothing else.  To let the GPU path and this oracle use
the *same* Lambda without passing it between them, each implements one
counter-based generator from its published definition:

  Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11): per round the two 64x64 -> 128-bit
  products of the first and third counter words with the multipliers M0, M1,
  the outputs (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), and the key bumped by
  the Weyl constants W0, W1 between rounds.

Element e = i + j*m (column-major index into the m x l matrix) takes the
counter (floor(e/2), stream, 0, 0) under the key (seed, 0).  From the first two
64-bit output words w0, w1:

  u1 = ((w0 >> 11) + 1) * 2^-53   in (0, 1]
  u2 = (w1 >> 11) * 2^-53         in [0, 1)
  z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2)

(Box and Muller 1958); even e takes z0, odd e takes z1.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def mulhilo64(a, b):
    """(hi, lo) 64-bit halves of the 128-bit product a*b, elementwise on uint64
    arrays, by 32-bit limbs."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a0, a1 = a & _MASK32, a >> _S32
    b0, b1 = b & _MASK32, b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _MASK32) + (p10 & _MASK32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64(counter, key, rounds: int = 10):
    """Philox4x64-`rounds` block function.  counter: (..., 4) uint64,
    key: (..., 2) uint64 (broadcast).  Returns (..., 4) uint64."""
    c = np.array(counter, dtype=np.uint64, copy=True)
    k = np.array(key, dtype=np.uint64, copy=True)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = mulhilo64(M0, c0)
            hi1, lo1 = mulhilo64(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack(np.broadcast_arrays(c0, c1, c2, c3), axis=-1)


def box_muller(w0, w1):
    """Two standard normals from two 64-bit words (top 53 bits of each)."""
    u1 = ((np.asarray(w0, np.uint64) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (np.asarray(w1, np.uint64) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def gaussian_sketch(seed: int, m: int, l: int, stream: int = 0) -> np.ndarray:
    """Lambda (m x l, FP64) of Alg. 1, first step: i.i.d. N(0, 1) entries,
    entry (i, j) from element counter e = i + j*m as described above."""
    e = np.arange(m * l, dtype=np.uint64)
    pairs = np.unique(e >> np.uint64(1))
    ctr = np.zeros((len(pairs), 4), dtype=np.uint64)
    ctr[:, 0] = pairs
    ctr[:, 1] = np.uint64(stream)
    key = np.array([seed, 0], dtype=np.uint64)
    w = philox4x64(ctr, key)
    z0, z1 = box_muller(w[:, 0], w[:, 1])
    z = np.empty(2 * len(pairs), dtype=np.float64)
    z[0::2] = z0
    z[1::2] = z1
    return z[: m * l].reshape(l, m).T.copy()   # column-major fill order

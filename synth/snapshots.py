"""Synthetic snapshot matrices that stand in for the paper's 2QGE snapshot data.

The paper's snapshot matrix S_Phi (Sec. 4.1, the matrix after Eq. (fluct_psi))
holds N^s = M * N^t fluctuation snapshots of one field on an N_C-cell grid,
column j = (k-1) N^t + p for parameter sample k and time t_p.  The paper's
data is not public, so every input here is synthetic with the same shape:

    S[:, p] = sum_j  amp_j * cos(omega_j t_p + theta_j) * phi_j  + eps * N(0, 1)

on the cell centres of an nx-by-ny grid over the rectangle [0, 1] x [0, 2]
(the paper's gyre domain [0, 1] x [-1, 1], shifted), with

    phi_j(x, y) = sin(pi a_j x) sin(pi b_j y / 2),
    x_i = (i + 1/2) / nx,  y_r = 2 (r + 1/2) / ny,  row index = i + nx * r,

the modes (a, b) ordered by the Laplacian eigenvalue a^2 + (b/2)^2 (ties by a,
then b), a < nx and b < ny.  On this grid the phi_j are discretely orthogonal
(a DST-II basis) with squared norm nx*ny/4, so the noise-free matrix has the
singular values (sqrt(n)/2) * sv(diag(amp) A^T), A[p, j] = cos(omega_j t_p +
theta_j): a closed form the tests use to pin the oracle.

Random draws come from numpy's Philox bit generator keyed by (seed, stream):
stream 1 for omega, 2 for theta, 3 for the noise, 16 + b for instance b of a
batch.  On a CUDA device the noise comes from torch's generator instead (the
matrix there is too large for a host round trip); tests that compare the GPU
path with the oracle build their inputs on the host.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

STREAM_OMEGA = 1
STREAM_THETA = 2
STREAM_NOISE = 3
STREAM_INSTANCE0 = 16


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(
        np.random.Philox(key=np.array([seed, stream], dtype=np.uint64)))


def mode_pairs(nx: int, ny: int, J: int) -> np.ndarray:
    """First J mode index pairs (a, b), 1 <= a < nx, 1 <= b < ny, ordered by
    a^2 + (b/2)^2 ascending, ties broken by a then b.  Returns int64 (J, 2)."""
    if J > (nx - 1) * (ny - 1):
        raise ValueError("more modes requested than the grid resolves")
    # the J smallest eigenvalues use a, b below about sqrt(J) * const; search
    # a generous box, then sort exactly in integers: key = 4a^2 + b^2
    amax = min(nx - 1, int(math.isqrt(4 * J)) + 4)
    bmax = min(ny - 1, 2 * amax + 4)
    a, b = np.meshgrid(np.arange(1, amax + 1), np.arange(1, bmax + 1),
                       indexing="ij")
    a, b = a.ravel(), b.ravel()
    key = 4 * a * a + b * b
    order = np.lexsort((b, a, key))
    pairs = np.stack([a[order], b[order]], axis=1)[:J]
    if len(pairs) < J:
        raise ValueError("mode search box too small")
    return pairs.astype(np.int64)


@dataclass
class ModeRecipe:
    """Parameters of one synthetic snapshot matrix (n = nx*ny rows, m columns)."""
    nx: int
    ny: int
    m: int
    amp: np.ndarray          # (J,) mode amplitudes sigma_j (times any scale)
    omega: np.ndarray        # (J,) angular frequencies
    theta: np.ndarray        # (J,) phases
    pairs: np.ndarray        # (J, 2) mode indices (a, b)
    seed: int = 0
    noise: float = 1e-6
    dt: float = 0.1
    t0: float = 0.0
    noise_stream: int = STREAM_NOISE
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def J(self) -> int:
        return len(self.amp)

    def times(self) -> np.ndarray:
        return self.t0 + self.dt * np.arange(self.m, dtype=np.float64)


def _decay(J: int, decay) -> np.ndarray:
    j = np.arange(1, J + 1, dtype=np.float64)
    kind, val = decay
    if kind == "power":
        return j ** (-float(val))
    if kind == "exp":
        return np.exp(-j / float(val))
    raise ValueError(f"unknown decay {decay!r}")


def make_recipe(nx: int, ny: int, m: int, J: int, decay=("power", 1.5),
                seed: int = 0, noise: float = 1e-6, dt: float = 0.1,
                omega_range=(0.1, 2.0), stream_offset: int = 0) -> ModeRecipe:
    """The base recipe: amp_j from `decay` (("power", a): j^-a, ("exp", tau):
    exp(-j/tau)), omega_j ~ U(omega_range), theta_j ~ U(0, 2 pi)."""
    J = min(J, (nx - 1) * (ny - 1))
    pairs = mode_pairs(nx, ny, J)
    omega = _rng(seed, STREAM_OMEGA + stream_offset).uniform(
        omega_range[0], omega_range[1], J)
    theta = _rng(seed, STREAM_THETA + stream_offset).uniform(0.0, 2 * np.pi, J)
    return ModeRecipe(nx=nx, ny=ny, m=m, amp=_decay(J, decay), omega=omega,
                      theta=theta, pairs=pairs, seed=seed, noise=noise, dt=dt,
                      noise_stream=STREAM_NOISE + stream_offset)


def parametric_recipe(nx: int, ny: int, m: int, J: int, mu, seed: int = 0,
                      noise: float = 1e-6, dt: float = 0.1,
                      noise_stream: int = STREAM_NOISE) -> ModeRecipe:
    """Recipe for one physical-parameter sample mu in [0, 1]^4:
    amp_j = (0.5 + mu_4) j^-(1 + mu_1), omega_j = omega0_j (0.5 + mu_2),
    theta_j = theta0_j + 2 pi mu_3, with omega0, theta0 drawn once from `seed`."""
    mu = np.asarray(mu, dtype=np.float64)
    base = make_recipe(nx, ny, m, J, ("power", 1.0 + mu[0]), seed=seed,
                       noise=noise, dt=dt)
    base.amp = base.amp * (0.5 + mu[3])
    base.omega = base.omega * (0.5 + mu[1])
    base.theta = base.theta + 2 * np.pi * mu[2]
    base.noise_stream = noise_stream
    base.extra["mu"] = mu
    return base


def batched_recipes(count: int = 64, nx: int = 128, ny: int = 256,
                    m_range=(500, 3000), k_choices=(10, 20, 30, 50),
                    tau_range=(5.0, 30.0), J: int = 200, seed: int = 0,
                    noise: float = 1e-6):
    """`count` independent instances (4 fields x 16 parameter samples by
    default): m_b ~ U{m_range}, k_b uniform over k_choices, amp_j =
    exp(-j/tau_b) with tau_b ~ U(tau_range).  Returns (recipes, ks)."""
    rng = _rng(seed, STREAM_INSTANCE0 - 1)
    ms = rng.integers(m_range[0], m_range[1] + 1, count)
    ks = rng.choice(np.asarray(k_choices), count)
    taus = rng.uniform(tau_range[0], tau_range[1], count)
    recs = []
    for b in range(count):
        off = STREAM_INSTANCE0 + 4 * b
        recs.append(make_recipe(nx, ny, int(ms[b]), J, ("exp", taus[b]),
                                seed=seed, noise=noise, stream_offset=off))
    return recs, [int(k) for k in ks]


def mode_matrix(rec: ModeRecipe) -> np.ndarray:
    """Phi (n x J), column j = phi_j at the cell centres, row i + nx*r."""
    x = (np.arange(rec.nx) + 0.5) / rec.nx
    y = 2.0 * (np.arange(rec.ny) + 0.5) / rec.ny
    a = rec.pairs[:, 0].astype(np.float64)
    b = rec.pairs[:, 1].astype(np.float64)
    sx = np.sin(np.pi * np.outer(x, a))          # (nx, J)
    sy = np.sin(np.pi * np.outer(y, b) / 2.0)    # (ny, J)
    return (sy[:, None, :] * sx[None, :, :]).reshape(rec.n, rec.J)


def steady_field(nx: int, ny: int, mu, amp: float = 1.0) -> np.ndarray:
    """A time-independent, parameter-dependent field standing in for the
    time-averaged part of the flow (the paper's snapshots have one; the
    oscillating recipe above averages to about zero):
    amp * [(1 + mu_1) phi_(1,1) + (0.5 + mu_2) phi_(1,2) + (0.25 + mu_3) phi_(2,1)]
    with phi_(a,b)(x, y) = sin(pi a x) sin(pi b y / 2) on the recipe's cell
    centres, as an n-vector (row i + nx * r)."""
    mu = np.asarray(mu, dtype=np.float64)
    x = (np.arange(nx) + 0.5) / nx
    y = 2.0 * (np.arange(ny) + 0.5) / ny

    def phi(a, b):
        return (np.sin(np.pi * b * y / 2.0)[:, None] * np.sin(np.pi * a * x)[None, :]).reshape(-1)

    return amp * ((1.0 + mu[0]) * phi(1, 1) + (0.5 + mu[1]) * phi(1, 2) + (0.25 + mu[2]) * phi(2, 1))


def time_matrix(rec: ModeRecipe) -> np.ndarray:
    """A (m x J), A[p, j] = cos(omega_j t_p + theta_j)."""
    return np.cos(np.outer(rec.times(), rec.omega) + rec.theta[None, :])


def snapshot_matrix(rec: ModeRecipe, device="cpu", dtype=torch.float64,
                    noise: bool = True, chunk_cols: int = 512, rows=None) -> torch.Tensor:
    """The n x m snapshot matrix as a column-major torch tensor (shape (n, m),
    strides (1, n)): each snapshot is contiguous.

    On the host it is computed in FP64 with numpy Philox noise and cast to
    `dtype`; `rows` (host only) keeps a subset of the grid cells (the noise is
    then drawn for the subset alone).  On a CUDA device it is built there by
    torch (FP32 products unless dtype is float64) with torch-generated noise,
    `chunk_cols` snapshots at a time so that no temporary of the full size is
    made."""
    device = torch.device(device)
    phi = mode_matrix(rec)                         # (n, J)
    if rows is not None:
        if device.type != "cpu":
            raise ValueError("row subsets are generated on the host")
        phi = phi[rows]
    coef = time_matrix(rec) * rec.amp[None, :]     # (m, J)
    if device.type == "cpu":
        st = coef @ phi.T                          # (m, n) row-major == S col-major
        if noise and rec.noise:
            st += rec.noise * _rng(rec.seed, rec.noise_stream).standard_normal(st.shape)
        return torch.from_numpy(st).to(dtype).t()
    wdt = torch.float64 if dtype == torch.float64 else torch.float32
    phi_t = torch.from_numpy(phi.T.copy()).to(device=device, dtype=wdt)   # (J, n)
    coef_t = torch.from_numpy(coef).to(device=device, dtype=wdt)          # (m, J)
    st = torch.empty((rec.m, rec.n), device=device, dtype=dtype)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rec.seed) * 1000003 + int(rec.noise_stream))
    for c0 in range(0, rec.m, chunk_cols):
        c1 = min(rec.m, c0 + chunk_cols)
        blk = coef_t[c0:c1] @ phi_t
        if noise and rec.noise:
            blk += rec.noise * torch.randn(blk.shape, device=device, dtype=wdt,
                                           generator=gen)
        st[c0:c1] = blk.to(dtype)
    del phi_t, coef_t
    return st.t()

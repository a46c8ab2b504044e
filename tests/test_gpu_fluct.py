"""GPU parity of rpod_fluctuations (Eqs. (time_av), (fluct_q)) and
rpod_energy_rank (Eq. (energy)) against the FP64 oracle, through the C ABI.

Tolerances follow the arithmetic: the kernel sums each row with Neumaier
compensation in FP64 (FP64 S) or FP32 (other S), so a mean is within a few
units of rounding u of max|S| over its sample's row (plus the oracle's own
uncompensated FP64 sum, within 2 nt 2^-53 max|S|), and a fluctuation adds
one rounding of the difference (u = 2^-53 or 2^-24) and, for a 16-bit
output, one rounding to that format (relative 2^-9 for BF16, 2^-12 for
FP16, doubled for the two roundings).  The energy rank is an integer decided
in FP64 by the same sequential sums on both sides: bit-exact."""
import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from oracle.rpod import energy_rank, fluctuations, rpod
from tests.rpod_checks import sigma_close

pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24
REL16 = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def make_S(n, m, nt, seed, dtype=torch.float64):
    """Random snapshots with a per-sample mean field well away from zero."""
    rng = np.random.default_rng(seed)
    M = m // nt
    mean = rng.standard_normal((n, M)) * 4.0 + 2.0
    S = np.repeat(mean, nt, axis=1) + rng.standard_normal((n, m))
    t = torch.from_numpy(S).to(dtype)
    return t, t.double().numpy()


def colmajor(A_np_or_t, dtype, device="cuda", ld=None, offset=0):
    """Column-major device copy with leading dimension ld (>= rows) starting
    `offset` elements into its storage."""
    A = torch.as_tensor(A_np_or_t)
    n, m = A.shape
    ld = ld or n
    buf = torch.zeros(offset + ld * m, dtype=dtype, device=device)
    view = buf[offset:].view(m, ld).t()[:n]
    view.copy_(A.to(dtype))
    return view


def absmax_per_sample(S64, nt):
    n, m = S64.shape
    return np.abs(S64).reshape(n, m // nt, nt).max(axis=2)


def check(S64, nt, F, Sbar, u, rel_out=0.0):
    Fo, Sbo = fluctuations(S64, nt)
    amax = absmax_per_sample(S64, nt)
    # the oracle's own FP64 sum (numpy, pairwise) is off by up to about
    # log2(nt) U64 max|S|: bounded here by 2 nt U64 max|S|
    orc = 2 * nt * U64 * amax
    got = Sbar.double().cpu().numpy()
    assert np.all(np.abs(got - Sbo) <= 4 * u * amax + orc), np.abs(got - Sbo).max()
    if F is not None:
        gf = F.double().cpu().numpy()
        tol = np.repeat(8 * u * amax + orc, nt, axis=1) + rel_out * np.abs(Fo)
        assert np.all(np.abs(gf - Fo) <= tol), np.abs(gf - Fo).max()


@pytest.mark.parametrize("n,nt,M", [(1000, 7, 5), (4099, 40, 3), (777, 400, 2), (33, 1, 9),
                                    (2500, 96, 1), (1, 5, 3)])
def test_f64_and_f32(n, nt, M):
    m = nt * M
    S, S64 = make_S(n, m, nt, seed=n + nt)
    for dtype, u in ((torch.float64, U64), (torch.float32, U32)):
        Sd = colmajor(S, dtype)
        S_in = Sd.double().cpu().numpy()       # the values the kernel sees
        F, _, Sbar = R.fluctuations(Sd, nt)
        check(S_in, nt, F, Sbar, u)


@pytest.mark.parametrize("hd", [torch.bfloat16, torch.float16])
def test_f32_with_16bit_outputs(hd):
    n, nt, M = 3000, 50, 4
    S, _ = make_S(n, nt * M, nt, seed=3)
    Sd = colmajor(S, torch.float32)
    S_in = Sd.double().cpu().numpy()
    # FP32 F plus a 16-bit copy H, then a 16-bit F alone
    F, H, Sbar = R.fluctuations(Sd, nt, h_dtype=hd)
    check(S_in, nt, F, Sbar, U32)
    check(S_in, nt, H, Sbar, U32, REL16[hd])
    F2, _, Sbar2 = R.fluctuations(Sd, nt, f_dtype=hd)
    check(S_in, nt, F2, Sbar2, U32, REL16[hd])


@pytest.mark.parametrize("sd", [torch.bfloat16, torch.float16])
def test_16bit_input(sd):
    n, nt, M = 2049, 24, 3
    S, _ = make_S(n, nt * M, nt, seed=4)
    Sd = colmajor(S, sd)
    S_in = Sd.double().cpu().numpy()
    F, _, Sbar = R.fluctuations(Sd, nt)
    assert F.dtype == sd and Sbar.dtype == torch.float32
    check(S_in, nt, F, Sbar, U32, REL16[sd])


def test_in_place_means_only_and_unaligned():
    n, nt, M = 1531, 30, 3
    S, _ = make_S(n, nt * M, nt, seed=5)
    # in place
    Sd = colmajor(S, torch.float32)
    S_in = Sd.double().cpu().numpy()
    F, _, Sbar = R.fluctuations(Sd, nt, in_place=True)
    assert F.data_ptr() == Sd.data_ptr()
    check(S_in, nt, F, Sbar, U32)
    # means only
    Sd = colmajor(S, torch.float32)
    _, _, Sbar = R.fluctuations(Sd, nt, f_dtype=None)
    check(S_in, nt, None, Sbar, U32)
    # odd leading dimension and a storage offset: no 16-byte copies or stores
    for ld, off in ((n + 1, 0), (n + 3, 1)):
        Sd = colmajor(S, torch.float32, ld=ld, offset=off)
        F = colmajor(np.zeros(S.shape), torch.float32, ld=ld + 2, offset=3)
        H = colmajor(np.zeros(S.shape), torch.bfloat16, ld=ld, offset=1)
        Sbar = colmajor(np.zeros((n, M)), torch.float32, ld=n + 5, offset=1)
        R.fluctuations(Sd, nt, out=(F, H, Sbar))
        check(S_in, nt, F, Sbar, U32)
        check(S_in, nt, H, Sbar, U32, REL16[torch.bfloat16])


@pytest.mark.parametrize("dtype,u", [(torch.float32, U32), (torch.float64, U64),
                                     (torch.bfloat16, U32)])
def test_streaming_variant_long_samples(dtype, u):
    # a 128-byte-high tile of 2048 snapshots exceeds shared memory: the
    # kernel sums from global memory and reads S again for the write
    n, nt, M = 300, 2048, 2
    S, _ = make_S(n, nt * M, nt, seed=6)
    Sd = colmajor(S, dtype)
    S_in = Sd.double().cpu().numpy()
    F, _, Sbar = R.fluctuations(Sd, nt)
    check(S_in, nt, F, Sbar, u, REL16.get(dtype, 0.0))


def test_argument_errors_on_device_tensors():
    S = torch.zeros(10, 12, device="cuda").t().contiguous().t()
    with pytest.raises(ValueError):
        R.fluctuations(S, 5)
    Sb = S.to(torch.bfloat16)
    with pytest.raises(R.RpodError) as e:
        R.fluctuations(Sb, 4, h_dtype=torch.float16)
    assert e.value.code == R.RPOD_ERR_UNSUPPORTED
    S64 = S.double()
    with pytest.raises(R.RpodError) as e:
        R.fluctuations(S64, 4, f_dtype=torch.float32)
    assert e.value.code == R.RPOD_ERR_UNSUPPORTED


def test_full_size_sampled_rows():
    """The bench's snapshot shape (262144 x 10000 FP32, 25 samples of 400
    snapshots) with the FP32 fluctuations and their BF16 copy: sampled rows
    against the oracle, and every sample's fluctuations summing to ~0."""
    n, m, nt = 262144, 10000, 400
    M = m // nt
    g = torch.Generator(device="cuda").manual_seed(11)
    S = torch.randn((m, n), device="cuda", generator=g).t()
    mean = torch.randn((n, M), device="cuda", generator=g) * 4 + 2
    S += mean.repeat_interleave(nt, dim=1)
    rows = torch.from_numpy(np.random.default_rng(0).choice(n, 48, replace=False)).cuda()
    S_rows = S[rows].double().cpu().numpy()
    F, H, Sbar = R.fluctuations(S, nt, h_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    check(S_rows, nt, F[rows], Sbar[rows], U32)
    check(S_rows, nt, H[rows], Sbar[rows], U32, REL16[torch.bfloat16])
    amax = S.abs().view(n, M, nt).amax(2)
    gs = F.view(n, M, nt).double().sum(2).abs()
    assert bool((gs <= nt * 8 * U32 * amax.double()).all())
    del S, F, H


def test_energy_rank_bit_exact():
    rng = np.random.default_rng(7)
    cases = []
    for l in (1, 2, 5, 30, 120, 128):
        for _ in range(20):
            s = np.sort(np.abs(rng.standard_normal(l)) * 10.0 ** rng.uniform(-3, 3, l))[::-1].copy()
            cases.append((s, float(rng.uniform(0.01, 1.0))))
    # ties at the threshold: the decision must match the oracle's rounding
    s = 0.5 ** np.arange(8)
    total = np.cumsum(s)[-1]
    for N in range(1, 9):
        cases.append((s, float(np.cumsum(s)[N - 1] / total)))
    cases += [(np.ones(10), 0.5), (np.ones(10), 1.0), (np.zeros(6), 0.9),
              (np.array([3.0, 1.0, 0.0, 0.0]), 1.0), (np.array([1e-300, 1e-310]), 0.99)]
    for s, delta in cases:
        sig = torch.from_numpy(s).cuda()
        got = int(R.energy_rank(sig, delta).item())
        assert got == energy_rank(s, delta), (s, delta)


def test_centered_rpod_matches_oracle():
    """Centering then Alg. 1 (BF16 passes, FP32 refinement) against the
    oracle's rPOD of its own fluctuations, on a config-1-sized input."""
    n, nt, M = 4096, 50, 10
    m = nt * M
    rng = np.random.default_rng(8)
    Ut, _ = np.linalg.qr(rng.standard_normal((n, 40)))
    Vt, _ = np.linalg.qr(rng.standard_normal((m, 40)))
    S64 = (Ut * 0.8 ** np.arange(40)) @ Vt.T * 50 + np.repeat(rng.standard_normal((n, M)), nt, 1)
    Sd = colmajor(S64, torch.float32)
    S_in = Sd.double().cpu().numpy()
    F, H, Sbar = R.fluctuations(Sd, nt, in_place=True, h_dtype=torch.bfloat16)
    plan = R.Plan(n, m, 20, 10, 1, seed=2, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U, sig, C = plan.basis(H, S_refine=F)
    rc, _ = plan.status()
    assert rc == R.RPOD_OK
    Fo, _ = fluctuations(S_in, nt)
    ref = rpod(Fo, 20, 10, 1, seed=2)
    ok, er, ea = sigma_close(sig.cpu().numpy()[:20], ref.sigma[:20], 1e-4, 1e-5)
    assert ok, (er, ea)
    N = int(R.energy_rank(torch.from_numpy(ref.sigma).cuda(), 0.9).item())
    assert N == energy_rank(ref.sigma, 0.9)

"""GPU tests of the tensor-core (tcgen05 + TMA) forms through the C ABI.

Pass kernels are checked against FP64 products of the same 16-bit operands
(exact inputs, so only FP32 accumulation separates them); the full 16-bit
rPOD with FP32 refinement is checked against the FP64 oracle run on the
16-bit-rounded snapshots and sketch (the storage error floor) and on the
original FP32 snapshots."""
import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from oracle.rpod import rpod as oracle_rpod
from oracle.rpod import round_to
from synth import make_recipe, snapshot_matrix
from tests.rpod_checks import max_angle, orth_err, sigma_close

pytestmark = pytest.mark.gpu

TDT = {"bf16": torch.bfloat16, "f16": torch.float16}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def colmajor(rows, cols, dtype, gen, device="cuda"):
    return torch.randn((cols, rows), generator=gen, dtype=torch.float32).to(dtype).to(device).t()


def rel_err(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("form", ["bf16", "f16"])
@pytest.mark.parametrize("n,m,kc", [(4096, 512, 32), (1000, 333, 17), (70000, 700, 120), (256, 64, 1)])
def test_wpass_project_matches_fp64(form, n, m, kc):
    g = torch.Generator().manual_seed(n + m + kc)
    l = min(128, max(kc, 2))
    plan = R.Plan(n, m if m >= l else l, kc, l - kc, 1, compute=form)
    U = colmajor(n, kc, torch.float32, g)
    S = colmajor(n, m, TDT[form], g)
    C = plan.project(U, S)
    torch.cuda.synchronize()
    ref = (U.to(TDT[form]).double().t() @ S.double())
    err = rel_err(C.double(), ref)
    assert err < 2e-5, err


@pytest.mark.parametrize("form", ["bf16", "f16"])
@pytest.mark.parametrize("n,m,l", [(4096, 512, 30), (1000, 333, 12), (70000, 1000, 128), (304, 64, 5)])
def test_ypass_sample_matches_fp64(form, n, m, l):
    g = torch.Generator().manual_seed(7 * n + m + l)
    plan = R.Plan(n, m, l, 0, 1, compute=form)
    A = colmajor(m, l, TDT[form], g)
    S = colmajor(n, m, TDT[form], g)
    Y = R.empty_colmajor(n, l, torch.float32, "cuda")
    rc = R.rpod_sample(plan.handle, A.data_ptr(), R.colmajor_ld(A), S.data_ptr(), R.colmajor_ld(S),
                       R.dtype_code(TDT[form]), Y.data_ptr(), n, plan.ws_ptr, plan.ws_bytes,
                       torch.cuda.current_stream().cuda_stream)
    assert rc == R.RPOD_OK
    torch.cuda.synchronize()
    ref = S.double() @ A.double()
    err = rel_err(Y.double(), ref)
    assert err < 2e-5, err
    assert plan.status()[0] == R.RPOD_OK


def _oracles(S64, k, p, q, form):
    Sr = round_to(S64, form)
    lowp = oracle_rpod(S64, k, p, q, seed=0, sketch_dtype=form, S_passes=Sr)
    orig = oracle_rpod(S64, k, p, q, seed=0)
    return lowp, orig


# sigma (i <= k) and largest principal angle of span(U_k) for the 16-bit
# forms with the refinement pass: BF16 (TF32 refinement) 1e-4 and 1e-2; FP16
# (exact FP32 refinement) 1e-5 and 2e-3.
BOUNDS_16 = {"bf16": (1e-4, 1e-2), "f16": (1e-5, 2e-3)}


@pytest.mark.parametrize("form", ["bf16", "f16"])
def test_basis_16bit_refine_config1(form):
    """Config 1 shape (n = 4096, m = 500, k = 20, p = 10, q = 1), 16-bit
    passes with the FP32 refinement pass; S handed over in FP32 and
    converted on the device.  Against the oracle on the 16-bit-rounded
    passes (the storage floor) and on the FP32 snapshots, with each form's
    own bounds."""
    rec = make_recipe(64, 64, 500, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec, dtype=torch.float32)
    S64 = S.double().numpy()
    k, p, q = 20, 10, 1
    lowp, orig = _oracles(S64, k, p, q, form)
    plan = R.Plan(rec.n, rec.m, k, p, q, seed=0, compute=form, flags=R.RPOD_FLAG_REFINE_FP32)
    U, sig, C = plan.basis(S.t().contiguous().cuda().t())
    rc, _ = plan.status()
    assert rc == R.RPOD_OK
    sig = sig.cpu().numpy()
    U = U.double().cpu().numpy()
    srel, ang = BOUNDS_16[form]
    for name, o in (("rounded-input", lowp), ("FP32-input", orig)):
        err = np.abs(sig[:k] - o.sigma[:k]) / o.sigma[:k]
        assert err.max() <= srel, (name, err.max())
        assert max_angle(o.U[:, :k], U) <= ang, (name, max_angle(o.U[:, :k], U))
    assert orth_err(U) <= 1e-5


@pytest.mark.parametrize("n,m", [(1000, 333), (2048, 700)])
def test_basis_bf16_ragged_and_16bit_input(n, m):
    rng = np.random.default_rng(n)
    S64 = (rng.standard_normal((n, m)) * np.logspace(0, -3, m)[None, :])
    S32 = torch.from_numpy(S64).float()
    k, p, q = 8, 6, 2
    lowp, orig = _oracles(S32.double().numpy(), k, p, q, "bf16")
    # 16-bit S plus an FP32 refinement copy
    Sd = S32.t().contiguous().cuda().t()
    Sb = Sd.t().contiguous().to(torch.bfloat16).t()
    plan = R.Plan(n, m, k, p, q, seed=0, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U, sig, C = plan.basis(Sb, S_refine=Sd)
    assert plan.status()[0] == R.RPOD_OK
    sig = sig.cpu().numpy()
    ok, er, ea = sigma_close(sig[:k], orig.sigma[:k], 1e-3, 1e-4)
    assert ok, (er, ea)
    assert orth_err(U.double().cpu().numpy()) <= 1e-5
    # without refinement: reported, loose bound
    plan2 = R.Plan(n, m, k, p, q, seed=0, compute="bf16")
    U2, sig2, _ = plan2.basis(Sb)
    assert plan2.status()[0] == R.RPOD_OK
    ok, er, ea = sigma_close(sig2.cpu().numpy()[:k], lowp.sigma[:k], 2e-2, 2e-3)
    assert ok, (er, ea)


def _padded(S64, ld, dtype):
    """Column-major n x m view with leading dimension ld (rows n..ld-1 zero)."""
    n, m = S64.shape
    buf = torch.zeros((m, ld), dtype=torch.float32)
    buf[:, :n] = torch.from_numpy(S64.T).float()
    return buf.to(dtype).cuda().t()[:n]


@pytest.mark.parametrize("n,m,ld", [(1001, 333, 1004), (4100, 700, 4100), (262, 64, 264)])
def test_fp32_input_first_pass_conversion_matches_16bit_input(n, m, ld):
    """An FP32 S is rounded to BF16 inside the first Y-pass, which also writes
    the BF16 copy the later passes read; the result must equal the pipeline
    fed with the same BF16 values converted on the host (ragged row counts,
    padded leading dimensions, a partial last row group)."""
    rng = np.random.default_rng(n + m)
    S64 = rng.standard_normal((n, m)) * np.logspace(0, -3, m)[None, :]
    Sd = _padded(S64, ld, torch.float32)
    Sb = _padded(S64, (n + 7) // 8 * 8, torch.bfloat16)
    k, p, q = 8, 6, 2
    fused = R.Plan(n, m, k, p, q, seed=0, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U1, s1, C1 = fused.basis(Sd)
    assert fused.status()[0] == R.RPOD_OK
    host = R.Plan(n, m, k, p, q, seed=0, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U2, s2, C2 = host.basis(Sb, S_refine=Sd)
    assert host.status()[0] == R.RPOD_OK
    s1, s2 = s1.cpu().numpy(), s2.cpu().numpy()
    assert np.abs(s1[:k] - s2[:k]).max() <= 1e-6 * s2[0]
    assert max_angle(U2.double().cpu().numpy(), U1.double().cpu().numpy()) <= 1e-4
    # a non-finite snapshot entry is reported by the fused pass
    Sd[n - 1, m - 1] = float("nan")
    fused.basis(Sd)
    assert fused.status()[0] == R.RPOD_ERR_NONFINITE


def test_basis_bf16_refine_65536_rows_matches_oracle():
    """The full-size code paths at a size the oracle finishes in seconds:
    n = 65536 (256 x 256 grid), m = 4000, k = 100, p = 20 (l = 120), q = 2,
    400 modes with exp(-j/40) amplitudes, FP32 S converted in the first pass.
    The Y-passes need two waves of CTAs and the W-passes split n into 48
    chunks (16 snapshot tiles of 256, about five waves of 152 SMs).  BF16 bounds against both oracles, sigma_i for every i <= k."""
    rec = make_recipe(256, 256, 4000, 400, ("exp", 40.0), seed=0, noise=1e-6)
    S = snapshot_matrix(rec, device="cuda", dtype=torch.float32)
    k, p, q = 100, 20, 2
    assert rec.n // 256 > 152          # Y-pass: 256 CTAs of 256 rows (512 of 128 in the first)
    plan = R.Plan(rec.n, rec.m, k, p, q, seed=0, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U, sig, C = plan.basis(S)
    assert plan.status()[0] == R.RPOD_OK
    sig = sig.cpu().numpy()
    U = U.double().cpu().numpy()
    S64 = S.cpu().double().numpy()
    lowp, orig = _oracles(S64, k, p, q, "bf16")
    for name, o in (("rounded-input", lowp), ("FP32-input", orig)):
        err = np.abs(sig[:k] - o.sigma[:k]) / o.sigma[:k]
        assert err.max() <= 1e-4, (name, err.max())
        assert max_angle(o.U[:, :k], U) <= 1e-2, name
    assert orth_err(U) <= 1e-5


def test_basis_bf16_refine_tail_tiles_split_over_snapshots():
    """Y-passes whose last wave of row tiles would fill at most 60 % of the
    GPU run their whole waves in one launch and the last tiles, split over
    the snapshots, in a second (partials summed into Y): n = 100352 rows
    (392 tiles of 256 in the S Z passes, two CTAs per SM, 88 in the tail;
    784 tiles of 128 in the first pass, 24 in the tail), m = 2000, k = 20,
    p = 10, q = 2.  BF16 bounds against both oracles."""
    # amplitudes j^-1.5 (the config-1 spectrum): sigma_20 / sigma_21 = 1.08,
    # so span(U_k) is well separated at the BF16 error level
    rec = make_recipe(256, 392, 2000, 400, ("power", 1.5), seed=3, noise=1e-6)
    S = snapshot_matrix(rec, device="cuda", dtype=torch.float32)
    k, p, q = 20, 10, 2
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < (rec.n // 256) % (2 * sms) <= 0.6 * 2 * sms
    assert 0 < (rec.n // 128) % sms <= 0.6 * sms
    plan = R.Plan(rec.n, rec.m, k, p, q, seed=0, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U, sig, C = plan.basis(S)
    assert plan.status()[0] == R.RPOD_OK
    sig = sig.cpu().numpy()
    U = U.double().cpu().numpy()
    assert orth_err(U) <= 1e-5
    S64 = S.cpu().double().numpy()
    lowp, orig = _oracles(S64, k, p, q, "bf16")
    for name, o in (("rounded-input", lowp), ("FP32-input", orig)):
        err = np.abs(sig[:k] - o.sigma[:k]) / o.sigma[:k]
        assert err.max() <= 1e-4, (name, err.max())
        assert max_angle(o.U[:, :k], U) <= 1e-2, name


def test_basis_bf16_refine_paper_shape_split_ypass():
    """The paper's own snapshot-matrix shape (Sec. 4.2, Table tab:cpu_time):
    n = 8192 grid cells (64 x 128), m = 90225 snapshots, k = 10, p = 75,
    q = 1.  With 32 row tiles of 256 (64 of 128 in the first pass) the
    Y-passes split the snapshots into chunks summed in the W-pass partial
    buffer; BF16 bounds against both oracles."""
    rec = make_recipe(64, 128, 90225, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec, device="cuda", dtype=torch.float32)
    k, p, q = 10, 75, 1
    plan = R.Plan(rec.n, rec.m, k, p, q, seed=0, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    U, sig, C = plan.basis(S)
    assert plan.status()[0] == R.RPOD_OK
    sig = sig.cpu().numpy()
    U = U.double().cpu().numpy()
    S64 = S.cpu().double().numpy()
    lowp, orig = _oracles(S64, k, p, q, "bf16")
    for name, o in (("rounded-input", lowp), ("FP32-input", orig)):
        err = np.abs(sig[:k] - o.sigma[:k]) / o.sigma[:k]
        assert err.max() <= 1e-4, (name, err.max())
        assert max_angle(o.U[:, :k], U) <= 1e-2, name
    assert orth_err(U) <= 1e-5

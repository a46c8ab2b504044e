"""GPU parity tests: librpod (through its C ABI) against the FP64 oracle on
the same seeded inputs and the same Philox sketch.  Tolerances follow the
rounding of each form: FP64 sigma within 1e-10 relative and the largest
principal angle of span(U_k) within 1e-8; FP32 within 1e-5 and 1e-4."""
import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from oracle.philox import gaussian_sketch
from oracle.rpod import project as oracle_project
from oracle.rpod import rpod as oracle_rpod
from synth import make_recipe, snapshot_matrix, time_matrix
from tests.rpod_checks import F64_FLOOR, max_angle, orth_err, sigma_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def dev(S_cpu, dtype):
    """Column-major device copy of a column-major host matrix."""
    return S_cpu.t().contiguous().to(dtype).cuda().t()


def lowrank(n, m, J, seed, decay=0.6, scale=10.0):
    rng = np.random.default_rng(seed)
    Uq, _ = np.linalg.qr(rng.standard_normal((n, J)))
    Vq, _ = np.linalg.qr(rng.standard_normal((m, J)))
    s = scale * decay ** np.arange(J)
    return torch.from_numpy((Uq * s) @ Vq.T).t().contiguous().t(), Uq, s


def run_gpu(S, k, p, q, seed, compute, flags=0):
    n, m = S.shape
    plan = R.Plan(n, m, k, p, q, seed=seed, compute=compute, flags=flags)
    U, sig, C = plan.basis(S)
    rc, warn = plan.status()
    torch.cuda.synchronize()
    return plan, U.double().cpu().numpy(), sig.cpu().numpy(), C.double().cpu().numpy(), rc, warn


def check_signs(U):
    idx = np.argmax(np.abs(U), axis=0)
    return np.all(U[idx, np.arange(U.shape[1])] >= 0)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m,l,seed", [(501, 12, 3), (500, 30, 0), (7, 1, 9)])
def test_sketch_matches_oracle(m, l, seed):
    plan = R.Plan(max(m, 64), m, l, 0, 1, seed=seed, compute="f64")
    lam = plan.sketch(torch.float64).cpu().numpy()
    ref = gaussian_sketch(seed, m, l, 0)
    assert np.abs(lam - ref).max() <= 1e-14
    lam32 = plan.sketch(torch.float32).cpu().numpy()
    assert np.abs(lam32 - ref).max() <= 4e-7


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_16bit_sketch_is_the_rounded_oracle_sketch(dtype):
    """16-bit sketches are evaluated in FP32: every entry is the oracle's FP64
    value rounded to the 16-bit type, except entries within a few FP32 ulps of
    a rounding boundary, which may land on the neighbouring 16-bit value."""
    m, l, seed = 3001, 120, 11
    plan = R.Plan(4096, m, l, 0, 1, seed=seed, compute="bf16")
    got = plan.sketch(dtype).float().cpu().numpy().astype(np.float64)
    ref64 = gaussian_sketch(seed, m, l, 0)
    ref = torch.from_numpy(ref64).to(dtype).double().numpy()
    diff = got != ref
    assert diff.mean() <= 2e-3, diff.mean()
    ulp = np.abs(ref) * (2.0 ** -7 if dtype == torch.bfloat16 else 2.0 ** -10)
    assert np.all(np.abs(got - ref)[diff] <= 1.01 * ulp[diff] + 2.0 ** -24)
    # and the shared mantissa bits agree with the FP64 value to FP32 accuracy
    assert np.abs(got - ref64).max() <= 2.0 ** -7 * np.abs(ref64).max()


def test_f64_config1_matches_oracle():
    rec = make_recipe(64, 64, 500, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec)
    k, p, q = 20, 10, 1
    o = oracle_rpod(S.numpy(), k, p, q, seed=0)
    plan, U, sig, C, rc, warn = run_gpu(dev(S, torch.float64), k, p, q, 0, "f64")
    assert rc == R.RPOD_OK and warn == 0
    ok, er, ea = sigma_close(sig, o.sigma, 1e-10, 1e-12, floor=F64_FLOOR)
    assert ok, (er, ea)
    assert max_angle(o.U[:, :k], U) <= 1e-8
    assert orth_err(U) <= 1e-12
    assert check_signs(U)
    # rows of C agree with the oracle's literal U_k^T S up to the row sign
    for i in range(k):
        d = min(np.abs(C[i] - o.C[i]).max(), np.abs(C[i] + o.C[i]).max())
        assert d <= 1e-9 * o.sigma[0]
    assert plan.launches() > 10


@pytest.mark.parametrize("n,m,k,p,q", [
    (1000, 333, 7, 5, 2),     # ragged tiles in every dimension
    (50, 300, 10, 5, 1),      # wide matrix
    (40, 24, 20, 4, 1),       # l = min(n, m): brute-force equality with the full SVD
    (300, 200, 1, 0, 0),      # l = 1, q = 0
    (257, 129, 60, 68, 3),    # l = 128, the one-block limit
])
def test_f64_shapes_match_oracle(n, m, k, p, q):
    rng = np.random.default_rng(n + m)
    S = torch.from_numpy(rng.standard_normal((n, m)) * np.logspace(0, -2, m)[None, :]).t().contiguous().t()
    o = oracle_rpod(S.numpy(), k, p, q, seed=5)
    _, U, sig, C, rc, _ = run_gpu(dev(S, torch.float64), k, p, q, 5, "f64")
    assert rc == R.RPOD_OK
    ok, er, ea = sigma_close(sig, o.sigma, 1e-10, 1e-12, floor=F64_FLOOR)
    assert ok, (er, ea)
    # compare subspaces only where the spectrum has a gap at k
    if k < len(o.sigma) and o.sigma[k - 1] > o.sigma[k] * (1 + 1e-6):
        gap = (o.sigma[k - 1] - o.sigma[k]) / o.sigma[0]
        assert max_angle(o.U[:, :k], U) <= max(1e-8, 1e-13 / gap)
    assert orth_err(U) <= 1e-12


def test_f64_exact_rank_flags_and_recovers():
    S, Uq, s = lowrank(600, 250, 5, seed=1)
    _, U, sig, C, rc, warn = run_gpu(dev(S, torch.float64), 8, 4, 1, 2, "f64")
    assert rc == R.RPOD_OK
    assert warn & R.RPOD_WARN_RANK_DEFICIENT
    assert np.allclose(sig[:5], s, rtol=1e-10)
    assert np.all(sig[5:] <= 1e-7 * s[0])
    assert max_angle(Uq, U[:, :5]) <= 1e-8


def graded(n, m, l, seed, lo=-8.0):
    """S = U0 diag(sigma) V0^T, sigma = logspace(0, lo, l), random orthonormal
    U0 (n x l) and V0 (m x l): a spectrum graded over 10^-lo within the top l."""
    rng = np.random.default_rng(seed)
    U0, _ = np.linalg.qr(rng.standard_normal((n, l)))
    V0, _ = np.linalg.qr(rng.standard_normal((m, l)))
    s = np.logspace(0.0, lo, l)
    return torch.from_numpy((U0 * s) @ V0.T).t().contiguous().t(), U0, s


@pytest.mark.parametrize("n,m,l,k", [(2048, 400, 40, 30), (4096, 500, 30, 20), (8192, 1000, 120, 100)])
def test_f64_graded_spectrum_every_sigma_relative(n, m, l, k):
    """sigma_i over eight decades (1 .. 1e-8): the sampled matrix has a
    condition number near 1e9 (shifted CholeskyQR3) and the small SVD must
    keep the relative accuracy of the smallest values (one-sided Jacobi on
    the transposed Cholesky factor of T T^T).  The exact spectrum is known,
    so GPU and oracle are both measured against it: 1e-10 relative wherever
    sigma_i >= 1e-7 sigma_1.  In the last decade the FP64 rounding of
    T = Q^T S itself (about c u sigma_1 / sigma_i with c ~ 1e-2, the same in
    every implementation) reaches 1e-10: the oracle is off the exact values
    by up to about 1.3e-10 there, and the GPU is held to 1e-9 of both."""
    S, U0, s = graded(n, m, l, seed=n + l)
    o = oracle_rpod(S.numpy(), k, l - k, 1, seed=0)
    top = s >= 1e-7 * s[0]
    e_oracle = np.abs(o.sigma - s) / s
    assert e_oracle[top].max() <= 1e-10 and e_oracle.max() <= 1e-9   # the oracle's own pin
    plan, U, sig, C, rc, warn = run_gpu(dev(S, torch.float64), k, l - k, 1, 0, "f64")
    assert rc == R.RPOD_OK and warn == 0
    e_gpu = np.abs(sig - s) / s
    e_rel = np.abs(sig - o.sigma) / o.sigma
    assert e_gpu[top].max() <= 1e-10, (e_gpu[top].max(), int(e_gpu[top].argmax()))
    assert e_rel[top].max() <= 1e-10, (e_rel[top].max(), int(e_rel[top].argmax()))
    assert e_gpu.max() <= 1e-9 and e_rel.max() <= 1e-9, (e_gpu.max(), e_rel.max())
    assert max_angle(o.U[:, :k], U) <= 1e-8
    assert orth_err(U) <= 1e-12
    assert check_signs(U)
    assert 1 <= plan.svd_sweeps() <= 12


def test_f64_jacobi_sweep_cap_reports_no_convergence():
    """A host-set cap of one Jacobi sweep on a graded spectrum: the sweep
    still rotates, so the device reports RPOD_ERR_NO_CONVERGENCE (outputs are
    written, the context stays usable); without the cap the same plan
    converges."""
    S, _, s = graded(2048, 400, 40, seed=3)
    Sd = dev(S, torch.float64)
    plan = R.Plan(2048, 400, 30, 10, 1, seed=0, compute="f64")
    plan.set_svd_sweeps(1)
    U, sig, C = plan.basis(Sd)
    rc, _ = plan.status()
    assert rc == R.RPOD_ERR_NO_CONVERGENCE
    assert plan.svd_sweeps() == 1
    assert np.all(np.isfinite(sig.cpu().numpy()))
    plan.set_svd_sweeps(30)
    plan.basis(Sd)
    assert plan.status()[0] == R.RPOD_OK
    # the cap applies to the FP64 form only
    with pytest.raises(R.RpodError) as e:
        R.Plan(2048, 400, 30, 10, 1, compute="f32").set_svd_sweeps(1)
    assert e.value.code == R.RPOD_ERR_UNSUPPORTED


@pytest.mark.parametrize("compute,dtype", [("f64", torch.float64), ("f32", torch.float32),
                                           ("bf16", torch.float32)])
def test_zero_snapshots_report_breakdown(compute, dtype):
    """An all-zero S: every column of the first Gram vanishes, the device
    reports RPOD_ERR_BREAKDOWN and the singular values are zero (finite)."""
    flags = R.RPOD_FLAG_REFINE_FP32 if compute == "bf16" else 0
    plan = R.Plan(1024, 300, 10, 6, 1, seed=0, compute=compute, flags=flags)
    S = torch.zeros((300, 1024), dtype=dtype, device="cuda").t()
    U, sig, C = plan.basis(S)
    rc, warn = plan.status()
    assert rc == R.RPOD_ERR_BREAKDOWN, R.rpod_strerror(rc)
    assert warn & R.RPOD_WARN_RANK_DEFICIENT
    sg = sig.cpu().numpy()
    assert np.all(np.isfinite(sg)) and np.all(sg == 0.0)
    # the plan recovers on the next call
    rng = np.random.default_rng(0)
    plan.basis(torch.from_numpy(rng.standard_normal((1024, 300))).to(dtype).t().contiguous().cuda().t())
    assert plan.status()[0] == R.RPOD_OK


def test_f32_config1_matches_oracle():
    rec = make_recipe(64, 64, 500, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec)
    k, p, q = 20, 10, 1
    o = oracle_rpod(S.float().double().numpy(), k, p, q, seed=0)
    _, U, sig, C, rc, warn = run_gpu(dev(S, torch.float32), k, p, q, 0, "f32")
    assert rc == R.RPOD_OK
    ok, er, ea = sigma_close(sig[:k], o.sigma[:k], 1e-5, 1e-6)
    assert ok, (er, ea)
    assert max_angle(o.U[:, :k], U) <= 1e-4
    assert orth_err(U) <= 1e-5
    for i in range(k):
        d = min(np.abs(C[i] - o.C[i]).max(), np.abs(C[i] + o.C[i]).max())
        assert d <= 1e-5 * o.sigma[0]


def test_f32_wide_basis_matches_oracle():
    """FP32 form with l = 80 > 64, where the products over S take the
    128 x 128 FP32 pass kernel: n = 4160 and m = 1001 leave ragged row,
    snapshot and column tiles, and the S^T Q passes split over rows.
    Against the oracle on the same FP32 snapshots: sigma_i within 1e-5
    relative (1e-6 sigma_1 below 1e-3 sigma_1); span(U_k) within the
    Davis-Kahan scale 10 u_32 sigma_1 / (sigma_k - sigma_{k+1}) of FP32
    rounding (this spectrum's gap at k = 70 is 5e-5 sigma_1, and a pair
    inside U_k lies 8e-6 sigma_1 apart, so single vectors are not compared);
    U orthonormal to 1e-5; C and the projection of new snapshots equal
    U^T S with the returned U to 1e-5 sigma_1."""
    rec = make_recipe(64, 65, 1001, 400, ("power", 1.2), seed=6, noise=1e-6)
    S = snapshot_matrix(rec)
    k, p, q = 70, 10, 1
    S64 = S.float().double().numpy()
    o = oracle_rpod(S64, k, p, q, seed=5)
    plan, U, sig, C, rc, warn = run_gpu(dev(S, torch.float32), k, p, q, 5, "f32")
    assert rc == R.RPOD_OK
    ok, er, ea = sigma_close(sig[:k], o.sigma[:k], 1e-5, 1e-6)
    assert ok, (er, ea)
    gap = o.sigma[k - 1] - o.sigma[k]
    assert max_angle(o.U[:, :k], U) <= 10 * 2.0**-24 * o.sigma[0] / gap
    assert orth_err(U) <= 1e-5
    assert np.abs(C - U.T @ S64).max() <= 1e-5 * o.sigma[0]
    Snew = S[:, 500:777].float()
    Cn = plan.project(dev(torch.from_numpy(U), torch.float32), dev(Snew, torch.float32))
    ref = oracle_project(U, Snew.double().numpy())
    assert np.abs(Cn.double().cpu().numpy() - ref).max() <= 1e-5 * o.sigma[0]


def test_f32_steep_spectrum_through_fp64_factorization():
    """Amplitudes exp(-j/5), k = 50, p = 10, q = 1 (l = 60): the Grams of the
    sampled and power-iterated matrices span condition numbers near 1e10,
    beyond the FP32 Cholesky's pivot test, so the first CholeskyQR round of
    every orthonormalization refactors the exact-product Gram in FP64 (the
    gated path).  FP32 form against the oracle on the same FP32 snapshots:
    sigma_i within 2e-5 where sigma_i >= 1e-2 sigma_1 and within 1e-6
    sigma_1 below, the top-10 span within 1e-4, U orthonormal to 1e-5 and
    no direction dropped."""
    rec = make_recipe(64, 64, 1500, 200, ("exp", 5.0), seed=4, noise=1e-6)
    S = snapshot_matrix(rec)
    k, p, q = 50, 10, 1
    o = oracle_rpod(S.float().double().numpy(), k, p, q, seed=3)
    _, U, sig, C, rc, warn = run_gpu(dev(S, torch.float32), k, p, q, 3, "f32")
    assert rc == R.RPOD_OK and warn == 0
    ok, er, ea = sigma_close(sig[:k], o.sigma[:k], 2e-5, 1e-6, floor=1e-2)
    assert ok, (er, ea)
    assert max_angle(o.U[:, :10], U[:, :10]) <= 1e-4
    assert orth_err(U) <= 1e-5


def test_project_matches_oracle():
    rec = make_recipe(32, 64, 300, 100, ("power", 1.5), seed=3)
    S = snapshot_matrix(rec)
    plan = R.Plan(S.shape[0], S.shape[1], 10, 5, 1, seed=1, compute="f64")
    Sd = dev(S, torch.float64)
    U, sig, C = plan.basis(Sd)
    rec2 = make_recipe(32, 64, 777, 100, ("power", 1.5), seed=4)
    S2 = snapshot_matrix(rec2)
    C2 = plan.project(U, dev(S2, torch.float64))
    ref = oracle_project(U.cpu().numpy(), S2.numpy())
    assert np.abs(C2.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    # projecting the training data reproduces the coefficients
    C1 = plan.project(U, Sd)
    assert np.abs(C1.cpu().numpy() - C.cpu().numpy()).max() <= 1e-10 * sig[0].item()


def test_nonfinite_input_reported():
    rng = np.random.default_rng(0)
    S = torch.from_numpy(rng.standard_normal((200, 100))).t().contiguous().t()
    S[17, 33] = float("nan")
    plan = R.Plan(200, 100, 5, 5, 1, compute="f64")
    plan.basis(dev(S, torch.float64))
    rc, _ = plan.status()
    assert rc == R.RPOD_ERR_NONFINITE
    # the status word is cleared by the read
    rng2 = np.random.default_rng(1)
    plan.basis(dev(torch.from_numpy(rng2.standard_normal((200, 100))).t().contiguous().t(), torch.float64))
    assert plan.status()[0] == R.RPOD_OK


def test_bad_arguments_rejected():
    plan = R.Plan(100, 50, 5, 5, 1, compute="f32")
    S = torch.zeros((50, 100), device="cuda").t()
    with pytest.raises(R.RpodError) as e:
        plan.basis(S.double())        # dtype mismatch
    assert e.value.code == R.RPOD_ERR_INVALID_ARG
    U = torch.empty(1, device="cuda")
    rc = R.rpod_basis(plan.handle, S.data_ptr(), 100, R.RPOD_F32, None, 0, U.data_ptr(), 100,
                      U.data_ptr(), U.data_ptr(), 5, plan.ws_ptr, plan.ws_bytes - 256, 0)
    assert rc == R.RPOD_ERR_WORKSPACE


def test_config2_fp32_full_size_properties():
    """n = 262144 (512 x 512 grid), m = 10000, 400 modes with exp(-j/40)
    amplitudes, k = 100, p = 20, q = 2, FP32: properties that hold at any size
    (the oracle cannot run here): Ritz values interlace the closed-form
    spectrum from below and match it where rPOD has converged, U is
    orthonormal, and sampled coefficient columns equal U_k^T S."""
    rec = make_recipe(512, 512, 10000, 400, ("exp", 40.0), seed=0, noise=1e-6)
    S = snapshot_matrix(rec, device="cuda", dtype=torch.float32)
    closed = np.sqrt(rec.n) / 2 * np.linalg.svd((time_matrix(rec) * rec.amp[None, :]).T,
                                                compute_uv=False)
    k, p, q = 100, 20, 2
    plan = R.Plan(rec.n, rec.m, k, p, q, seed=0, compute="f32")
    U, sig, C = plan.basis(S)
    rc, _ = plan.status()
    assert rc == R.RPOD_OK
    sig = sig.cpu().numpy()
    fp32_floor = 1e-6 * closed[0] + 1e-6 * (np.sqrt(rec.n) + np.sqrt(rec.m))
    assert np.all(sig[:k] <= closed[:k] + fp32_floor)          # interlacing
    assert np.all(np.abs(sig[:50] - closed[:50]) <= 1e-5 * closed[:50] + fp32_floor)
    Uh = U.double().cpu().numpy()
    assert orth_err(Uh) <= 2e-5
    cols = np.random.default_rng(0).choice(rec.m, 16, replace=False)
    Scols = S[:, cols].double().cpu().numpy()
    ref = oracle_project(Uh, Scols)
    Cg = C[:, cols].double().cpu().numpy()
    err = np.abs(Cg - ref).max(axis=0) / np.linalg.norm(Scols, axis=0)
    assert np.all(err <= 2e-5)
    del S
    torch.cuda.empty_cache()


@pytest.mark.parametrize("compute,flags", [("f64", 0), ("bf16", R.RPOD_FLAG_REFINE_FP32 | R.RPOD_FLAG_RETURN_ALL_L)])
def test_basis_file_roundtrip(compute, flags, tmp_path):
    """A basis written by rpod_basis_save and read by rpod_basis_load is the
    same bit for bit, and the plan recreated from the file recomputes it."""
    rec = make_recipe(32, 32, 300, 100, ("power", 1.5), seed=2, noise=1e-6)
    S = snapshot_matrix(rec, dtype=torch.float64 if compute == "f64" else torch.float32)
    plan = R.Plan(rec.n, rec.m, 10, 6, 1, seed=7, compute=compute, flags=flags)
    Sd = S.t().contiguous().cuda().t()
    U, sig, C = plan.basis(Sd)
    path = tmp_path / "basis.rpod"
    plan.save_basis(path, U, sig, C)
    assert R.rpod_basis_file_info(path) == (rec.n, rec.m, 10, 6, 1, 7, plan.compute, flags,
                                            U.shape[1])
    plan2, U2, sig2, C2 = R.load_basis(path)
    assert torch.equal(U, U2) and torch.equal(sig, sig2) and torch.equal(C, C2)
    U3, sig3, C3 = plan2.basis(Sd)
    torch.cuda.synchronize()
    assert torch.equal(sig3, sig2) and torch.equal(U3, U2)


@pytest.mark.parametrize("compute", ["f64", "f32", "bf16"])
def test_workspace_canary_and_output_padding(compute):
    """Stands in for a memory checker: the whole workspace filled with NaN
    bytes before the call changes nothing (no read of workspace bytes the call
    has not written, the status block included), and the padding rows of U and
    C (leading dimensions above n and k) keep their sentinel (no write outside
    the outputs)."""
    rng = np.random.default_rng(17)
    n, m, k, p, q = 1003, 301, 9, 7, 1
    dt = torch.float64 if compute == "f64" else torch.float32
    S = torch.from_numpy(rng.standard_normal((n, m)) * np.logspace(0, -2, m)[None, :]).to(dt)
    Sd = S.t().contiguous().cuda().t()
    flags = R.RPOD_FLAG_REFINE_FP32 if compute == "bf16" else 0

    def run(canary):
        plan = R.Plan(n, m, k, p, q, seed=4, compute=compute, flags=flags)
        if canary:
            plan.ws.fill_(0xFF)
        Ubuf = torch.full((k, n + 5), -7.0, dtype=plan.out_dtype, device="cuda")
        U = Ubuf.t()[:n]                                   # n x k, ld n + 5
        Cbuf = torch.full((m, k + 3), -7.0, dtype=plan.out_dtype, device="cuda")
        C = Cbuf.t()[:k]                                   # k x m, ld k + 3
        sig = torch.empty(k + p, dtype=torch.float64, device="cuda")
        plan.basis(Sd, out=(U, sig, C))
        rc, _ = plan.status()
        return rc, Ubuf, sig, Cbuf

    rc0, U0, s0, C0 = run(False)
    rc1, U1, s1, C1 = run(True)
    assert rc0 == R.RPOD_OK and rc1 == R.RPOD_OK
    assert torch.equal(U0, U1) and torch.equal(s0, s1) and torch.equal(C0, C1)
    assert bool((U1[:, n:] == -7.0).all()) and bool((C1[:, k:] == -7.0).all())
    assert bool(torch.isfinite(U1[:, :n]).all()) and bool(torch.isfinite(C1[:, :k]).all())


def test_bounded_wait_times_out_and_context_survives():
    """Failure detection without a GPU fault: a wait on an mbarrier that
    nothing arrives on gives up after its limit and reports
    RPOD_ERR_TIMEOUT through the status path; the context stays usable."""
    import time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = R.rpod_selftest_wait_timeout(0.05, None)
    dt = time.perf_counter() - t0
    assert rc == R.RPOD_ERR_TIMEOUT
    assert 0.05 <= dt < 1.5, dt
    # the next calls run normally
    rng = np.random.default_rng(3)
    S = torch.from_numpy(rng.standard_normal((300, 120))).t().contiguous().t()
    _, U, sig, C, rc2, _ = run_gpu(dev(S, torch.float64), 5, 3, 1, 1, "f64")
    assert rc2 == R.RPOD_OK and np.all(np.isfinite(sig))


@pytest.mark.parametrize("compute", ["f64", "f32", "bf16"])
def test_host_io_plan_matches_device_plan(compute):
    """RPOD_FLAG_HOST_IO: rpod_basis on pinned host S, U, sigma and C (the
    copies inside the call) gives the device plan's result."""
    rng = np.random.default_rng(21)
    n, m, k, p, q = 1030, 257, 8, 6, 1
    dt = torch.float64 if compute == "f64" else torch.float32
    S = torch.from_numpy(rng.standard_normal((n, m)) * np.logspace(0, -2, m)[None, :]).to(dt)
    flags = R.RPOD_FLAG_REFINE_FP32 if compute == "bf16" else 0
    pd = R.Plan(n, m, k, p, q, seed=6, compute=compute, flags=flags)
    # the device S with the staging copy's 16-element-aligned columns, so both
    # plans take the same (tensor-map) path
    Sd = torch.zeros((m, (n + 15) // 16 * 16), dtype=dt, device="cuda").t()[:n]
    Sd.copy_(S)
    U0, s0, C0 = pd.basis(Sd)
    ph = R.Plan(n, m, k, p, q, seed=6, compute=compute, flags=flags | R.RPOD_FLAG_HOST_IO)
    Sh = torch.empty((m, n + 3), dtype=dt, pin_memory=True).t()[:n]    # ld n + 3
    Sh.copy_(S)
    U1, s1, C1 = ph.basis(Sh)
    torch.cuda.synchronize()
    assert not U1.is_cuda and not C1.is_cuda
    assert ph.status()[0] == R.RPOD_OK
    tol = 1e-12 if compute == "f64" else 1e-6
    assert np.abs(s1.numpy() - s0.cpu().numpy()).max() <= tol * float(s0[0])
    assert np.abs(U1.double().numpy() - U0.double().cpu().numpy()).max() <= 1e3 * tol
    assert np.abs(C1.double().numpy() - C0.double().cpu().numpy()).max() <= tol * 10 * float(s0[0])


@pytest.mark.parametrize("compute", ["f64", "f32", "bf16"])
def test_graph_replay_matches_direct_launches(compute):
    """rpod_plan_set_graph: the second call with the same buffers records the
    plan's kernels into one CUDA graph and later calls replay it.  Replays
    give bit-identical outputs to direct launches, see new contents of S,
    launch the same kernel count, and a call with other buffers launches
    directly (and is still correct)."""
    rng = np.random.default_rng(31)
    n, m, k, p, q = 4100, 700, 20, 10, 2
    dt = torch.float64 if compute == "f64" else torch.float32
    S0, _, _ = lowrank(n, m, 60, seed=5, decay=0.9)
    S1 = S0 * torch.from_numpy(rng.uniform(0.5, 1.5, size=(1, m)))
    flags = R.RPOD_FLAG_REFINE_FP32 if compute == "bf16" else 0
    Sd = dev(S0, dt)
    direct = R.Plan(n, m, k, p, q, seed=4, compute=compute, flags=flags)
    direct.set_graph(False)
    ref0 = [t.clone() for t in direct.basis(Sd)]
    plan = R.Plan(n, m, k, p, q, seed=4, compute=compute, flags=flags)
    odt = torch.float64 if compute == "f64" else torch.float32
    out = (R.empty_colmajor(n, k, odt, "cuda"), torch.empty(k + p, dtype=torch.float64, device="cuda"),
           R.empty_colmajor(k, m, odt, "cuda"))
    counts = []
    for _ in range(4):   # direct, capture + launch, replay, replay
        for t in out:
            t.fill_(float("nan"))
        plan.basis(Sd, out=out)
        torch.cuda.synchronize()
        counts.append(plan.launches())
        assert plan.status()[0] == R.RPOD_OK
        for a, b in zip(out, ref0):
            assert torch.equal(a, b)
    assert len(set(counts)) == 1 and counts[0] > 10
    # new contents of S at the same address: the replay sees them
    Sd.copy_(dev(S1, dt))
    ref1 = [t.clone() for t in direct.basis(Sd)]
    plan.basis(Sd, out=out)
    torch.cuda.synchronize()
    for a, b in zip(out, ref1):
        assert torch.equal(a, b)
    # other buffers: a direct call with the right result
    U2, s2, C2 = plan.basis(Sd)
    torch.cuda.synchronize()
    for a, b in zip((U2, s2, C2), ref1):
        assert torch.equal(a, b)
    # inside a caller's own capture the plan launches directly into it
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.basis(Sd, out=out)
    torch.cuda.current_stream().wait_stream(side)
    Sd.copy_(dev(S0, dt))
    with torch.cuda.graph(g):
        plan.basis(Sd, out=out)
    for t in out:
        t.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert plan.status()[0] == R.RPOD_OK
    for a, b in zip(out, ref0):
        assert torch.equal(a, b)

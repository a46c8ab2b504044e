"""GPU tests of the batched form (many independent instances of Alg. 1 in one
captured CUDA graph) through the C ABI: every instance equals the single-plan
result and the FP64 oracle, graph replays follow the data behind the
pointers, the autotuner keeps results unchanged, and per-instance device
errors are reported with their index."""
import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from oracle.rpod import rpod as oracle_rpod
from synth import batched_recipes, make_recipe, snapshot_matrix, time_matrix
from tests.rpod_checks import max_angle, orth_err, sigma_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def small_batch(count=8, nx=64, ny=64, dtype=torch.float32, seed=1):
    recs, ks = batched_recipes(count=count, nx=nx, ny=ny, m_range=(200, 600), k_choices=(5, 10, 20),
                               J=100, seed=seed)
    S_cpu = [snapshot_matrix(r) for r in recs]
    S = [s.t().contiguous().to(dtype).cuda().t() for s in S_cpu]
    return recs, ks, S_cpu, S


def test_batch_matches_single_plans_and_oracle():
    recs, ks, S_cpu, S = small_batch()
    p, q = 10, 1
    seeds = list(range(100, 100 + len(S)))
    B = R.Batch(S, ks, p, q, seeds, compute="f32")
    B.run()
    rc, bad, _ = B.status()
    assert rc == R.RPOD_OK, (rc, bad)
    for b in range(len(S)):
        plan = R.Plan(S[b].shape[0], S[b].shape[1], ks[b], p, q, seed=seeds[b], compute="f32")
        U, sig, C = plan.basis(S[b])
        torch.cuda.synchronize()
        assert torch.equal(B.sigma[b], sig)
        assert torch.equal(B.U[b], U)
        assert torch.equal(B.C[b], C)
    for b in (0, 3):
        o = oracle_rpod(S_cpu[b].float().double().numpy(), ks[b], p, q, seed=seeds[b])
        k = ks[b]
        ok, er, ea = sigma_close(B.sigma[b].cpu().numpy()[:k], o.sigma[:k], 1e-5, 1e-6)
        assert ok, (b, er, ea)
        assert max_angle(o.U[:, :k], B.U[b].double().cpu().numpy()) <= 1e-4
    assert B.launches() > 10 * len(S)


def test_batch_replay_tracks_data_and_tuning_keeps_results():
    recs, ks, S_cpu, S = small_batch(count=6, seed=2)
    p, q = 10, 1
    B = R.Batch(S, ks, p, q, list(range(6)), compute="f32")
    B.run()
    first = [s.clone() for s in B.sigma]
    # new data behind the same pointers: the replayed graph sees it
    for s in S:
        s.mul_(2.0)
    B.run()
    torch.cuda.synchronize()
    for a, b in zip(first, B.sigma):
        assert torch.allclose(b, 2.0 * a, rtol=1e-5, atol=0)
    streams, split, stages = B.tune(trials=1)
    # the tuner's own candidate sets (worker streams up to the instance count;
    # the FP32 form has no tensor-core passes, so the stage count stays 0)
    assert streams in (1, 2, 4) and split in (25, 50, 100, 200) and stages == 0
    B.run()
    assert B.status()[0] == R.RPOD_OK
    torch.cuda.synchronize()
    # other split counts change the FP32 summation order: compare at FP32
    # rounding relative to sigma_1
    for a, b in zip(first, B.sigma):
        assert torch.allclose(b, 2.0 * a, rtol=1e-5, atol=2e-6 * 2.0 * a[0].item())


def test_batch_reports_failing_instance():
    recs, ks, S_cpu, S = small_batch(count=5, seed=3)
    S[3][5, 7] = float("nan")
    B = R.Batch(S, ks, 10, 1, list(range(5)), compute="f32")
    B.run()
    rc, bad, _ = B.status()
    assert rc == R.RPOD_ERR_NONFINITE and bad == 3


def test_batch_bf16_refine_config4_shapes():
    """Four instances of the 64-instance batch recipe (n = 32768 on a 128 x 256
    grid; m_b 631..2668, k_b 10..50, amplitudes exp(-j/tau_b)), BF16 passes
    with the FP32 refinement pass.  Against the oracle run on the
    BF16-rounded passes (the same storage): sigma_i within 1e-4 for every
    i <= k_b and span(U_k) within 1e-2.  Against the oracle on the FP32
    snapshots: 1e-4 where sigma_i >= 5e-2 sigma_1, and everywhere within the
    storage floor (the rounded-input oracle's own distance from it) plus
    1e-4; the angle within the floor's angle plus 1e-2."""
    from oracle.rpod import round_to
    recs, ks = batched_recipes(count=64, nx=128, ny=256, J=200, seed=0)
    sel = [5, 9, 17, 44]
    recs, ks = [recs[b] for b in sel], [ks[b] for b in sel]
    assert max(ks) == 50 and max(r.m for r in recs) > 2500
    S_cpu = [snapshot_matrix(r, dtype=torch.float32) for r in recs]
    S = [s.t().contiguous().cuda().t() for s in S_cpu]
    seeds = [16 + b for b in sel]
    p, q = 10, 1
    B = R.Batch(S, ks, p, q, seeds, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    B.run()
    assert B.status()[0] == R.RPOD_OK
    for b in range(len(sel)):
        S64 = S_cpu[b].double().numpy()
        k = ks[b]
        orig = oracle_rpod(S64, k, p, q, seed=seeds[b])
        lowp = oracle_rpod(S64, k, p, q, seed=seeds[b], sketch_dtype="bf16",
                           S_passes=round_to(S64, "bf16"))
        sg = B.sigma[b].cpu().numpy()[:k]
        Ub = B.U[b].double().cpu().numpy()
        e_low = np.abs(sg - lowp.sigma[:k]) / lowp.sigma[:k]
        assert e_low.max() <= 1e-4, (b, e_low.max())
        assert max_angle(lowp.U[:, :k], Ub) <= 1e-2, b
        e_orig = np.abs(sg - orig.sigma[:k]) / orig.sigma[:k]
        floor = np.abs(lowp.sigma[:k] - orig.sigma[:k]) / orig.sigma[:k]
        top = orig.sigma[:k] >= 5e-2 * orig.sigma[0]
        assert e_orig[top].max() <= 1e-4, (b, e_orig[top].max())
        assert np.all(e_orig <= floor + 1e-4), (b, (e_orig - floor).max())
        assert max_angle(orig.U[:, :k], Ub) <= max_angle(orig.U[:, :k], lowp.U[:, :k]) + 1e-2, b
        assert orth_err(Ub) <= 1e-5


def test_batch_64_instances_full_size():
    """64 instances (4 fields x 16 parameter samples) on a 128 x 256 grid
    (n = 32768), m_b ~ U{500..3000}, k_b in {10, 20, 30, 50}, p = 10, q = 1,
    amplitudes exp(-j/tau_b), FP32: interlacing against each instance's closed
    form spectrum and orthonormal bases."""
    recs, ks = batched_recipes(count=64, nx=128, ny=256, J=200, seed=0)
    S = [snapshot_matrix(r, device="cuda", dtype=torch.float32) for r in recs]
    B = R.Batch(S, ks, 10, 1, [16 + b for b in range(64)], compute="f32")
    B.run()
    rc, bad, _ = B.status()
    assert rc == R.RPOD_OK, (rc, bad)
    for b in range(0, 64, 9):
        r = recs[b]
        closed = np.sqrt(r.n) / 2 * np.linalg.svd((time_matrix(r) * r.amp[None, :]).T, compute_uv=False)
        sg = B.sigma[b].cpu().numpy()
        k = ks[b]
        floor = 2e-6 * closed[0] + 1e-6 * (np.sqrt(r.n) + np.sqrt(r.m))
        assert np.all(sg[:k] <= closed[:k] + floor)
        # with q = 1 and p = 10 rPOD has its own approximation error on slowly
        # decaying spectra; the leading value is within 1 %
        assert abs(sg[0] - closed[0]) <= 1e-2 * closed[0]
        Ub = B.U[b].double().cpu().numpy()
        keep = sg[:k] > 1e-4 * sg[0]           # directions FP32 resolves
        assert orth_err(Ub[:, keep]) <= 5e-5


def test_tuning_cache_and_pass_stages(tmp_path):
    """The BF16 form's tuner searches the passes' pipeline depth too; a
    second batch of the same shapes takes the configuration from the JSON
    cache without timing, and every configuration gives the same results
    up to FP32 summation order."""
    import time
    recs, ks, S_cpu, S = small_batch(count=4, seed=6)
    p, q = 10, 1
    cache = str(tmp_path / "tune.json")
    B1 = R.Batch(S, ks, p, q, list(range(4)), compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    best = B1.tune(trials=3, cache=cache)
    assert best[2] in (2, 4)
    B1.run()
    assert B1.status()[0] == R.RPOD_OK
    B2 = R.Batch(S, ks, p, q, list(range(4)), compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32)
    t0 = time.perf_counter()
    assert tuple(B2.tune(trials=3, cache=cache)) == tuple(best)
    assert time.perf_counter() - t0 < 0.5          # a cache hit times nothing
    for stages in (2, 4):
        B2.configure(best[0], best[1], stages)
        B2.run()
        assert B2.status()[0] == R.RPOD_OK
        torch.cuda.synchronize()
        for a, b in zip(B1.sigma, B2.sigma):
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * a[0].item())
    assert R.rpod_batch_set_pass_stages(B2.handle, 3) == R.RPOD_ERR_INVALID_ARG

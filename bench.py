#!/usr/bin/env python
"""rPOD time-to-basis benchmark (Alg. 1, Sec. 4.2) on GB300.

Workload: one randomized POD of an FP32 snapshot matrix with n = 262144 rows
(512 x 512 grid) and m = 10000 snapshots of 400 synthetic modes with
amplitudes exp(-j/40) (10.5 GB, column-major, resident in HBM), k = 100,
p = 20, q = 2.  A step is one full rpod_basis call: sketch, every pass over S,
CholeskyQR, T = Q^T S, the small SVD, lift, signs and coefficients.

Forms: "bf16" (16-bit tensor-core passes with the FP32 refinement pass; the
FP32 input is converted during the first pass) and "f32" (plain FP32 SIMT
passes); --form picks the headline, the other is timed beside it when
available.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(nx=512, ny=512, m=10000, J=400, decay=("exp", 40.0), k=100, p=20, q=2,
                seed=0, noise=1e-6)
WORKLOAD_NAME = ("rPOD of FP32 snapshot matrix n=262144 (512x512 grid) x m=10000, "
                 "400 modes exp(-j/40), k=100 p=20 q=2")
METRIC = "rPOD time-to-basis (s)"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
SM_COUNT = 152
FP32_LANES_PER_SM = 128
CPU_SAMPLE_ROWS = (4096, 8192)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto", "bf16", "f32"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="time only the headline form (skip the other precision form)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-instance batched leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the LSTM leg")
    ap.add_argument("--fields-epochs", type=int, default=0,
                    help="epochs of an extra leg with one ROM per field and Table tab:hyperparam's "
                         "networks (0: skipped)")
    ap.add_argument("--no-centered", action="store_true",
                    help="skip the leg with per-sample centering (Eqs. time_av, fluct_q)")
    ap.add_argument("--nt", type=int, default=400,
                    help="snapshots per parameter sample for the centered leg")
    ap.add_argument("--learned-epochs", type=int, default=60)
    ap.add_argument("--learned-centered", action="store_true",
                    help="also run the learned leg on per-sample centered snapshots")
    ap.add_argument("--ny", type=int, default=512,
                    help="grid rows (n = 512 * ny); smaller values make the small profiling case")
    ap.add_argument("--only-batched", choices=["bf16", "f32"], default=None,
                    help="profiling aid: run only the batched leg in this form and print its "
                         "JSON object")
    ap.add_argument("--only-leg", choices=["small-configs", "config6", "learned"], default=None,
                    help="profiling aid: run only this leg and print its JSON object")
    ap.add_argument("--batched-config", default=None,
                    help="STREAMS,SPLIT_PCT[,STAGES]: skip the tuner and use this launch configuration")
    ap.add_argument("--no-small-configs", action="store_true",
                    help="skip the config-1 (FP64) and config-3 (16-bit + refinement) timings")
    ap.add_argument("--no-config6", action="store_true",
                    help="skip the paper-shaped leg (n=8192, m=90225, k=10, p=75, q=1)")
    ap.add_argument("--no-oracle-full", action="store_true",
                    help="skip the full-size FP64 oracle run (cpu_baseline and parity); the "
                         "baseline is then extrapolated from row samples")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_sha(*names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2504_15350_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(form: str):
    """Per-launch DRAM bytes of the dominant pass kernel from profiles/traffic.txt
    (lines: form sha16 bytes_per_launch kernel), valid only while the kernel
    source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_sha(*(["rpod_tc.cu"] if form == "bf16" else ["rpod_simt.cu"]))
    for ln in open(path):
        f = ln.split()
        if len(f) >= 3 and not ln.startswith("#") and f[0] == form and f[1] == want:
            return float(f[2])
    return None


# ---------------------------------------------------------------------------
def cpu_oracle_time(rows: int) -> float:
    """Seconds the FP64 oracle takes for Alg. 1 on the first `rows` grid cells
    of the workload (all m snapshots).  Runs in this process (the caller
    spawns a fresh interpreter)."""
    import numpy as np
    from oracle.rpod import rpod as oracle_rpod
    from synth import make_recipe, snapshot_matrix
    w = WORKLOAD
    rec = make_recipe(w["nx"], w["ny"], w["m"], w["J"], w["decay"], seed=w["seed"], noise=w["noise"])
    S = snapshot_matrix(rec, rows=np.arange(rows), dtype=__import__("torch").float32).double().numpy()
    t0 = time.perf_counter()
    oracle_rpod(S, w["k"], w["p"], w["q"], seed=w["seed"])
    return time.perf_counter() - t0


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_single_thread_sample(rows=4096):
    """The oracle on `rows` of the n grid cells (all m snapshots) in a fresh
    interpreter whose BLAS is limited to one thread."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_oracle_time(%d)))" % (ROOT, rows))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800,
                         env=env)
    if out.returncode != 0:
        return None
    return {"seconds": json.loads(out.stdout.strip().splitlines()[-1]), "threads": 1, "rows": rows,
            "sample": f"FP64 oracle, one BLAS thread, first {rows} of the "
                      f"{WORKLOAD['nx'] * WORKLOAD['ny']} rows, all {WORKLOAD['m']} snapshots"}


def oracle_full_size(S, U, sigma, k, p, q, seed):
    """Runs the FP64 oracle (all host cores) on the full bench matrix -- the
    same device data, copied to the host -- and compares the GPU result
    with it: sigma_i relative error for i <= k and the largest principal
    angle between span(U_k) of the two.  Returns the timing and errors."""
    import numpy as np
    from oracle.rpod import max_principal_angle
    from oracle.rpod import rpod as oracle_rpod
    S64 = S.cpu().double().numpy()                  # column-major (Fortran order)
    t0 = time.perf_counter()
    o = oracle_rpod(S64, k, p, q, seed=seed)
    secs = time.perf_counter() - t0
    del S64
    sg = sigma.cpu().numpy()
    Ug = U.double().cpu().numpy()
    rel = np.abs(sg[:k] - o.sigma[:k]) / o.sigma[:k]
    return {"seconds": secs, "cores": os.cpu_count(), "cpu": cpu_model(),
            "sigma_max_rel_err_i_le_k": float(rel.max()),
            "sigma_rel_err_at": int(rel.argmax()) + 1,
            "max_principal_angle_Uk": max_principal_angle(o.U[:, :k], Ug),
            "bounds": {"sigma": 1e-4, "angle": 1e-2},
            "what": "GPU bf16+f32-refine result vs FP64 oracle (Alg. 1 in numpy, same S and sketch)"}


def cpu_baseline(samples=CPU_SAMPLE_ROWS, repeats=1):
    """Times the oracle in a spawned interpreter at two row counts and
    extrapolates linearly in n (passes, QR of Y, lift and C scale with n;
    the Jacobi SVD of T and the QR of Z do not)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps([min(bench.cpu_oracle_time(r) for _ in range(%d)) for r in %r]))"
            % (ROOT, repeats, list(samples)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        return None, out.stderr[-500:]
    t = json.loads(out.stdout.strip().splitlines()[-1])
    n = WORKLOAD["nx"] * WORKLOAD["ny"]
    n1, n2 = samples
    slope = (t[1] - t[0]) / (n2 - n1)
    est = t[1] + slope * (n - n2)
    return {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 oracle (numpy, default BLAS threads) on the first {n1} and {n2} of the "
                       f"{n} rows, all {WORKLOAD['m']} snapshots: {t[0]:.2f} s and {t[1]:.2f} s, "
                       f"extrapolated linearly in n to the full matrix")}, None


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np
    n = WORKLOAD["nx"] * WORKLOAD["ny"]
    n1, n2 = CPU_SAMPLE_ROWS
    # warm-up steps at both sample sizes give the slope of the linear model
    t1 = min(cpu_oracle_time(n1) for _ in range(max(1, args.warmup // 2)))
    t2w = min(cpu_oracle_time(n2) for _ in range(max(1, args.warmup - args.warmup // 2)))
    times = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = time.perf_counter()
        cpu_oracle_time(n2)
        times.append(time.perf_counter() - s)
    total = time.perf_counter() - t0
    step = total / args.steps
    slope = (t2w - t1) / (n2 - n1)
    value = step + slope * (n - n2)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD_NAME, "sample_rows": n2, "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"each step: FP64 oracle on the first {n2} of {n} rows (all "
                                        f"{WORKLOAD['m']} snapshots); value extrapolated linearly in "
                                        f"n with the slope from warm-up runs at {n1} and {n2} rows")},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_batched(dev, max_over_ranks, barrier, rank=0, world=1, steps=5, form="f32", config=None):
    """64 independent instances (4 fields x 16 parameter samples) on a
    128 x 256 grid, m_b ~ U{500..3000}, k_b in {10, 20, 30, 50}, p = 10,
    q = 1, FP32 snapshots, one captured CUDA graph per run; the launch
    configuration is tuned first.  form "f32": FP32 passes; form "bf16":
    BF16 tensor-core passes (the first one also writes the BF16 copy of
    S) with the FP32 refinement pass.  With N ranks the instances are split
    by cost across ranks (no collective on the data path)."""
    import torch
    import paper_2504_15350_gb300.rpod as R
    from paper_2504_15350_gb300.shard import instance_cost, shard
    from synth import batched_recipes, snapshot_matrix
    recs, ks = batched_recipes(count=64, nx=128, ny=256, J=200, seed=0)
    mine = shard([instance_cost(r.n, r.m, k, 10, 1) for r, k in zip(recs, ks)], world)[rank]
    recs, ks, seeds = [recs[b] for b in mine], [ks[b] for b in mine], [16 + b for b in mine]
    S = [snapshot_matrix(r, device=dev, dtype=torch.float32) for r in recs]
    flags = R.RPOD_FLAG_REFINE_FP32 if form == "bf16" else 0
    B = R.Batch(S, ks, 10, 1, seeds, compute=form, flags=flags, device=dev)
    if config:
        best = tuple(int(v) for v in config.split(","))
        best = best + (0,) * (3 - len(best))
        B.configure(*best)
    else:
        best = B.tune(trials=3)
    B.run()
    rc, bad, _ = B.status()
    if rc != R.RPOD_OK:
        raise RuntimeError(f"batched: instance {bad}: {R.rpod_strerror(rc)}")
    stream = torch.cuda.current_stream(dev)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        B.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps)
    nm = sum(r.n * r.m for r in recs)
    if form == "bf16":
        # first Y-pass reads FP32 S and writes its BF16 copy, 2q BF16 passes,
        # the FP32 refinement pass reads FP32 S
        nbytes = (4 + 2 + 2 * 2 * 1 + 4) * nm
    else:
        nbytes = 4 * (2 * 1 + 2) * nm   # (2q + 2) passes over FP32 S
    out = {"form": form, "instances": 64, "instances_this_rank": len(recs), "n": recs[0].n,
           "sum_m_this_rank": int(sum(r.m for r in recs)),
           "ms_per_batch": ms, "pass_bytes_GB": nbytes / 1e9,
           "effective_GBps": nbytes / (ms * 1e-3) / 1e9, "streams": best[0], "split_pct": best[1],
           "pass_stages": best[2],
           "gpu_launches_per_batch": B.launches(), "graph_launches_per_batch": 1}
    del B, S
    torch.cuda.empty_cache()
    return out


def time_basis(dev, S, k, p, q, compute, flags, warmup, steps, seed=0):
    """Mean CUDA-event time (ms) of rpod_basis on the device matrix S, and
    the plan's pass profile of the timed steps."""
    import torch
    import paper_2504_15350_gb300.rpod as R
    n, m = S.shape
    plan = R.Plan(n, m, k, p, q, seed=seed, compute=compute, flags=flags, device=dev)
    l = k + p
    odt = torch.float64 if compute == "f64" else torch.float32
    out = (R.empty_colmajor(n, k, odt, dev), torch.empty(l, dtype=torch.float64, device=dev),
           R.empty_colmajor(k, m, odt, dev))
    for _ in range(max(warmup, 3)):
        plan.basis(S, out=out)
    rc, _ = plan.status()
    if rc != R.RPOD_OK:
        raise RuntimeError(f"{compute}: device status {R.rpod_strerror(rc)}")
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.basis(S, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    # pass times from a profiled repeat (direct launches, events per pass)
    plan.profile(True)
    for _ in range(steps):
        plan.basis(S, out=out)
    torch.cuda.synchronize()
    passes, pass_ms, pbytes, _ = plan.profile_read()
    plan.profile(False)
    if plan.status()[0] != R.RPOD_OK:
        raise RuntimeError(f"{compute}: device status after timing")
    return e0.elapsed_time(e1) / steps, passes, pass_ms, pbytes, plan.launches()


def run_small_configs(dev, warmup):
    """The config-1 shape (n = 4096 on a 64 x 64 grid, m = 500, 400 modes with
    amplitudes j^-1.5, k = 20, p = 10, q = 1): the plain FP64 form and the
    precision forms (BF16 and FP16 passes with the FP32 refinement pass).  S
    (16 MB in FP64) stays in L2, so these are latency-bound: time-to-basis
    only.  Their accuracy against the oracle is asserted by the GPU tests."""
    import torch
    import paper_2504_15350_gb300.rpod as R
    from synth import make_recipe, snapshot_matrix
    rec = make_recipe(64, 64, 500, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec)
    out = {}
    for name, compute, dtype, flags in (("config1_f64", "f64", torch.float64, 0),
                                        ("config3_bf16_refine", "bf16", torch.float32,
                                         R.RPOD_FLAG_REFINE_FP32),
                                        ("config3_f16_refine", "f16", torch.float32,
                                         R.RPOD_FLAG_REFINE_FP32)):
        Sd = S.t().contiguous().to(dtype).to(dev).t()
        ms, _, _, _, launches = time_basis(dev, Sd, 20, 10, 1, compute, flags, warmup, 20)
        out[name] = {"time_to_basis_s": ms / 1e3, "n": rec.n, "m": rec.m, "k": 20, "p": 10, "q": 1,
                     "form": compute, "kernels_per_call": launches,
                     "note": "S resident in L2: latency-bound, no roofline"}
    return out


def run_config6(dev, warmup, hbm_peak):
    """The paper's own shape (Sec. 4.2, Table tab:cpu_time): n = 8192 grid
    cells (64 x 128, h = 1/64), m = 90225 snapshots (225 parameter samples x
    401 times), k = N^r = 10, p = 75, q = 1, synthetic modes with amplitudes
    j^-1.5 (2.96 GB FP32).  Time-to-basis of both forms, next to the paper's
    worst-case rPOD time of about 6 s on an unstated CPU (context only)."""
    import torch
    import paper_2504_15350_gb300.rpod as R
    from synth import make_recipe, snapshot_matrix
    rec = make_recipe(64, 128, 90225, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec, device=dev, dtype=torch.float32)
    out = {"n": rec.n, "m": rec.m, "k": 10, "p": 75, "q": 1,
           "paper_rpod_s": 6.0, "paper_hardware": "CPU, unstated (Table tab:cpu_time)"}
    for compute, flags in (("bf16", R.RPOD_FLAG_REFINE_FP32), ("f32", 0)):
        ms, passes, pass_ms, pbytes, _ = time_basis(dev, S, 10, 75, 1, compute, flags, warmup, 5)
        d = {"time_to_basis_s": ms / 1e3, "pass_ms_avg": pass_ms / max(passes, 1),
             "passes_per_step": passes / 5}
        if compute == "bf16":
            gbs = pbytes / (pass_ms * 1e-3) / 1e9
            d.update(pass_GBps=gbs, pass_frac_of_measured_hbm=gbs / hbm_peak)
        out[compute] = d
    out["speedup_vs_paper_bf16"] = out["paper_rpod_s"] / out["bf16"]["time_to_basis_s"]
    del S
    torch.cuda.empty_cache()
    return out


def run_learned(dev, epochs, center=False):
    """rPOD-LSTM run (Sec. 4.3, config 5): 2 layers x 256, window 10, batch
    512, rPOD coefficients (k = 50) of 32 parameter samples x 2000 steps of
    the config-1 mode recipe plus a steady parameter-dependent field;
    pushforward training (half of the batches train on windows of the
    network's own predictions, up to 10 steps), stopped when the validation
    loss has not improved for 15 epochs; rollouts of 500 steps for 8
    held-out samples against Galerkin projection.  With `center` the
    snapshots are centered per training sample and the held-out field
    starts from the nearest sample's time average (Eqs. q_approx,
    time_av_zero)."""
    from paper_2504_15350_gb300 import rom
    r = rom.run(rom.ROMConfig(epochs=epochs, patience=15, mean_amp=1.0, center=center,
                              pushforward=10), device=dev)
    return {"epochs": r.epochs_run, "centered": center, "mean_amp": 1.0, "pushforward": 10,
            "val_loss_curve": [round(v, 6) for v in r.val_loss],
            "train_windows_per_s": r.samples_per_s,
            "rollout_steps_per_s": r.rollout_steps_per_s, "rollout_seconds": r.rollout_seconds,
            "final_val_loss": r.val_loss[-1],
            # relative L2 coefficient errors against the Galerkin projection of
            # the held-out snapshots: one step from true windows, the first 10
            # and all 500 autoregressive steps; then Eq. (l2-error) on the
            # time-averaged field with the projection's own floor
            "onestep_err": {"lstm": r.onestep_err_lstm, "persistence": r.onestep_err_persistence},
            "first10_err": {"lstm": r.err_lstm_first10, "persistence": r.err_persistence_first10,
                            "nearest_mu": r.err_nearest_first10},
            "rollout500_err": {"lstm": r.err_lstm, "persistence": r.err_persistence,
                               "nearest_mu": r.err_nearest},
            "tavg_field_err": {"lstm": r.tavg_err_lstm, "persistence": r.tavg_err_persistence,
                               "nearest_mu": r.tavg_err_nearest,
                               "projection_floor": r.tavg_err_projection}}


def run_fields_leg(dev, epochs):
    """One centered rPOD-LSTM ROM per field (q1, q2, psi1, psi2) with the
    paper's per-field networks (M_q: 1 x 100, batch 8; M_psi: 3 x 50, batch
    16, dropout 0.1) on the learned leg's data size."""
    from paper_2504_15350_gb300 import rom
    base = rom.ROMConfig(epochs=epochs, patience=max(4, epochs), mean_amp=1.0, center=True)
    out = {}
    for f, r in rom.run_fields(base, device=dev).items():
        out[f] = {"network": r.network, "epochs": r.epochs_run,
                  "train_windows_per_s": r.samples_per_s, "final_val_loss": r.val_loss[-1],
                  "onestep_err": {"lstm": r.onestep_err_lstm, "persistence": r.onestep_err_persistence},
                  "first10_err": {"lstm": r.err_lstm_first10, "persistence": r.err_persistence_first10,
                                  "nearest_mu": r.err_nearest_first10},
                  "tavg_field_err": {"lstm": r.tavg_err_lstm, "persistence": r.tavg_err_persistence,
                                     "nearest_mu": r.tavg_err_nearest,
                                     "projection_floor": r.tavg_err_projection}}
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    cpu, cpu_err, cpu1 = None, None, None
    full_oracle = (not args.no_cpu_baseline and not args.no_oracle_full and rank == 0 and world == 1
                   and args.ny == 512)
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        # the sampled oracle runs in spawned interpreters before any CUDA work here
        cpu1 = cpu_single_thread_sample()
        if not full_oracle:
            cpu, cpu_err = cpu_baseline()

    import torch
    import torch.distributed as dist
    import paper_2504_15350_gb300.rpod as R
    from paper_2504_15350_gb300.build import build
    from synth import make_recipe, snapshot_matrix

    build()
    R.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    if args.only_leg:
        peaks, _ = load_peaks()
        if args.only_leg == "small-configs":
            out = run_small_configs(dev, args.warmup)
        elif args.only_leg == "config6":
            out = run_config6(dev, args.warmup, peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
        else:
            out = run_learned(dev, args.learned_epochs)
        if rank == 0:
            print(json.dumps({args.only_leg: out}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    if args.only_batched:
        out = run_batched(dev, max_over_ranks, barrier, rank, world, steps=args.steps,
                          form=args.only_batched, config=args.batched_config)
        if rank == 0:
            print(json.dumps({"batched": out}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    w = dict(WORKLOAD)
    w["ny"] = args.ny
    rec = make_recipe(w["nx"], w["ny"], w["m"], w["J"], w["decay"], seed=w["seed"], noise=w["noise"])
    n, m, k, p, q, l = rec.n, rec.m, w["k"], w["p"], w["q"], w["k"] + w["p"]
    S = snapshot_matrix(rec, device=dev, dtype=torch.float32)
    torch.cuda.synchronize()

    forms = []
    have_tc = True
    try:
        probe = R.Plan(256, 256, 4, 4, 1, compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32, device=dev)
        tmp = torch.zeros((256, 256), device=dev).t()
        probe.basis(tmp)
    except R.RpodError as e:
        have_tc = e.code != R.RPOD_ERR_UNSUPPORTED
    head = args.form if args.form != "auto" else ("bf16" if have_tc else "f32")
    forms = [head] + [f for f in ("bf16", "f32") if f != head and (f != "bf16" or have_tc)]
    if args.no_compare:
        forms = forms[:1]

    peaks, peak_src = load_peaks()
    results = {}
    for form in forms:
        if form == "bf16":
            plan = R.Plan(n, m, k, p, q, seed=w["seed"], compute="bf16", flags=R.RPOD_FLAG_REFINE_FP32,
                          device=dev)
        else:
            plan = R.Plan(n, m, k, p, q, seed=w["seed"], compute="f32", device=dev)
        U = R.empty_colmajor(n, k, torch.float32, dev)
        sig = torch.empty(l, dtype=torch.float64, device=dev)
        C = R.empty_colmajor(k, m, torch.float32, dev)
        out = (U, sig, C)
        for _ in range(args.warmup):
            plan.basis(S, out=out)
        rc, _ = plan.status()
        if rc != R.RPOD_OK:
            raise RuntimeError(f"{form}: device status {R.rpod_strerror(rc)}")
        steps = args.steps if form == head else max(3, min(args.steps, 5))
        stream = torch.cuda.current_stream(dev)
        barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local) if form == head else None
        if clk:
            clk.start()
            time.sleep(0.5)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.basis(S, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        clocks = clk.stop() if clk else None
        launches = plan.launches()
        # the same steps again with CUDA events around every pass (a profiled
        # plan launches its kernels directly; the timed steps above replay the
        # plan's CUDA graph)
        plan.profile(True)
        for _ in range(steps):
            plan.basis(S, out=out)
        torch.cuda.synchronize()
        passes, pass_ms, pbytes, pflops = plan.profile_read()
        plan.profile(False)
        rc, _ = plan.status()
        if rc != R.RPOD_OK:
            raise RuntimeError(f"{form}: device status {R.rpod_strerror(rc)}")
        ms = max_over_ranks(ms)
        results[form] = dict(ms=ms, passes=passes, pass_ms=pass_ms, bytes=pbytes, flops=pflops,
                             launches=launches, steps=steps, clocks=clocks, plan=plan, out=out,
                             sigma=sig.cpu().numpy().copy())
    hr = results[head]
    # roofline of the dominant kernel: the passes over S
    per_ms = hr["pass_ms"] / hr["passes"]
    per_bytes = hr["bytes"] / hr["passes"]
    per_flops = hr["flops"] / hr["passes"]
    if head == "bf16":
        peak = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
        ach = per_bytes / (per_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": f"{peak_src} hbm_gbs", "kernel": "passes over S (tcgen05)"}
    else:
        mhz = (hr["clocks"] or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        ach = per_flops / (per_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": f"FP32 FFMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                               f"{mhz:.0f} MHz (median SM clock under load)",
                "kernel": "passes over S (SIMT FP32 GEMM)",
                "achieved_hbm_gbs": per_bytes / (per_ms * 1e-3) / 1e9}
    # recorded for the full bench workload only
    roof["traffic"] = recorded_traffic(head) if args.ny == 512 else None
    roof["pass_ms_avg"] = per_ms
    roof["passes_per_step"] = hr["passes"] / hr["steps"]

    # centering (Eqs. time_av, fluct_q) of M = m / nt samples, then the 16-bit
    # rPOD of the fluctuations: F (FP32) is the refinement copy, H (BF16) the
    # copy the tensor-core passes read
    centered = None
    if not args.no_centered and head == "bf16" and m % args.nt == 0:
        nt = args.nt
        M = m // nt
        F = R.empty_colmajor(n, m, torch.float32, dev)
        H = R.empty_colmajor(n, m, torch.bfloat16, dev)
        Sbar = R.empty_colmajor(n, M, torch.float32, dev)
        fl_out = (F, H, Sbar)
        cplan = R.Plan(n, m, k, p, q, seed=w["seed"], compute="bf16",
                       flags=R.RPOD_FLAG_REFINE_FP32, device=dev)
        Uc = R.empty_colmajor(n, k, torch.float32, dev)
        sigc = torch.empty(l, dtype=torch.float64, device=dev)
        Cc = R.empty_colmajor(k, m, torch.float32, dev)
        stream = torch.cuda.current_stream(dev)

        def centered_step():
            R.fluctuations(S, nt, out=fl_out)
            cplan.basis(H, S_refine=F, out=(Uc, sigc, Cc))

        for _ in range(args.warmup):
            centered_step()
        rc, _ = cplan.status()
        if rc != R.RPOD_OK:
            raise RuntimeError(f"centered: device status {R.rpod_strerror(rc)}")
        csteps = max(3, min(args.steps, 5))
        barrier()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(csteps):
            R.fluctuations(S, nt, out=fl_out)
        c1.record(stream)
        torch.cuda.synchronize()
        fl_ms = max_over_ranks(c0.elapsed_time(c1) / csteps)
        c0.record(stream)
        for _ in range(csteps):
            centered_step()
        c1.record(stream)
        torch.cuda.synchronize()
        barrier()
        cms = max_over_ranks(c0.elapsed_time(c1) / csteps)
        rc, _ = cplan.status()
        if rc != R.RPOD_OK:
            raise RuntimeError(f"centered: device status {R.rpod_strerror(rc)}")
        fl_bytes = n * m * (4 + 4 + 2) + 4 * n * M
        hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
        fl_gbs = fl_bytes / (fl_ms * 1e-3) / 1e9
        centered = {
            "nt": nt, "samples": M, "fluct_ms": fl_ms, "fluct_bytes": fl_bytes,
            "fluct_gbs": fl_gbs, "fluct_frac": fl_gbs / hbm,
            "fluct_peak_source": f"{peak_src} hbm_gbs",
            "time_to_basis_s": cms / 1e3, "steps": csteps,
            "energy_rank_delta_0.9": int(R.energy_rank(sigc, 0.9).item()),
            "energy_rank_delta_0.99": int(R.energy_rank(sigc, 0.99).item()),
            "sigma_1": float(sigc[0]),
        }
        del F, H, Sbar, fl_out, cplan

    # end to end through the C ABI with host buffers: a plan with
    # RPOD_FLAG_HOST_IO takes pinned host S, U, sigma and C, and the copies
    # run inside rpod_basis
    e2e = None
    if not args.no_e2e:
        hflags = (R.RPOD_FLAG_REFINE_FP32 if head == "bf16" else 0) | R.RPOD_FLAG_HOST_IO
        plan = R.Plan(n, m, k, p, q, seed=w["seed"], compute=head, flags=hflags, device=dev)
        S_host = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
        S_host.copy_(S.t())
        U_h = torch.empty((k, n), dtype=torch.float32, pin_memory=True)
        s_h = torch.empty(l, dtype=torch.float64, pin_memory=True)
        C_h = torch.empty((m, k), dtype=torch.float32, pin_memory=True)
        stream = torch.cuda.current_stream(dev)

        def e2e_step():
            plan.basis(S_host.t(), out=(U_h.t(), s_h, C_h.t()))

        for _ in range(2):  # the second call records the plan's graph
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        a1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(a0.elapsed_time(a1) / args.e2e_steps)
        rc, _ = plan.status()
        if rc != R.RPOD_OK:
            raise RuntimeError(f"e2e: device status {R.rpod_strerror(rc)}")
        e2e = {"value": ems / 1e3, "unit": "s", "h2d_bytes_per_step": 4 * n * m,
               "d2h_bytes_per_step": 4 * n * k + 8 * l + 4 * k * m, "steps": args.e2e_steps,
               "api": "rpod_basis with RPOD_FLAG_HOST_IO (pinned host S, U, sigma, C)"}
        del S_host, plan

    batched = batched_f32 = None
    if not args.no_batched:
        batched = run_batched(dev, max_over_ranks, barrier, rank, world, form="bf16")
        batched_f32 = run_batched(dev, max_over_ranks, barrier, rank, world, form="f32")
    small = None if (args.no_small_configs or rank != 0) else run_small_configs(dev, args.warmup)
    hbm_peak = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    cfg6 = None if (args.no_config6 or rank != 0) else run_config6(dev, args.warmup, hbm_peak)
    learned = None if (args.no_learned or rank != 0) else run_learned(dev, args.learned_epochs)
    learned_c = (run_learned(dev, args.learned_epochs, center=True)
                 if (args.learned_centered and not args.no_learned and rank == 0) else None)
    fields = (run_fields_leg(dev, args.fields_epochs)
              if (args.fields_epochs > 0 and rank == 0) else None)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    oracle_full = None
    if full_oracle and "bf16" in results:
        # the FP64 oracle on the same device matrix: the measured CPU baseline
        # and the headline result's parity at full size
        Ub, sb, _ = results["bf16"]["out"]
        oracle_full = oracle_full_size(S, Ub, sb, k, p, q, w["seed"])
        cpu = {"value": oracle_full["seconds"], "unit": "s", "cores": oracle_full["cores"],
               "kind": "oracle", "cpu": oracle_full["cpu"],
               "sample": (f"the full matrix ({n} x {m}, FP64 copy of the device data), numpy "
                          f"BLAS on all {oracle_full['cores']} host cores, one run"),
               "single_thread_sample": cpu1}
    elif cpu is not None:
        cpu["single_thread_sample"] = cpu1
    line = {
        "metric": METRIC, "value": hr["ms"] / 1e3, "unit": "s", "n_gpus": world,
        "steps": hr["steps"], "warmup": args.warmup, "ms_per_step": hr["ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32-refine" if head == "bf16" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME if args.ny == 512 else
                   f"reduced profiling case: {WORKLOAD_NAME} with n={n} (512x{args.ny} grid)",
                   "n": n, "m": m, "k": k, "p": p, "q": q,
                   "form": head, "l2": "inputs larger than L2 (S is 10.5 GB)",
                   "replicas": world},
        "roofline": roof,
        "cpu_baseline": cpu if cpu else ({"value": None, "error": cpu_err} if cpu_err else None),
        "e2e": e2e,
        "gpu_launches": hr["launches"] * hr["steps"],
        "launch_mode": ("each timed call replays the plan's CUDA graph of its kernels "
                        "(rpod_plan_set_graph); pass times from a profiled repeat of the "
                        "same steps with CUDA events around every pass"),
        "clocks": hr["clocks"],
        "throughput_rpod_per_s": world / (hr["ms"] / 1e3),
        "batched": batched,
        "batched_f32": batched_f32,
        "learned": learned,
        "learned_centered": learned_c,
        "centered": centered,
        "oracle_full": oracle_full,
        "small_configs": small,
        "config6_paper_shape": cfg6,
    }
    if fields is not None:
        line["fields"] = fields
    for f, r in results.items():
        if f != head:
            line[f"{f}_time_to_basis_s"] = r["ms"] / 1e3
            line[f"{f}_pass_ms_avg"] = r["pass_ms"] / r["passes"]
    if "f32" in results and head == "bf16":
        line["speedup_vs_f32_plain"] = results["f32"]["ms"] / hr["ms"]
        # accuracy of the 16-bit form on this workload: the FP32 SIMT result
        # (independent kernels, FP32 error ~1e-6 here) as reference, i <= k
        s16, s32 = results["bf16"]["sigma"][:k], results["f32"]["sigma"][:k]
        line["sigma_max_rel_err_vs_f32"] = float(max(abs(a - b) / b for a, b in zip(s16, s32)))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""rPOD-LSTM reduced-order model on synthetic parametric snapshots (Sec. 4.3).

Pipeline (every numerical step of the method runs in librpod's kernels;
torch holds device memory and does the data bookkeeping around them):
  1. snapshot matrix S = [S(mu_1) ... S(mu_M)] (Sec. 4.1 column order: by
     parameter sample, then time) of the synthetic parametric recipe;
  2. with `center`: per-sample time averages and fluctuation snapshots
     (Eqs. (time_av), (fluct_q)) in place, by rpod_fluctuations; then
     randomized POD (Alg. 1) -> basis U_N and coefficients C = U_N^T S;
  3. z-scored coefficient series and parameters, windows of sigma_L steps
     (Eq. (input) without the time column) -> next coefficients;
  4. LSTM training (MSE, Adam with Table tab:hyperparam's learning rate and
     weight decay) on 80 % of the windows, validation loss on the rest, stop
     when it has not improved for `patience` epochs;
  5. held-out parameters: Galerkin projection C' = U_N^T S' of their
     snapshots (the reference coefficients), LSTM rollout from the first sigma_L projected
     steps, and two predictors without the network: persistence of the last
     seed step, and the coefficients of the nearest training parameter sample
     at the same times (the zero-order choice of Eq. (time_av_zero)).
     With `center` the held-out coefficients are those of the snapshots minus
     the zero-order field of Eq. (time_av_zero) (the time average of the
     nearest training sample) and the reconstructed field is that zero-order
     field plus the modes, Eq. (q_approx).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import rpod as R


@dataclass
class ROMConfig:
    nx: int = 64
    ny: int = 64
    J: int = 400
    n_train_mu: int = 32
    n_steps: int = 2000
    n_test_mu: int = 8
    rollout: int = 500
    k: int = 50
    p: int = 10
    q: int = 1
    hidden: int = 256
    layers: int = 2
    window: int = 10
    batch: int = 512
    epochs: int = 500
    lr: float = 1e-3
    weight_decay: float = 1e-5
    seed: int = 0
    patience: int = 25
    fp32_weights: bool = False
    # steady part of the synthetic snapshots (synth.steady_field; 0: none)
    # and per-sample centering with the zero-order field of Eq. (time_av_zero)
    mean_amp: float = 0.0
    center: bool = False
    # dropout between stacked LSTM layers (training passes only)
    dropout: float = 0.0
    # pushforward training: in a fraction of the batches the network first
    # predicts K steps (1 <= K <= pushforward, no gradient through them) from
    # a true window, and the training step then maps the window made of its
    # own last predictions to the true next coefficients -- the inputs a
    # long rollout feeds it (0: one-step training only)
    pushforward: int = 0
    pushforward_frac: float = 0.5


# Table tab:hyperparam: the networks M_{q_l} (potential vorticity) and
# M_{psi_l} (stream function); both MSE, Adam, lr 1e-3, weight decay 1e-5,
# 20 % validation, 500 epochs, tanh.
PAPER_NETWORKS = {
    "q": dict(layers=1, hidden=100, batch=8, dropout=0.0),
    "psi": dict(layers=3, hidden=50, batch=16, dropout=0.1),
}
# the four fields of the two-layer quasi-geostrophic model, one ROM each
FIELDS = ("q1", "q2", "psi1", "psi2")


@dataclass
class ROMResult:
    train_loss: list = field(default_factory=list)
    val_loss: list = field(default_factory=list)
    err_lstm: float = math.nan
    err_persistence: float = math.nan
    err_nearest: float = math.nan
    train_seconds: float = 0.0
    samples_per_s: float = 0.0
    rollout_seconds: float = 0.0
    rollout_steps_per_s: float = 0.0
    epochs_run: int = 0
    network: dict = field(default_factory=dict)   # layers, hidden, batch, dropout
    sigma: list = field(default_factory=list)
    # Eq. (l2-error): relative L2 error of the time-averaged field over the
    # prediction window, for the LSTM, the two predictors without it, and the
    # projection of the true coefficients (the floor set by the basis)
    tavg_err_lstm: float = math.nan
    tavg_err_persistence: float = math.nan
    tavg_err_nearest: float = math.nan
    tavg_err_projection: float = math.nan
    err_lstm_first50: float = math.nan
    err_lstm_first10: float = math.nan
    err_persistence_first10: float = math.nan
    err_nearest_first10: float = math.nan
    # held-out one-step prediction from true windows (teacher forcing)
    onestep_err_lstm: float = math.nan
    onestep_err_persistence: float = math.nan
    onestep_err_nearest: float = math.nan


def _snapshots(cfg: ROMConfig, mus, m, device, noise_stream0):
    from synth import parametric_recipe, snapshot_matrix, steady_field
    blocks = []
    for i, mu in enumerate(mus):
        rec = parametric_recipe(cfg.nx, cfg.ny, m, cfg.J, mu, seed=cfg.seed,
                                noise_stream=noise_stream0 + i)
        blk = snapshot_matrix(rec, device=device, dtype=torch.float32).t()  # (m, n)
        if cfg.mean_amp:
            sf = steady_field(cfg.nx, cfg.ny, mu, cfg.mean_amp)
            blk += torch.from_numpy(sf).to(device=device, dtype=torch.float32)[None, :]
        blocks.append(blk)
    return torch.cat(blocks, 0).t()   # column-major n x (M m)


def _rel_err(pred, ref):
    """Relative L2 error over all steps and modes, averaged over samples."""
    num = torch.linalg.vector_norm(pred - ref, dim=(1, 2))
    den = torch.linalg.vector_norm(ref, dim=(1, 2))
    return float((num / den).mean())


def _pushforward_batch(net, zs, zmu, rows, K, d, T, n_steps):
    """Training pair for pushforward: the true window at (series, t0) (t0
    moved back so that t0 + T + K is a step of the series), K predictions of
    the network from it (the library's rollout; only data bookkeeping here),
    the window of the last T steps of [true window, predictions], and the
    true coefficients at t0 + T + K."""
    rows = rows.clone()
    rows[:, 1] = torch.clamp(rows[:, 1], max=n_steps - T - 1 - K)
    Xt, _ = net.gather(zs, zmu, rows)
    pred = net.rollout(Xt, d, K)                                 # (B, K, O)
    alpha = torch.cat([Xt[:, :, d:], pred], 1)[:, -T:]
    X = torch.cat([Xt[:, :, :d], alpha], -1).contiguous()
    Y = zs[rows[:, 0].long(), (rows[:, 1] + T + K).long()].contiguous()
    return X, Y


def init_params(net: "R.LSTM", seed: int) -> torch.Tensor:
    """U(-1/sqrt(H), 1/sqrt(H)) for every parameter (the usual LSTM init)."""
    g = torch.Generator().manual_seed(seed)
    H = net.dims[1]
    return (torch.rand(net.P, generator=g, dtype=torch.float32) * 2 - 1) / math.sqrt(H)


def run(cfg: ROMConfig = ROMConfig(), device="cuda", log=None) -> ROMResult:
    dev = torch.device(device)
    rng = np.random.default_rng(cfg.seed + 12345)
    mu_tr = rng.uniform(0.0, 1.0, (cfg.n_train_mu, 4))
    mu_te = rng.uniform(0.0, 1.0, (cfg.n_test_mu, 4))
    res = ROMResult()
    res.network = dict(layers=cfg.layers, hidden=cfg.hidden, batch=cfg.batch, dropout=cfg.dropout)
    O, d, T = cfg.k, 4, cfg.window
    # 1-2: snapshots and randomized POD
    S = _snapshots(cfg, mu_tr, cfg.n_steps, dev, 100)
    n, m = S.shape
    Sbar = None
    if cfg.center:
        # Eqs. (time_av), (fluct_q): S becomes the fluctuation snapshots
        _, _, Sbar = R.fluctuations(S, cfg.n_steps, in_place=True)   # n x M
    plan = R.Plan(n, m, cfg.k, cfg.p, cfg.q, seed=cfg.seed, compute="f32", device=dev)
    U, sig, C = plan.basis(S)
    rc, _ = plan.status()
    if rc != R.RPOD_OK:
        raise R.RpodError(rc, "rpod_basis")
    res.sigma = sig[: cfg.k].cpu().tolist()
    if log:
        log(f"rPOD of {n} x {m} done: sigma_1 {res.sigma[0]:.4e}, sigma_k {res.sigma[-1]:.4e}")
    del S
    series = C.t().contiguous().reshape(cfg.n_train_mu, cfg.n_steps, O)      # (M, t, N)
    # 3: z-scores from the training series
    c_mean = series.reshape(-1, O).mean(0)
    c_std = series.reshape(-1, O).std(0) + 1e-12
    mu_t = torch.tensor(mu_tr, dtype=torch.float32, device=dev)
    m_mean, m_std = mu_t.mean(0), mu_t.std(0) + 1e-12
    zs = ((series - c_mean) / c_std).contiguous()
    zmu = ((mu_t - m_mean) / m_std).contiguous()
    starts = cfg.n_steps - T
    ii, tt = torch.meshgrid(torch.arange(cfg.n_train_mu), torch.arange(starts), indexing="ij")
    idx_all = torch.stack([ii.reshape(-1), tt.reshape(-1)], -1).to(torch.int32)
    g = torch.Generator().manual_seed(cfg.seed)
    perm = torch.randperm(idx_all.shape[0], generator=g)
    n_val = idx_all.shape[0] // 5
    idx_val = idx_all[perm[:n_val]].to(dev)
    idx_tr = idx_all[perm[n_val:]].to(dev)
    # 4: training
    net = R.LSTM(d + O, cfg.hidden, cfg.layers, O, T, max_batch=cfg.batch, device=dev,
                 fp32_weights=cfg.fp32_weights)
    net.set_params(init_params(net, cfg.seed))
    if cfg.dropout > 0.0:
        net.set_dropout(cfg.dropout, cfg.seed)
    B = cfg.batch
    nb = idx_tr.shape[0] // B
    best, best_theta, since = math.inf, None, 0
    t0 = time.perf_counter()
    samples = 0
    pf_rng = np.random.default_rng(cfg.seed + 7)
    for ep in range(cfg.epochs):
        order = idx_tr[torch.randperm(idx_tr.shape[0], generator=g).to(dev)]
        loss_sum = torch.zeros((), device=dev)
        for b in range(nb):
            rows = order[b * B:(b + 1) * B]
            if cfg.pushforward > 0 and pf_rng.random() < cfg.pushforward_frac:
                X, Y = _pushforward_batch(net, zs, zmu, rows, int(pf_rng.integers(1, cfg.pushforward + 1)),
                                          d, T, cfg.n_steps)
            else:
                X, Y = net.gather(zs, zmu, rows)
            loss_sum += net.train_step(X, Y, lr=cfg.lr, weight_decay=cfg.weight_decay)[0]
        samples += nb * B
        vl = torch.zeros((), device=dev)
        nvb = max(1, idx_val.shape[0] // B)
        for b in range(nvb):
            X, Y = net.gather(zs, zmu, idx_val[b * B:(b + 1) * B])
            yh = net.forward(X)
            vl += ((yh - Y) ** 2).mean()
        tl, vl = float(loss_sum) / nb, float(vl) / nvb
        res.train_loss.append(tl)
        res.val_loss.append(vl)
        if log:
            log(f"epoch {ep}: train {tl:.3e} val {vl:.3e}")
        if vl < best * (1 - 1e-3):
            best, best_theta, since = vl, net.get_params().clone(), 0
        else:
            since += 1
            if since >= cfg.patience:
                break
    torch.cuda.synchronize(dev)
    res.train_seconds = time.perf_counter() - t0
    res.samples_per_s = samples / res.train_seconds
    res.epochs_run = len(res.train_loss)
    if best_theta is not None:
        net.set_params(best_theta)
    # 5: held-out parameters, judged by Galerkin projection
    dist = torch.cdist(torch.tensor(mu_te), torch.tensor(mu_tr))
    near = dist.argmin(1).to(dev)
    Ste = _snapshots(cfg, mu_te, T + cfg.rollout, dev, 500)
    Cte = plan.project(U, Ste)                                   # k x (M' (T + r))
    L_ = T + cfg.rollout
    q0 = None
    if cfg.center:
        # zero-order fields of Eq. (time_av_zero): the time average of the
        # nearest training sample; coefficients of the snapshots minus it
        q0 = Sbar[:, near.cpu()].t().contiguous().t()               # n x M'
        c0 = plan.project(U, q0)                                  # k x M'
        Cte = Cte - c0.repeat_interleave(L_, dim=1)
    # time-averaged true fields over the prediction window, one per sample
    fom_avg = torch.stack([Ste[:, i * L_ + T:(i + 1) * L_].mean(1) for i in range(cfg.n_test_mu)], 0)
    del Ste
    truth = Cte.t().contiguous().reshape(cfg.n_test_mu, T + cfg.rollout, O)
    zmu_te = ((torch.tensor(mu_te, dtype=torch.float32, device=dev) - m_mean) / m_std)
    zt = (truth - c_mean) / c_std
    win = torch.cat([zmu_te[:, None, :].expand(-1, T, -1), zt[:, :T]], -1).contiguous()
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    pred = net.rollout(win, d, cfg.rollout)
    torch.cuda.synchronize(dev)
    res.rollout_seconds = time.perf_counter() - t1
    res.rollout_steps_per_s = cfg.rollout / res.rollout_seconds
    pred = pred * c_std + c_mean
    ref = truth[:, T:]
    res.err_lstm = _rel_err(pred, ref)
    res.err_persistence = _rel_err(truth[:, T - 1:T].expand(-1, cfg.rollout, -1), ref)
    res.err_nearest = _rel_err(series[near, T:T + cfg.rollout], ref)
    res.err_lstm_first50 = _rel_err(pred[:, :50], ref[:, :50])
    res.err_lstm_first10 = _rel_err(pred[:, :10], ref[:, :10])
    res.err_persistence_first10 = _rel_err(truth[:, T - 1:T].expand(-1, 10, -1), ref[:, :10])
    res.err_nearest_first10 = _rel_err(series[near, T:T + 10], ref[:, :10])
    # one-step predictions from true held-out windows
    idx_te = torch.stack(torch.meshgrid(torch.arange(cfg.n_test_mu), torch.arange(cfg.rollout),
                                        indexing="ij"), -1).reshape(-1, 2).to(torch.int32).to(dev)
    one = []
    for b0 in range(0, idx_te.shape[0], B):
        Xw, _ = net.gather(zt.contiguous(), zmu_te.contiguous(), idx_te[b0:b0 + B])
        one.append(net.forward(Xw))
    one = (torch.cat(one, 0) * c_std + c_mean).reshape(cfg.n_test_mu, cfg.rollout, O)
    res.onestep_err_lstm = _rel_err(one, ref)
    res.onestep_err_persistence = _rel_err(truth[:, T - 1:T + cfg.rollout - 1], ref)
    res.onestep_err_nearest = res.err_nearest

    def tavg_err(coeffs):   # coeffs (M', r, N) -> mean over samples of Eq. (l2-error)
        rom_avg = coeffs.mean(1) @ U.t()                       # (M', n)
        if q0 is not None:                                     # Eq. (q_approx)
            rom_avg = rom_avg + q0.t()
        num = torch.linalg.vector_norm(rom_avg - fom_avg, dim=1)
        return float((num / torch.linalg.vector_norm(fom_avg, dim=1)).mean())

    res.tavg_err_lstm = tavg_err(pred)
    res.tavg_err_persistence = tavg_err(truth[:, T - 1:T].expand(-1, cfg.rollout, -1))
    res.tavg_err_nearest = tavg_err(series[near, T:T + cfg.rollout])
    res.tavg_err_projection = tavg_err(ref)
    if log:
        log(f"rollout {cfg.rollout} steps in {res.rollout_seconds:.3f} s; trajectory rel err LSTM "
            f"{res.err_lstm:.4f} (first 50 steps {res.err_lstm_first50:.4f}), persistence "
            f"{res.err_persistence:.4f}, nearest mu {res.err_nearest:.4f}; time-averaged field err "
            f"LSTM {res.tavg_err_lstm:.4f}, persistence {res.tavg_err_persistence:.4f}, nearest mu "
            f"{res.tavg_err_nearest:.4f}, projection floor {res.tavg_err_projection:.4f}; one-step err "
            f"LSTM {res.onestep_err_lstm:.4f}, persistence {res.onestep_err_persistence:.4f}; first 10 steps "
            f"LSTM {res.err_lstm_first10:.4f}, persistence {res.err_persistence_first10:.4f}, nearest mu "
            f"{res.err_nearest_first10:.4f}")
    return res


def run_fields(base: ROMConfig = ROMConfig(mean_amp=1.0, center=True), fields=FIELDS,
               device="cuda", log=None) -> dict:
    """One rPOD-LSTM ROM per field (Sec. 4.3: M_{q_l} and M_{psi_l}), each
    with its own synthetic snapshots (the field's seed offsets the base
    seed) and the per-field network of Table tab:hyperparam; everything else
    (grid, samples, steps, epochs, centering) from `base`.  Returns
    {field: ROMResult}."""
    from dataclasses import replace
    out = {}
    for i, fname in enumerate(fields):
        kind = "q" if fname.startswith("q") else "psi"
        cfg = replace(base, seed=base.seed + 101 * (i + 1), **PAPER_NETWORKS[kind])
        if log:
            log(f"field {fname}: {PAPER_NETWORKS[kind]}")
        out[fname] = run(cfg, device=device, log=log)
    return out

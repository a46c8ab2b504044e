"""End-to-end rPOD-LSTM ROM (Sec. 4.3) on the GPU: rPOD coefficients of 32
parameter samples x 2000 steps, LSTM trained by the library's kernels, rollouts
for 8 held-out parameter samples judged against the Galerkin projection of
their snapshots.

The trained network must do better than the two predictors without it --
persistence of the last seed step and the nearest training sample's
coefficients -- on the held-out one-step (teacher-forced) prediction, on the
first 10 autoregressive steps, and at the paper's horizon: over all 500
autoregressive steps and on the time-averaged field of Eq. (l2-error).  The
long horizon needs pushforward training (the network also learns from
windows made of its own predictions): trained one step at a time, its
free-running rollout drifts out of phase and loses to both predictors."""
import math

import pytest

from paper_2504_15350_gb300 import rom

pytestmark = pytest.mark.gpu


def test_lstm_beats_no_lstm_predictors_short_horizon():
    from paper_2504_15350_gb300.build import build
    build()
    import time
    t0 = time.time()
    cfg = rom.ROMConfig(epochs=40, patience=40)
    res = rom.run(cfg, log=lambda s: print(f"[{time.time() - t0:7.1f}s] {s}", flush=True))
    print(f"\none-step LSTM {res.onestep_err_lstm:.4f} persistence {res.onestep_err_persistence:.4f}; "
          f"first 10 LSTM {res.err_lstm_first10:.4f} persistence {res.err_persistence_first10:.4f} "
          f"nearest-mu {res.err_nearest_first10:.4f}; 500 steps LSTM {res.err_lstm:.4f} "
          f"persistence {res.err_persistence:.4f} nearest-mu {res.err_nearest:.4f}; "
          f"train {res.samples_per_s:.0f} windows/s  rollout {res.rollout_steps_per_s:.0f} steps/s")
    assert math.isfinite(res.err_lstm)
    assert res.val_loss[-1] < res.val_loss[0]
    assert res.onestep_err_lstm <= 0.6 * res.onestep_err_persistence
    assert res.err_lstm_first10 <= 0.5 * min(res.err_persistence_first10,
                                             res.err_nearest_first10)


def test_lstm_beats_no_lstm_predictors_at_500_steps():
    """Config 5 with a steady parameter-dependent part in the snapshots (so
    that Eq. (l2-error) is well posed), raw rPOD coefficients, pushforward
    training (up to 10 predicted steps in half of the batches), 60 epochs.
    Over the 500-step rollout the LSTM's coefficient error is below both
    predictors without it, and its time-averaged field error is below both
    and within 0.1, the top of the paper's stated field-error range (1e-2 ..
    1e-1).  Measured: 500 steps 0.42 vs persistence 0.58 and nearest sample
    0.48; time-averaged field 0.059 vs 0.44 and 0.100."""
    from paper_2504_15350_gb300.build import build
    build()
    cfg = rom.ROMConfig(epochs=60, patience=15, mean_amp=1.0, center=False, pushforward=10)
    res = rom.run(cfg)
    print(f"\n500 steps: LSTM {res.err_lstm:.4f} persistence {res.err_persistence:.4f} nearest-mu "
          f"{res.err_nearest:.4f}; time-averaged field: LSTM {res.tavg_err_lstm:.4f} persistence "
          f"{res.tavg_err_persistence:.4f} nearest-mu {res.tavg_err_nearest:.4f} floor "
          f"{res.tavg_err_projection:.4f}; epochs {res.epochs_run}")
    assert res.err_lstm <= 0.95 * min(res.err_persistence, res.err_nearest)
    assert res.tavg_err_lstm <= 0.8 * min(res.tavg_err_persistence, res.tavg_err_nearest)
    assert res.tavg_err_lstm <= 0.1
    assert res.tavg_err_projection <= 0.02


def test_centered_rom_zero_order_field():
    """Snapshots with steady parameter-dependent mean fields, centered per
    training sample (Eqs. (time_av), (fluct_q)) before the rPOD; held-out
    fields reconstructed as the nearest sample's time average plus the modes
    (Eqs. (q_approx), (time_av_zero)).  The time-averaged-field error of
    Eq. (l2-error) is then well posed: the projection floor is small, and the
    LSTM's time-averaged field beats persistence of the seed window (measured
    0.16 vs 0.44, floor 0.003, at 15 epochs)."""
    from paper_2504_15350_gb300.build import build
    build()
    cfg = rom.ROMConfig(epochs=15, patience=15, mean_amp=1.0, center=True)
    res = rom.run(cfg)
    print(f"\ntime-averaged field err: LSTM {res.tavg_err_lstm:.4f} persistence "
          f"{res.tavg_err_persistence:.4f} nearest-mu {res.tavg_err_nearest:.4f} floor "
          f"{res.tavg_err_projection:.4f}; one-step LSTM {res.onestep_err_lstm:.4f} persistence "
          f"{res.onestep_err_persistence:.4f}")
    assert math.isfinite(res.tavg_err_lstm)
    assert res.tavg_err_projection <= 0.02
    assert res.tavg_err_lstm <= 0.6 * res.tavg_err_persistence
    assert res.onestep_err_lstm <= 0.8 * res.onestep_err_persistence


def test_per_field_networks_of_the_paper():
    """One ROM per field (q1, q2, psi1, psi2) with Table tab:hyperparam's
    networks: M_q 1 layer x 100 cells, batch 8; M_psi 3 layers x 50 cells,
    batch 16, dropout 0.1.  A small configuration (8 samples x 300 steps,
    10 epochs): every field's validation loss falls by at least 5x and its
    basis reproduces the held-out time-averaged field to within 5 %.  (At
    this size the networks do not yet beat persistence on held-out samples;
    that comparison is the 2 x 256 network's, above.)"""
    from paper_2504_15350_gb300.build import build
    build()
    base = rom.ROMConfig(mean_amp=1.0, center=True, n_train_mu=8, n_steps=300, n_test_mu=4,
                         rollout=100, k=20, p=10, epochs=10, patience=10)
    res = rom.run_fields(base)
    assert set(res) == set(rom.FIELDS)
    for f, r in res.items():
        kind = "q" if f.startswith("q") else "psi"
        assert r.network == rom.PAPER_NETWORKS[kind], f
        assert math.isfinite(r.tavg_err_lstm), f
        assert r.val_loss[-1] <= 0.2 * r.val_loss[0], (f, r.val_loss[0], r.val_loss[-1])
        assert r.tavg_err_projection <= 0.05, (f, r.tavg_err_projection)

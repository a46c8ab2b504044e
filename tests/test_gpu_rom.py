"""End-to-end rPOD-LSTM ROM (Sec. 4.3) on the GPU: rPOD coefficients of 32
parameter samples x 2000 steps, LSTM trained by the library's kernels, 500-step
rollouts for 8 held-out parameter samples judged against the Galerkin
projection of their snapshots.  The trained network must do clearly better
than the two predictors without it: persistence of the last seed step and
the nearest training sample's coefficients (Eq. (time_av_zero))."""
import math

import pytest

from paper_2504_15350_gb300 import rom

pytestmark = pytest.mark.gpu


def test_lstm_rollout_beats_no_lstm_predictors():
    from paper_2504_15350_gb300.build import build
    build()
    import time
    t0 = time.time()
    cfg = rom.ROMConfig(epochs=40, patience=8)
    res = rom.run(cfg, log=lambda s: print(f"[{time.time() - t0:7.1f}s] {s}", flush=True))
    print(f"\nLSTM {res.err_lstm:.4f}  persistence {res.err_persistence:.4f}  "
          f"nearest-mu {res.err_nearest:.4f}  epochs {res.epochs_run}  "
          f"train {res.samples_per_s:.0f} windows/s  rollout {res.rollout_steps_per_s:.0f} steps/s")
    assert math.isfinite(res.err_lstm)
    assert res.val_loss[-1] < res.val_loss[0]
    assert res.err_lstm <= 0.5 * min(res.err_persistence, res.err_nearest)

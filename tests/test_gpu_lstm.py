"""GPU tests of the LSTM kernels (Sec. 4.3) through the C ABI against the FP64
oracle (oracle/lstm.py).  By default the library multiplies by BF16 copies of
the weight matrices, so the oracle runs at the same BF16-rounded weights
(biases exact); what remains is FP32 activations and accumulation.  With FP32
weights the oracle runs at the FP32 parameters themselves."""
import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from oracle import lstm as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def bf16_weights(theta, I, H, L, O):
    """theta with every weight matrix rounded to BF16 (biases unchanged)."""
    out = theta.copy()
    off = 0
    for shp in OL.param_shapes(I, H, L, O):
        n = int(np.prod(shp))
        if len(shp) == 2:
            blk = torch.from_numpy(out[off:off + n].astype(np.float32)).to(torch.bfloat16).double().numpy()
            out[off:off + n] = blk
        off += n
    return out


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-30))


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("I,H,L,O,T,B", [(6, 32, 2, 4, 5, 16), (54, 64, 2, 50, 10, 40), (5, 16, 1, 3, 3, 7)])
def test_forward_and_gradients_match_oracle(I, H, L, O, T, B, fp32):
    rng = np.random.default_rng(I * H + B)
    theta = rng.uniform(-0.3, 0.3, OL.param_count(I, H, L, O)).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((B, T, I)).astype(np.float32)
    Yt = rng.standard_normal((B, O)).astype(np.float32)
    te = theta if fp32 else bf16_weights(theta, I, H, L, O)
    y_o, cache = OL.forward(te, X.astype(np.float64), H, L, O)
    loss_o, dy = OL.mse(y_o, Yt.astype(np.float64))
    g_o = OL.backward(te, cache, dy, H, L, O)

    net = R.LSTM(I, H, L, O, T, max_batch=64, theta=theta, fp32_weights=fp32)
    Xd = torch.from_numpy(X).cuda()
    y = net.forward(Xd).cpu().numpy()
    assert rel(y, y_o) < 2e-5
    loss, g = net.loss_grad(Xd, torch.from_numpy(Yt).cuda())
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_o) <= 1e-5 * loss_o
    g = g.cpu().numpy()
    # every parameter block separately (relative to the block's scale)
    off = 0
    for shp in OL.param_shapes(I, H, L, O):
        n = int(np.prod(shp))
        assert rel(g[off:off + n], g_o[off:off + n]) < 2e-4, shp
        off += n
    assert net.launches() > 2 * T


def test_adam_step_matches_oracle():
    I, H, L, O, T, B = 6, 32, 2, 4, 5, 16
    rng = np.random.default_rng(3)
    theta = rng.uniform(-0.3, 0.3, OL.param_count(I, H, L, O)).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((B, T, I)).astype(np.float32)
    Yt = rng.standard_normal((B, O)).astype(np.float32)
    net = R.LSTM(I, H, L, O, T, max_batch=B, theta=theta)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Yt).cuda()
    th = theta.copy()
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for step in (1, 2, 3):
        te = bf16_weights(th, I, H, L, O)
        y_o, cache = OL.forward(te, X.astype(np.float64), H, L, O)
        _, dy = OL.mse(y_o, Yt.astype(np.float64))
        g_o = OL.backward(te, cache, dy, H, L, O)
        th, m, v = OL.adam_step(th, g_o, m, v, step, lr=1e-3, weight_decay=1e-5)
        net.train_step(Xd, Yd, lr=1e-3, weight_decay=1e-5)
    got = net.get_params().cpu().numpy()
    # three Adam steps move each weight by about 3e-3; compare the moves
    assert rel(got - theta, th - theta) < 2e-3


@pytest.mark.parametrize("fp32", [False, True])
def test_rollout_matches_oracle(fp32):
    I, H, L, O, T, B = 7, 32, 2, 5, 4, 3
    rng = np.random.default_rng(5)
    theta = rng.uniform(-0.4, 0.4, OL.param_count(I, H, L, O)).astype(np.float32).astype(np.float64)
    win = rng.standard_normal((B, T, I)).astype(np.float32)
    te = theta if fp32 else bf16_weights(theta, I, H, L, O)
    ref = OL.rollout(te, win.astype(np.float64), 2, 6, H, L, O)
    net = R.LSTM(I, H, L, O, T, max_batch=8, theta=theta, fp32_weights=fp32)
    out = net.rollout(torch.from_numpy(win).cuda(), 2, 6).cpu().numpy()
    assert rel(out, ref) < 1e-4


def test_gather_builds_windows():
    I, H, L, O, T = 7, 16, 1, 5, 4
    net = R.LSTM(I, H, L, O, T, max_batch=8)
    rng = np.random.default_rng(0)
    series = torch.from_numpy(rng.standard_normal((3, 20, O)).astype(np.float32)).cuda()
    mu = torch.from_numpy(rng.standard_normal((3, 2)).astype(np.float32)).cuda()
    idx = torch.tensor([[0, 0], [2, 15], [1, 7]], dtype=torch.int32).cuda()
    X, Y = net.gather(series, mu, idx)
    s, m_, X, Y = series.cpu(), mu.cpu(), X.cpu(), Y.cpu()
    for b, (si, t0) in enumerate([(0, 0), (2, 15), (1, 7)]):
        for t in range(T):
            assert torch.equal(X[b, t, :2], m_[si])
            assert torch.equal(X[b, t, 2:], s[si, t0 + t])
        assert torch.equal(Y[b], s[si, t0 + T])


@pytest.mark.parametrize("p", [0.1, 0.5])
@pytest.mark.parametrize("I,H,L,O,T,B", [(54, 50, 3, 50, 10, 16), (6, 32, 2, 4, 5, 13)])
def test_dropout_training_passes_match_oracle(I, H, L, O, T, B, p):
    """Training passes with dropout between stacked layers (Table
    tab:hyperparam's stream-function networks: 3 layers x 50, dropout 0.1):
    loss and gradients of passes 0 and 1 against the oracle drawing the same
    counter-based masks; inference is unmasked."""
    rng = np.random.default_rng(I + H + L + int(10 * p))
    theta = rng.uniform(-0.3, 0.3, OL.param_count(I, H, L, O)).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((B, T, I)).astype(np.float32)
    Yt = rng.standard_normal((B, O)).astype(np.float32)
    te = bf16_weights(theta, I, H, L, O)
    seed = 1234
    net = R.LSTM(I, H, L, O, T, max_batch=64, theta=theta)
    net.set_dropout(p, seed)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Yt).cuda()
    for step in range(2):
        y_o, cache = OL.forward(te, X.astype(np.float64), H, L, O, dropout=(p, seed, step))
        loss_o, dy = OL.mse(y_o, Yt.astype(np.float64))
        g_o = OL.backward(te, cache, dy, H, L, O)
        loss, g = net.loss_grad(Xd, Yd)
        torch.cuda.synchronize()
        assert abs(loss.item() - loss_o) <= 1e-5 * loss_o, step
        g = g.cpu().numpy()
        off = 0
        for shp in OL.param_shapes(I, H, L, O):
            n = int(np.prod(shp))
            assert rel(g[off:off + n], g_o[off:off + n]) < 2e-4, (step, shp)
            off += n
    # inference ignores the mask
    y_o, _ = OL.forward(te, X.astype(np.float64), H, L, O)
    assert rel(net.forward(Xd).cpu().numpy(), y_o) < 2e-5
    # p = 0 switches it off again
    net.set_dropout(0.0, seed)
    y_o, cache = OL.forward(te, X.astype(np.float64), H, L, O)
    loss_o, _ = OL.mse(y_o, Yt.astype(np.float64))
    loss, _ = net.loss_grad(Xd, Yd)
    assert abs(loss.item() - loss_o) <= 1e-5 * loss_o


def _series(n_series=5, t_len=40, O=4, d=2, seed=0):
    g = torch.Generator().manual_seed(seed)
    series = torch.randn((n_series, t_len, O), generator=g).cuda()
    mu = torch.rand((n_series, d), generator=g).cuda()
    return series, mu


def test_train_epoch_equals_step_loop():
    """rpod_lstm_train_epoch = gather + train_step over the same batches:
    the same kernels in the same order, so the parameters agree bit for bit
    and the reported loss is the mean of the step losses."""
    I, H, L, O, T, B = 6, 16, 2, 4, 5, 8
    series, mu = _series(O=O, d=I - O)
    n_series, t_len = series.shape[:2]
    g = torch.Generator().manual_seed(3)
    pairs = torch.stack(torch.meshgrid(torch.arange(n_series), torch.arange(t_len - T),
                                       indexing="ij"), -1).reshape(-1, 2)
    idx = pairs[torch.randperm(pairs.shape[0], generator=g)].to(torch.int32).cuda()
    theta = np.random.default_rng(1).uniform(-0.3, 0.3, OL.param_count(I, H, L, O))
    a = R.LSTM(I, H, L, O, T, max_batch=B, theta=theta)
    b = R.LSTM(I, H, L, O, T, max_batch=B, theta=theta)
    a.set_dropout(0.2, 9)
    b.set_dropout(0.2, 9)
    mean = a.train_epoch(series, mu, idx, B).item()
    losses = []
    nb = idx.shape[0] // B
    for k in range(nb):
        X, Y = b.gather(series, mu, idx[k * B:(k + 1) * B])
        losses.append(b.train_step(X, Y)[0].item())
    torch.cuda.synchronize()
    assert torch.equal(a.get_params(), b.get_params())
    assert abs(mean - float(np.mean(losses))) <= 1e-6 * abs(float(np.mean(losses)))
    assert a.launches() > nb * 10


def test_save_load_restore_continues_training(tmp_path):
    """A saved network, loaded and restored into a new workspace, holds the
    same parameters and continues with the same Adam state and dropout
    pass count: the next training step matches the original bit for bit."""
    I, H, L, O, T, B = 6, 16, 3, 4, 5, 8
    series, mu = _series(O=O, d=I - O, seed=2)
    idx = torch.tensor([[s, t] for s in range(3) for t in range(0, 30, 3)], dtype=torch.int32).cuda()
    theta = np.random.default_rng(2).uniform(-0.3, 0.3, OL.param_count(I, H, L, O))
    a = R.LSTM(I, H, L, O, T, max_batch=B, theta=theta)
    a.set_dropout(0.1, 4)
    a.train_epoch(series, mu, idx, B)
    path = tmp_path / "net.rpodlstm"
    a.save(path)
    c = R.LSTM.load(path)
    assert c.dims == a.dims and c.max_batch == a.max_batch
    assert torch.equal(a.get_params(), c.get_params())
    X, Y = a.gather(series, mu, idx[:B])
    la = a.train_step(X, Y)[0].item()
    lc = c.train_step(X, Y)[0].item()
    torch.cuda.synchronize()
    assert la == lc
    assert torch.equal(a.get_params(), c.get_params())


def test_config5_shape_forward_gradients_and_rollout():
    """Config 5's network at full size: 54 inputs (4 parameters + 50
    coefficients), 2 layers x 256 cells, window 10, batch 512, weights
    U(+-1/sqrt(H)) as trained; forward, loss and every gradient block
    against the FP64 oracle at the same BF16-rounded weights, and a 50-step
    autoregressive rollout of 8 windows."""
    I, H, L, O, T, B = 54, 256, 2, 50, 10, 512
    rng = np.random.default_rng(55)
    theta = (rng.uniform(-1.0, 1.0, OL.param_count(I, H, L, O)) / np.sqrt(H)).astype(np.float32)
    theta = theta.astype(np.float64)
    X = rng.standard_normal((B, T, I)).astype(np.float32)
    Yt = rng.standard_normal((B, O)).astype(np.float32)
    te = bf16_weights(theta, I, H, L, O)
    y_o, cache = OL.forward(te, X.astype(np.float64), H, L, O)
    loss_o, dy = OL.mse(y_o, Yt.astype(np.float64))
    g_o = OL.backward(te, cache, dy, H, L, O)
    net = R.LSTM(I, H, L, O, T, max_batch=B, theta=theta)
    Xd = torch.from_numpy(X).cuda()
    assert rel(net.forward(Xd).cpu().numpy(), y_o) < 2e-5
    loss, g = net.loss_grad(Xd, torch.from_numpy(Yt).cuda())
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_o) <= 1e-5 * loss_o
    g = g.cpu().numpy()
    off = 0
    for shp in OL.param_shapes(I, H, L, O):
        n = int(np.prod(shp))
        assert rel(g[off:off + n], g_o[off:off + n]) < 2e-4, shp
        off += n
    win = rng.standard_normal((8, T, I)).astype(np.float32)
    ref = OL.rollout(te, win.astype(np.float64), 4, 50, H, L, O)
    out = net.rollout(torch.from_numpy(win).cuda(), 4, 50).cpu().numpy()
    assert rel(out, ref) < 1e-4, rel(out, ref)


def test_persistent_and_per_step_rollouts_agree():
    """8 windows fit the persistent rollout kernel (weights resident in
    shared memory, a grid barrier per anti-diagonal of layer x time cells);
    64 windows of the same network exceed its shared memory and take the
    per-step kernels.  Both match the oracle and each other on the shared
    windows over 60 steps, and the persistent run leaves an OK status."""
    I, H, L, O, T = 54, 256, 2, 50, 10
    rng = np.random.default_rng(77)
    theta = (rng.uniform(-1.0, 1.0, OL.param_count(I, H, L, O)) / np.sqrt(H)).astype(np.float32)
    theta = theta.astype(np.float64)
    win = rng.standard_normal((64, T, I)).astype(np.float32)
    net = R.LSTM(I, H, L, O, T, max_batch=64, theta=theta)
    big = net.rollout(torch.from_numpy(win).cuda(), 4, 60).cpu().numpy()
    small = net.rollout(torch.from_numpy(win[:8]).cuda(), 4, 60).cpu().numpy()
    assert net.status() == R.RPOD_OK
    assert rel(small, big[:8]) < 1e-5, rel(small, big[:8])
    ref = OL.rollout(bf16_weights(theta, I, H, L, O), win[:8].astype(np.float64), 4, 60, H, L, O)
    assert rel(small, ref) < 1e-4
    assert net.launches() < 5      # one cooperative launch (plus the window copy)


def test_grid_barrier_limit_reports_timeout():
    """A grid barrier whose last arrival never comes: the bounded wait runs
    out after 50 ms, the kernel records RPOD_ERR_TIMEOUT and returns, and the
    context stays usable (a rollout right after it succeeds)."""
    st = torch.cuda.current_stream().cuda_stream
    assert R.rpod_selftest_grid_barrier(0.05, st) == R.RPOD_ERR_TIMEOUT
    assert R.rpod_selftest_grid_barrier(3.0, st) == R.RPOD_ERR_INVALID_ARG
    I, H, L, O, T = 7, 32, 2, 5, 4
    rng = np.random.default_rng(1)
    theta = rng.uniform(-0.4, 0.4, OL.param_count(I, H, L, O))
    net = R.LSTM(I, H, L, O, T, max_batch=8, theta=theta)
    out = net.rollout(torch.from_numpy(rng.standard_normal((3, T, I)).astype(np.float32)).cuda(), 2, 5)
    assert net.status() == R.RPOD_OK and torch.isfinite(out).all()

"""Pins for the FP64 LSTM oracle (Sec. 4.3, Table tab:hyperparam): forward and
gradients against torch.nn.LSTM/autograd in float64 (a library routine with
the same cell), central finite differences, and a hand-worked Adam step."""
import numpy as np
import pytest
import torch

from oracle import lstm as L


def _rand_theta(I, H, Ly, O, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, L.param_count(I, H, Ly, O))


def _torch_model(theta, I, H, Ly, O):
    P = L.unflatten(theta, I, H, Ly, O)
    lstm = torch.nn.LSTM(I, H, num_layers=Ly, batch_first=True).double()
    head = torch.nn.Linear(H, O).double()
    with torch.no_grad():
        for l in range(Ly):
            getattr(lstm, f"weight_ih_l{l}").copy_(torch.from_numpy(P[3 * l]))
            getattr(lstm, f"weight_hh_l{l}").copy_(torch.from_numpy(P[3 * l + 1]))
            getattr(lstm, f"bias_ih_l{l}").copy_(torch.from_numpy(P[3 * l + 2]))
            getattr(lstm, f"bias_hh_l{l}").zero_()
        head.weight.copy_(torch.from_numpy(P[3 * Ly]))
        head.bias.copy_(torch.from_numpy(P[3 * Ly + 1]))
    return lstm, head


@pytest.mark.parametrize("I,H,Ly,O,T,B", [(5, 4, 2, 3, 3, 2), (7, 6, 1, 2, 5, 3), (3, 5, 3, 4, 4, 2)])
def test_forward_and_grad_match_torch(I, H, Ly, O, T, B):
    theta = _rand_theta(I, H, Ly, O, seed=I * H)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((B, T, I))
    tgt = rng.standard_normal((B, O))
    y, cache = L.forward(theta, X, H, Ly, O)
    loss, dy = L.mse(y, tgt)
    g = L.backward(theta, cache, dy, H, Ly, O)

    lstm, head = _torch_model(theta, I, H, Ly, O)
    out, _ = lstm(torch.from_numpy(X))
    yt = head(out[:, -1, :])
    lt = torch.nn.functional.mse_loss(yt, torch.from_numpy(tgt))
    lt.backward()
    assert np.allclose(y, yt.detach().numpy(), rtol=1e-13, atol=1e-14)
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    gt = []
    for l in range(Ly):
        gt += [getattr(lstm, f"weight_ih_l{l}").grad, getattr(lstm, f"weight_hh_l{l}").grad,
               getattr(lstm, f"bias_ih_l{l}").grad]
    gt += [head.weight.grad, head.bias.grad]
    gt = np.concatenate([x.numpy().ravel() for x in gt])
    assert np.allclose(g, gt, rtol=1e-12, atol=1e-14)


def test_grad_central_differences():
    I, H, Ly, O, T, B = 5, 4, 2, 3, 3, 2
    theta = _rand_theta(I, H, Ly, O, seed=3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((B, T, I))
    tgt = rng.standard_normal((B, O))
    y, cache = L.forward(theta, X, H, Ly, O)
    _, dy = L.mse(y, tgt)
    g = L.backward(theta, cache, dy, H, Ly, O)
    h = 1e-6
    fd = np.zeros_like(theta)
    for j in range(theta.size):
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        fd[j] = (L.mse(L.forward(tp, X, H, Ly, O)[0], tgt)[0]
                 - L.mse(L.forward(tm, X, H, Ly, O)[0], tgt)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)


def test_zero_weights_special_case():
    # all weights zero, gate biases (b_i, b_f, b_g, b_o): every unit follows
    # c_t = s(b_f) c_{t-1} + s(b_i) tanh(b_g), a geometric series
    I, H, O, T = 2, 3, 1, 6
    theta = np.zeros(L.param_count(I, H, 1, O))
    P = L.unflatten(theta, I, H, 1, O)
    bi, bf, bg, bo = 0.3, 1.2, -0.7, 0.1
    b = np.concatenate([np.full(H, bi), np.full(H, bf), np.full(H, bg), np.full(H, bo)])
    off = 4 * H * I + 4 * H * H
    theta[off:off + 4 * H] = b
    theta[off + 4 * H:off + 4 * H + H] = 1.0     # W_y = ones
    s = lambda x: 1 / (1 + np.exp(-x))
    a, r = s(bi) * np.tanh(bg), s(bf)
    cT = a * (1 - r ** T) / (1 - r)
    y, _ = L.forward(theta, np.random.default_rng(0).standard_normal((2, T, I)), H, 1, O)
    assert np.allclose(y, H * s(bo) * np.tanh(cT), rtol=1e-14)


def test_rollout_zero_weights_closed_form():
    """Rollout of a two-layer network whose weights are zero and whose gate
    biases are (b_i, b_f, b_g, b_o) in both layers: each unit of each layer
    follows c_t = s(b_f) c_{t-1} + s(b_i) tanh(b_g) whatever its input, so
    every step predicts H s(b_o) tanh(c_T) + b_y for each output (W_y = ones)
    -- the same value at all steps, from any window; the rollout's output
    has one row per step and output."""
    I, H, Ly, O, T, B, mu = 5, 3, 2, 3, 4, 2, 2
    theta = np.zeros(L.param_count(I, H, Ly, O))
    bi, bf, bg, bo, by = -0.4, 0.8, 0.6, 0.3, -0.25
    b = np.concatenate([np.full(H, bi), np.full(H, bf), np.full(H, bg), np.full(H, bo)])
    off = 0
    for l in range(Ly):
        il = I if l == 0 else H
        off += 4 * H * il + 4 * H * H
        theta[off:off + 4 * H] = b
        off += 4 * H
    theta[off:off + O * H] = 1.0                  # W_y = ones
    theta[off + O * H:off + O * H + O] = by       # b_y
    s = lambda x: 1 / (1 + np.exp(-x))
    a, r = s(bi) * np.tanh(bg), s(bf)
    cT = a * (1 - r ** T) / (1 - r)
    expect = H * s(bo) * np.tanh(cT) + by
    win = np.random.default_rng(4).standard_normal((B, T, I)) * 3.0
    out = L.rollout(theta, win, mu, 7, H, Ly, O)
    assert out.shape == (B, 7, O)
    assert np.allclose(out, expect, rtol=1e-14, atol=1e-15)


def test_adam_hand_example():
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2); v = np.zeros(2)
    th, m, v = L.adam_step(theta, g, m, v, 1, lr=0.1, weight_decay=0.0)
    # first step with bias correction moves each weight by lr * sign(g) (eps aside)
    assert np.allclose(th, [0.9, -1.9], atol=1e-7)
    th2, m2, v2 = L.adam_step(th, np.array([0.5, 0.5]), m, v, 2, lr=0.1, weight_decay=0.0)
    # m = 0.9*0.05 + 0.05 = 0.095 / (1-0.81); v = 0.999*0.00025 + 0.00025
    m_hat = np.array([0.095, 0.9 * -0.025 + 0.05]) / 0.19
    v_hat = np.array([0.999 * 0.00025 + 0.001 * 0.25, 0.999 * 0.0000625 + 0.001 * 0.25]) / (1 - 0.999 ** 2)
    assert np.allclose(th2, th - 0.1 * m_hat / (np.sqrt(v_hat) + 1e-8), rtol=1e-14)
    # weight decay enters as g + wd * theta
    th3, _, _ = L.adam_step(np.array([2.0]), np.array([0.0]), np.zeros(1), np.zeros(1), 1,
                            lr=0.1, weight_decay=0.5)
    assert th3[0] == pytest.approx(1.9, abs=1e-7)


def test_rollout_shifts_window():
    I, H, Ly, O, T, B = 6, 4, 1, 4, 3, 2
    theta = _rand_theta(I, H, Ly, O, seed=9)
    rng = np.random.default_rng(2)
    win = rng.standard_normal((B, T, I))
    out = L.rollout(theta, win, 2, 3, H, Ly, O)
    y0, _ = L.forward(theta, win, H, Ly, O)
    assert np.allclose(out[:, 0], y0)
    w1 = np.concatenate([win[:, 1:], np.concatenate([win[:, -1:, :2], y0[:, None]], axis=2)], axis=1)
    y1, _ = L.forward(theta, w1, H, Ly, O)
    assert np.allclose(out[:, 1], y1)


# ---- dropout between stacked layers (Table tab:hyperparam) ----------------
def test_dropout_mask_words_from_numpy_philox():
    # word e mod 4 of the block with counter (e div 4, layer, step, 0) under
    # key (seed, 1): numpy's Philox increments the counter before each block
    seed, step, layer, T, B, H, p = 11, 7, 2, 3, 5, 6, 0.3
    keep = L.dropout_keep(p, seed, step, layer, T, B, H).ravel()
    thr = int(np.ceil(p * 2.0 ** 53))
    n = T * B * H
    ref = np.empty(n)
    for blk in range((n + 3) // 4):
        c = blk + (layer << 64) + (step << 128)
        c -= 1
        ctr = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        bg = np.random.Philox(key=np.array([seed, 1], dtype=np.uint64), counter=ctr)
        w = bg.random_raw(4)
        for q in range(4):
            if 4 * blk + q < n:
                ref[4 * blk + q] = 1.0 if (int(w[q]) >> 11) >= thr else 0.0
    assert np.array_equal(keep, ref)


def test_dropout_zero_probability_is_no_dropout():
    I, H, Ly, O, T, B = 5, 4, 3, 3, 4, 3
    theta = _rand_theta(I, H, Ly, O, seed=5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((B, T, I))
    tgt = rng.standard_normal((B, O))
    y0, c0 = L.forward(theta, X, H, Ly, O)
    y1, c1 = L.forward(theta, X, H, Ly, O, dropout=(0.0, 3, 9))
    assert np.array_equal(y0, y1)
    _, dy = L.mse(y0, tgt)
    assert np.array_equal(L.backward(theta, c0, dy, H, Ly, O), L.backward(theta, c1, dy, H, Ly, O))


def test_dropout_keep_fraction_and_independence():
    p, T, B, H = 0.1, 10, 64, 50
    k = L.dropout_keep(p, 1, 0, 1, T, B, H)
    n = k.size
    assert abs(k.mean() - (1 - p)) <= 5 * np.sqrt(p * (1 - p) / n)
    # other passes, layers and seeds draw other masks
    for args in ((1, 1, 1), (1, 0, 2), (2, 0, 1)):
        k2 = L.dropout_keep(p, args[0], args[1], args[2], T, B, H)
        agree = (k == k2).mean()
        # independent masks agree on (1-p)^2 + p^2 of the entries
        assert abs(agree - ((1 - p) ** 2 + p * p)) <= 5 * np.sqrt(0.25 / n)


def test_dropout_grad_central_differences():
    # with a fixed mask the loss is a smooth function of theta
    I, H, Ly, O, T, B = 4, 5, 3, 2, 3, 4
    theta = _rand_theta(I, H, Ly, O, seed=8)
    rng = np.random.default_rng(9)
    X = rng.standard_normal((B, T, I))
    tgt = rng.standard_normal((B, O))
    drop = (0.3, 21, 4)
    y, cache = L.forward(theta, X, H, Ly, O, dropout=drop)
    _, dy = L.mse(y, tgt)
    g = L.backward(theta, cache, dy, H, Ly, O)
    # the mask really removes inputs of layers 1 and 2
    assert cache[1][4] is not None and (cache[1][4] == 0).any()
    h = 1e-6
    fd = np.zeros_like(theta)
    for j in range(theta.size):
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        fd[j] = (L.mse(L.forward(tp, X, H, Ly, O, dropout=drop)[0], tgt)[0]
                 - L.mse(L.forward(tm, X, H, Ly, O, dropout=drop)[0], tgt)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)


def test_dropout_first_layer_input_untouched():
    # one layer: nothing to mask, dropout changes nothing
    I, H, O, T, B = 3, 4, 2, 3, 2
    theta = _rand_theta(I, H, 1, O, seed=10)
    X = np.random.default_rng(11).standard_normal((B, T, I))
    assert np.array_equal(L.forward(theta, X, H, 1, O)[0],
                          L.forward(theta, X, H, 1, O, dropout=(0.5, 1, 0))[0])

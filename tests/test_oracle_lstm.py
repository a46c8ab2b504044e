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

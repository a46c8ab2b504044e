"""LSTM forward, backpropagation through time and Adam in FP64 (oracle; test
infrastructure).

Sec. 4.3 trains one LSTM (Hochreiter & Schmidhuber 1997) per field on windows
of sigma_L time steps of the modal coefficients plus the physical parameters
(Eq. (input)) and targets the coefficients at the next time; Table
(tab:hyperparam) fixes MSE loss, Adam with learning rate 1e-3 and weight
decay 1e-5, tanh activation.  The paper writes no cell equations; the oracle
takes the standard cell:

    z = W_x x_t + W_h h_{t-1} + b,   z = [z_i, z_f, z_g, z_o]  (4H rows)
    i = logistic(z_i), f = logistic(z_f), g = tanh(z_g), o = logistic(z_o)
    c_t = f * c_{t-1} + i * g,        h_t = o * tanh(c_t),   h_0 = c_0 = 0

stacked in `layers` layers (layer l+1 reads h of layer l), followed by a
linear head y = W_y h_T + b_y on the top layer's last state.  Loss
L = mean((y - y*)^2) over batch and outputs.  Adam (Kingma & Ba 2015) with the
weight decay added to the gradient (g <- g + wd * theta), beta1 = 0.9,
beta2 = 0.999, eps = 1e-8, bias-corrected moments.

Flat parameter layout (shared by the oracle and the library's interface, not
its code): for each layer l: W_x (4H x I_l, row-major), W_h (4H x H), b (4H);
then W_y (O x H), b_y (O).  I_0 = in_dim, I_l = H above.

Dropout (Table tab:hyperparam gives probability 0.1 for the stream-function
networks and no placement): in training, the input of every layer above the
first (the h_1..h_T of the layer below) is multiplied by keep / (1 - p), the
usual placement between stacked layers; the recurrent state, the first
layer's input and the head's input are not masked, and inference uses no
mask.  keep for element e = (t B + b) H + j of the input to layer l at
training pass s comes from a counter-based generator so that any
implementation draws the same mask: word e mod 4 of the Philox4x64-10 block
with counter (e div 4, l, s, 0) and key (seed, 1); keep = 1 when that word
shifted right by 11 bits is at least ceil(p 2^53).
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x64


def param_shapes(in_dim: int, hidden: int, layers: int, out_dim: int):
    shapes = []
    for l in range(layers):
        il = in_dim if l == 0 else hidden
        shapes += [(4 * hidden, il), (4 * hidden, hidden), (4 * hidden,)]
    shapes += [(out_dim, hidden), (out_dim,)]
    return shapes


def param_count(in_dim, hidden, layers, out_dim) -> int:
    return int(sum(np.prod(s) for s in param_shapes(in_dim, hidden, layers, out_dim)))


def unflatten(theta, in_dim, hidden, layers, out_dim):
    out, off = [], 0
    for s in param_shapes(in_dim, hidden, layers, out_dim):
        n = int(np.prod(s))
        out.append(np.asarray(theta[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return out


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def dropout_keep(p: float, seed: int, step: int, layer: int, T: int, B: int, H: int) -> np.ndarray:
    """The keep mask (T, B, H) of the input to `layer` at training pass
    `step`, as defined in the module header (1 = kept)."""
    n = T * B * H
    e = np.arange(n, dtype=np.uint64)
    blocks = np.arange((n + 3) // 4, dtype=np.uint64)
    ctr = np.zeros((len(blocks), 4), dtype=np.uint64)
    ctr[:, 0] = blocks
    ctr[:, 1] = np.uint64(layer)
    ctr[:, 2] = np.uint64(step)
    key = np.array([seed, 1], dtype=np.uint64)
    w = philox4x64(ctr, key)                                  # (blocks, 4)
    word = w[(e >> np.uint64(2)).astype(np.int64), (e & np.uint64(3)).astype(np.int64)]
    thr = np.uint64(int(np.ceil(p * 2.0 ** 53)))
    return ((word >> np.uint64(11)) >= thr).astype(np.float64).reshape(T, B, H)


def forward(theta, X, hidden, layers, out_dim, dropout=None):
    """X: (B, T, I).  Returns (y (B, O), cache).  dropout = (p, seed, step)
    for a training pass with dropout, None for none."""
    X = np.asarray(X, dtype=np.float64)
    B, T, I = X.shape
    P = unflatten(theta, I, hidden, layers, out_dim)
    H = hidden
    inp = X
    cache = []
    for l in range(layers):
        Wx, Wh, b = P[3 * l], P[3 * l + 1], P[3 * l + 2]
        scale = None
        if dropout is not None and l > 0 and dropout[0] > 0.0:
            p, seed, step = dropout
            keep = dropout_keep(p, seed, step, l, T, B, H)          # (T, B, H)
            scale = keep.transpose(1, 0, 2) / (1.0 - p)            # (B, T, H)
            inp = inp * scale
        h = np.zeros((B, H))
        c = np.zeros((B, H))
        hs, cs, gates = [h], [c], []
        for t in range(T):
            z = inp[:, t, :] @ Wx.T + h @ Wh.T + b
            i = _sig(z[:, 0:H])
            f = _sig(z[:, H:2 * H])
            g = np.tanh(z[:, 2 * H:3 * H])
            o = _sig(z[:, 3 * H:4 * H])
            c = f * c + i * g
            h = o * np.tanh(c)
            hs.append(h)
            cs.append(c)
            gates.append((i, f, g, o))
        cache.append((inp, hs, cs, gates, scale))
        inp = np.stack(hs[1:], axis=1)
    Wy, by = P[3 * layers], P[3 * layers + 1]
    hT = cache[-1][1][-1]
    y = hT @ Wy.T + by
    return y, cache


def mse(y, target):
    d = np.asarray(y, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(theta, cache, dy, hidden, layers, out_dim):
    """Gradient of the loss w.r.t. the flat parameters, given dL/dy."""
    inp0 = cache[0][0]
    B, T, I = inp0.shape
    H = hidden
    P = unflatten(theta, I, hidden, layers, out_dim)
    G = [np.zeros_like(p) for p in P]
    Wy = P[3 * layers]
    hT = cache[-1][1][-1]
    G[3 * layers] = dy.T @ hT
    G[3 * layers + 1] = dy.sum(axis=0)
    dh_ext = np.zeros((B, T, H))
    dh_ext[:, T - 1, :] = dy @ Wy
    for l in reversed(range(layers)):
        Wx, Wh = P[3 * l], P[3 * l + 1]
        inp, hs, cs, gates, scale = cache[l]
        dWx = np.zeros_like(Wx)
        dWh = np.zeros_like(Wh)
        db = np.zeros(4 * H)
        dinp = np.zeros_like(inp)
        dh_rec = np.zeros((B, H))
        dc_next = np.zeros((B, H))
        for t in reversed(range(T)):
            i, f, g, o = gates[t]
            c, c_prev, h_prev = cs[t + 1], cs[t], hs[t]
            dh = dh_ext[:, t, :] + dh_rec
            tc = np.tanh(c)
            do = dh * tc
            dc = dc_next + dh * o * (1.0 - tc * tc)
            di = dc * g
            dg = dc * i
            df = dc * c_prev
            dc_next = dc * f
            dz = np.concatenate([di * i * (1 - i), df * f * (1 - f),
                                 dg * (1 - g * g), do * o * (1 - o)], axis=1)
            dWx += dz.T @ inp[:, t, :]
            dWh += dz.T @ h_prev
            db += dz.sum(axis=0)
            dinp[:, t, :] = dz @ Wx
            dh_rec = dz @ Wh
        G[3 * l], G[3 * l + 1], G[3 * l + 2] = dWx, dWh, db
        # the masked input was scale * h of the layer below
        dh_ext = dinp if scale is None else dinp * scale
    return np.concatenate([g.ravel() for g in G])


def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999,
              eps=1e-8, weight_decay=1e-5):
    """One Adam update (step counts from 1).  Returns (theta, m, v)."""
    g = np.asarray(grad, np.float64) + weight_decay * np.asarray(theta, np.float64)
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def rollout(theta, window, mu_cols: int, steps: int, hidden, layers, out_dim):
    """Autoregressive prediction (Sec. 4.3; online stage of Sec. 6): from a
    (B, T, I) window whose first `mu_cols` columns are the (fixed) parameter
    inputs and whose remaining columns are the coefficients, predict the next
    coefficients, append [mu, prediction] as the newest row, drop the oldest,
    repeat.  Returns (B, steps, out_dim)."""
    win = np.array(window, dtype=np.float64, copy=True)
    B, T, I = win.shape
    assert I == mu_cols + out_dim
    out = np.zeros((B, steps, out_dim))
    for s in range(steps):
        y, _ = forward(theta, win, hidden, layers, out_dim)
        out[:, s, :] = y
        new = np.concatenate([win[:, -1, :mu_cols], y], axis=1)
        win = np.concatenate([win[:, 1:, :], new[:, None, :]], axis=1)
    return out

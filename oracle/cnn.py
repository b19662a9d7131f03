"""Plain CPU reference of the learned initial-guess network (oracle, test infrastructure).

The paper has no learned component; this network is the GMRES initial-guess
model of the GPU build.  It is L layers of 3x3 convolutions with circular
padding on an H x W grid, ReLU after every layer but the last:

    a_0 = input                       (Cin_0 channels)
    y_l[co, p] = b_l[co] + sum_{t, ci} W_l[t, co, ci] a_{l-1}[ci, p + d_t]
    a_l = relu(y_l)  (l < L),  a_L = y_L

with taps t = 3 (dy + 1) + (dx + 1), d_t = (dy, dx) in {-1, 0, 1}^2 and
p + d_t taken modulo the grid.  Arrays are NHWC: a[n, y, x, c].

Precision: float64 throughout.  With ``bf16=True`` the weights and every
stored activation are rounded to bfloat16 (round to nearest even) where the
GPU kernels store them, so that both compute the same function up to the
order of the float32 sums.

Backward pass for a loss with gradient G = dloss/da_L: for l = L..1,
    g = G (l = L)  or  G * [y_l > 0]
    dW_l[t, co, ci] = sum_{n, p} g[n, p, co] a_{l-1}[n, p + d_t, ci]
    db_l[co]        = sum_{n, p} g[n, p, co]
    G <- dloss/da_{l-1}[n, q, ci] = sum_{t, co} W_l[t, co, ci] g[n, q - d_t, co]
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(a: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[n, y, x, c] = a[n, (y + dy) mod H, (x + dx) mod W, c]."""
    return np.roll(a, (-dy, -dx), axis=(1, 2))


def conv(a: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n, p, co] = b[co] + sum_{t, ci} W[t, co, ci] a[n, p + d_t, ci]."""
    y = np.zeros(a.shape[:3] + (W.shape[1],)) + b
    for t, (dy, dx) in enumerate(TAPS):
        y += shift(a, dy, dx) @ W[t].T
    return y


def forward(x, weights, biases, bf16=False):
    """Returns (activations a_0..a_L, pre-activations y_1..y_L)."""
    acts = [bf16_round(x) if bf16 else np.asarray(x, np.float64)]
    pres = []
    L = len(weights)
    for l, (W, b) in enumerate(zip(weights, biases)):
        Wq = bf16_round(W) if bf16 else W
        y = conv(acts[-1], Wq, b)
        pres.append(y)
        a = y if l == L - 1 else np.maximum(y, 0.0)
        acts.append(bf16_round(a) if (bf16 and l < L - 1) else a)
    return acts, pres


def backward(acts, pres, weights, grad_out, bf16=False):
    """Gradients (dW list, db list, d input) for dloss/da_L = grad_out."""
    L = len(weights)
    dWs, dbs = [None] * L, [None] * L
    G = np.asarray(grad_out, np.float64)
    for l in range(L - 1, -1, -1):
        g = G if l == L - 1 else G * (pres[l] > 0)
        if bf16:
            g = bf16_round(g)
        a = acts[l]
        dW = np.zeros_like(weights[l])
        for t, (dy, dx) in enumerate(TAPS):
            dW[t] = np.einsum("nyxo,nyxi->oi", g, shift(a, dy, dx))
        dWs[l] = dW
        dbs[l] = g.sum(axis=(0, 1, 2))
        Wq = bf16_round(weights[l]) if bf16 else weights[l]
        Gn = np.zeros(a.shape)
        for t, (dy, dx) in enumerate(TAPS):
            Gn += shift(g, -dy, -dx) @ Wq[t]
        G = Gn
    return dWs, dbs, G


def init(channels, seed=0):
    """He-normal weights [9, co, ci] and zero biases for channels[0] -> ... -> channels[-1]."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for ci, co in zip(channels[:-1], channels[1:]):
        Ws.append(rng.standard_normal((9, co, ci)) * np.sqrt(2.0 / (9 * ci)))
        bs.append(np.zeros(co))
    return Ws, bs

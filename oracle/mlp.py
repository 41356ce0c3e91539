"""FP64 oracle of the per-node MLP used for the learned Newton initial guess.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network: x (F features) -> tanh(W1 x + b1) -> tanh(W2 . + b2) -> tanh(W3 . + b3)
-> W4 . + b4 (4 outputs), i.e. four affine layers, width 256, tanh between
them.  Loss: L = 1/(2 N) sum_n sum_o w_o (y_no - t_no)^2 with per-output
weights w_o.  Optimiser: Adam (Kingma & Ba, 2015) with bias correction:
m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def init_params(sizes, seed=0):
    """Weights W_l [out, in] ~ U(-a, a), a = sqrt(6 / (in + out)); biases zero."""
    rng = np.random.default_rng(seed)
    params = []
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / (fin + fout))
        params.append([rng.uniform(-a, a, size=(fout, fin)), np.zeros(fout)])
    return params


def forward(params, X):
    """Returns the output and the list of layer inputs / pre-activations."""
    acts = [X]
    zs = []
    h = X
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        h = np.tanh(z) if l < len(params) - 1 else z
        acts.append(h)
    return h, acts, zs


def loss_and_grads(params, X, T, w_out=None):
    n = X.shape[0]
    Y, acts, zs = forward(params, X)
    w_out = np.ones(Y.shape[1]) if w_out is None else np.asarray(w_out, dtype=np.float64)
    diff = Y - T
    loss = 0.5 * np.sum(w_out * diff * diff) / n
    grads = [None] * len(params)
    d = diff * w_out / n                              # dL/dz of the last layer
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = [d.T @ acts[l], d.sum(axis=0)]
        if l > 0:
            d = (d @ W) * (1.0 - np.tanh(zs[l - 1]) ** 2)
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; ``state`` = {"t": int, "m": [...], "v": [...]}."""
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        state["v"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    state["t"] += 1
    t = state["t"]
    for l in range(len(params)):
        for q in range(2):
            g = grads[l][q]
            m = state["m"][l][q]
            v = state["v"][l][q]
            m *= b1
            m += (1 - b1) * g
            v *= b2
            v += (1 - b2) * g * g
            params[l][q] -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return params

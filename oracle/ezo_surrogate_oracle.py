"""FP64 CPU oracle of the learned signed-distance surrogate (test
infrastructure only; not part of the paper, whose method does not learn).

Network: features phi(q) = [sin q_1 .. sin q_n, cos q_1 .. cos q_n, 0 .. 0]
(64 values), then z_l = h_{l-1} W_l^T + b_l and h_l = SiLU(z_l) = z_l
sigmoid(z_l) for three hidden layers of 256, and y = h_3 . w_4 + b_4. Loss:
mean squared error (1/N) sum_i (y_i - t_i)^2. The backward pass is the chain
rule written out layer by layer; SiLU'(z) = s (1 + z (1 - s)) with
s = sigmoid(z). Pinned by central finite differences in tests.

Parameter vector layout (matches the library): W1 [256 x 64] | b1 [256] |
W2 [256 x 256] | b2 | W3 [256 x 256] | b3 | w4 [256] | b4 [1].
"""
from __future__ import annotations

import numpy as np

F, H = 64, 256
SHAPES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("w4", (H,)), ("b4", (1,))]


def num_params() -> int:
    return int(sum(np.prod(s) for _, s in SHAPES))


def unpack(p):
    out, o = {}, 0
    for name, shp in SHAPES:
        c = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + c], dtype=np.float64).reshape(shp)
        o += c
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def features(q) -> np.ndarray:
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    N, n = q.shape
    X = np.zeros((N, F))
    X[:, :n] = np.sin(q)
    X[:, n:2 * n] = np.cos(q)
    return X


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, X):
    P = unpack(params) if not isinstance(params, dict) else params
    cache = {"X": X}
    h = X
    for l in (1, 2, 3):
        z = h @ P[f"W{l}"].T + P[f"b{l}"]
        cache[f"z{l}"] = z
        h = z * _sig(z)
        cache[f"h{l}"] = h
    y = h @ P["w4"] + P["b4"][0]
    return y, cache


def loss_and_grad(params, X, t):
    P = unpack(params)
    y, c = forward(P, X)
    N = X.shape[0]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / N
    g = {"w4": c["h3"].T @ dy, "b4": np.array([dy.sum()])}
    dh = np.outer(dy, P["w4"])
    for l in (3, 2, 1):
        z = c[f"z{l}"]
        s = _sig(z)
        dz = dh * s * (1.0 + z * (1.0 - s))
        hin = c[f"h{l - 1}"] if l > 1 else c["X"]
        g[f"W{l}"] = dz.T @ hin
        g[f"b{l}"] = dz.sum(axis=0)
        dh = dz @ P[f"W{l}"]
    return loss, pack(g)

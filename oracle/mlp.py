"""fp64 reference for the schedule MLP -- TEST INFRASTRUCTURE ONLY.

The schedule network is not in the paper: it replaces the paper's single
tunable tau (Sec. 2.1, "tau ... is a tunable parameter") and the
direction-optimisation switch (Sec. 2.2) by a per-round choice.  This file
is the plain fp64 statement of what the CUDA forward, backward and Adam
kernels compute, so that their results can be checked element by element.

Network (row-major weights, "out x in"):
    h1 = relu(W1 x + b1)          W1: 32 x 5,  b1: 32
    h2 = relu(W2 h1 + b2)         W2: 32 x 32, b2: 32
    y  = W3 h2 + b3               W3: A x 32,  b3: A      (A = 8 actions)
Packed parameter vector order: W1, b1, W2, b2, W3, b3 (1512 floats for A=8).

Loss over a batch of B rows with taken action a_i and target t_i:
    L = (1/B) * sum_i (y_i[a_i] - t_i)^2
Adam (Kingma & Ba, 2015) with bias correction:
    m <- b1 m + (1-b1) g ; v <- b2 v + (1-b2) g^2
    p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Features of a round (same definition the in-loop kernel uses):
    x0 = log2(1 + |F|) / 24          frontier size
    x1 = log2(1 + E_F) / 32          out-edges of the frontier
    x2 = log2(1 + E_F / |F|) / 8     mean degree of the frontier
    x3 = log2(1 + r) / 24            round index
    x4 = log2(1 + t_prev_us) / 16    previous round's time in microseconds
"""
from __future__ import annotations

import numpy as np

F_IN, HID, N_ACT = 5, 32, 8
SHAPES = [("W1", (HID, F_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (N_ACT, HID)), ("b3", (N_ACT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(p: np.ndarray, X: np.ndarray):
    """Returns (y, cache).  X: B x 5."""
    P = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"].T + P["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, act, target) -> float:
    y, _ = forward(p, X)
    B = X.shape[0]
    sel = y[np.arange(B), np.asarray(act, dtype=np.int64)]
    return float(np.mean((sel - np.asarray(target, dtype=np.float64)) ** 2))


def backward(p, X, act, target):
    """Returns (loss, grad) with grad packed like p."""
    P = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    act = np.asarray(act, dtype=np.int64)
    t = np.asarray(target, dtype=np.float64)
    sel = y[np.arange(B), act]
    L = float(np.mean((sel - t) ** 2))
    dy = np.zeros_like(y)
    dy[np.arange(B), act] = 2.0 * (sel - t) / B
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ P["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return L, pack(g)


def adam_step(p, g, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; returns new (p, m, v).  t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


ROUND_CAP = 2.0 ** 14  # the round-index feature saturates here (the training range)


def features(frontier, out_edges, rnd, prev_ns) -> np.ndarray:
    """Feature rows from raw per-round statistics (arrays of equal length)."""
    Fz = np.asarray(frontier, dtype=np.float64)
    E = np.asarray(out_edges, dtype=np.float64)
    r = np.minimum(np.asarray(rnd, dtype=np.float64), ROUND_CAP)
    tp = np.asarray(prev_ns, dtype=np.float64) / 1000.0
    mean = np.where(Fz > 0, E / np.maximum(Fz, 1.0), 0.0)
    return np.stack([np.log2(1 + Fz) / 24, np.log2(1 + E) / 32, np.log2(1 + mean) / 8,
                     np.log2(1 + r) / 24, np.log2(1 + tp) / 16], axis=1)

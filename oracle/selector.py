"""CPU oracle of the learned variant selector -- TEST INFRASTRUCTURE.

Like the rest of ``oracle/``, only ``tests/`` may import this module; the
selector's device code (the feature kernel and the perceptron's forward,
backward and Adam kernels) shares nothing with it.  Everything here is plain
float64 numpy written from the definitions:

* ``features(row_ptr, n)``  the 16 row-pointer statistics, each from its
  definition over the row lengths (no histogram shortcuts except the
  percentiles, which are defined on the power-of-two length bins).
* ``forward``/``loss_and_grad``  a perceptron F -> H1 -> H2 -> K with ReLU
  hidden layers and linear outputs, mean squared error over all B*K outputs
  (NaN targets contribute nothing); the gradient by the chain rule, layer by
  layer (Rumelhart, Hinton & Williams 1986).
* ``adam_step``  one Adam update (Kingma & Ba 2015, Algorithm 1) with L2
  weight decay added to the gradient.

Parameters are one flat array in the library's layout:
W1[H1][F], b1[H1], W2[H2][H1], b2[H2], W3[K][H2], b3[K].
"""
from __future__ import annotations

import numpy as np


def _bin(lengths: np.ndarray) -> np.ndarray:
    """Power-of-two bin of each length: 0 for empty rows, b >= 1 for lengths
    in [2^(b-1), 2^b), capped at 31."""
    out = np.zeros(lengths.shape, dtype=np.int64)
    nz = lengths > 0
    out[nz] = np.minimum(np.floor(np.log2(lengths[nz])).astype(np.int64) + 1, 31)
    return out


def features(row_ptr, n: int) -> np.ndarray:
    rp = np.asarray(row_ptr, dtype=np.int64)
    m = len(rp) - 1
    nnz = int(rp[-1]) if m >= 0 else 0
    L = np.diff(rp).astype(np.float64)
    md = float(m) if m > 0 else 1.0
    mean = nnz / md
    var = float(np.sum(L * L)) / md - mean * mean
    sd = np.sqrt(var) if var > 0 else 0.0
    nz = float(nnz) if nnz > 0 else 1.0
    bins = np.bincount(_bin(L.astype(np.int64)), minlength=32) if m > 0 else np.zeros(32)
    cum = np.cumsum(bins)
    pct = []
    for q in (0.5, 0.9, 0.99):
        hit = np.nonzero(cum >= q * md)[0]
        pct.append(float(hit[0]) if hit.size else 0.0)
    prev = L[:-1]
    cur = L[1:]
    jump = np.sum((cur > 2 * prev + 1) | (prev > 2 * cur + 1)) if m > 1 else 0
    erun = np.sum((cur == 0) & (prev == 0)) if m > 1 else 0
    f = np.array([
        np.log2(md + 1.0) / 24.0,
        np.log2(nnz + 1.0) / 32.0,
        np.log2(mean + 1.0) / 8.0,
        sd / (mean + 1.0),
        np.log2((L.max() if m > 0 else 0.0) + 1.0) / 24.0,
        np.sum(L == 0) / md,
        np.sum(L <= 4) / md,
        np.sum(L >= 2.0 * mean) / md,
        np.sum(L[L > 1024]) / nz,
        pct[0] / 16.0,
        pct[1] / 16.0,
        pct[2] / 16.0,
        jump / md,
        np.log2(480.0 / (mean + 1e-9) + 1.0) / 16.0,
        erun / md,
        np.sum(L[L >= 32.0 * mean]) / nz,
    ], dtype=np.float64)
    return f


def sizes(F: int, H1: int, H2: int, K: int) -> int:
    return H1 * F + H1 + H2 * H1 + H2 + K * H2 + K


def unpack(p: np.ndarray, F: int, H1: int, H2: int, K: int):
    o = 0

    def take(n, shape):
        nonlocal o
        a = p[o:o + n].reshape(shape)
        o += n
        return a
    W1 = take(H1 * F, (H1, F))
    b1 = take(H1, (H1,))
    W2 = take(H2 * H1, (H2, H1))
    b2 = take(H2, (H2,))
    W3 = take(K * H2, (K, H2))
    b3 = take(K, (K,))
    return W1, b1, W2, b2, W3, b3


def forward(p, X, F, H1, H2, K):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(p, np.float64), F, H1, H2, K)
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    out = a2 @ W3.T + b3
    return out, (X, z1, a1, z2, a2)


def loss_and_grad(p, X, T, F, H1, H2, K):
    p = np.asarray(p, np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H1, H2, K)
    out, (X, z1, a1, z2, a2) = forward(p, X, F, H1, H2, K)
    T = np.asarray(T, np.float64)
    mask = ~np.isnan(T)
    d = np.where(mask, out - np.where(mask, T, 0.0), 0.0)
    count = out.size
    loss = float(np.sum(d * d) / count)
    g3 = 2.0 * d / count                      # dL/dout
    dW3 = g3.T @ a2
    db3 = g3.sum(axis=0)
    g2 = (g3 @ W3) * (z2 > 0)                 # through ReLU
    dW2 = g2.T @ a1
    db2 = g2.sum(axis=0)
    g1 = (g2 @ W2) * (z1 > 0)
    dW1 = g1.T @ X
    db1 = g1.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad


def adam_step(p, g, m1, m2, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0, t=1):
    p = np.asarray(p, np.float64).copy()
    g = np.asarray(g, np.float64) + wd * p
    m1 = b1 * np.asarray(m1, np.float64) + (1 - b1) * g
    m2 = b2 * np.asarray(m2, np.float64) + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    p -= lr * mh / (np.sqrt(vh) + eps)
    return p, m1, m2

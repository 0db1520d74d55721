"""Pins of the selector oracle (oracle/selector.py) to facts outside itself:
a hand-worked feature example, central finite differences of the loss,
closed forms of the perceptron with zero weights, and the first Adam step
(which moves every parameter by lr * g / (|g| + eps))."""
import numpy as np

from oracle import selector as O


def test_features_hand_example():
    # row lengths 0, 3, 0, 0, 5, 1: nnz 9, mean 1.5
    rp = np.array([0, 0, 3, 3, 3, 8, 9])
    f = O.features(rp, n=7)
    assert np.isclose(f[0], np.log2(7.0) / 24)
    assert np.isclose(f[1], np.log2(10.0) / 32)
    assert np.isclose(f[2], np.log2(2.5) / 8)
    var = (0 + 9 + 0 + 0 + 25 + 1) / 6 - 1.5 ** 2
    assert np.isclose(f[3], np.sqrt(var) / 2.5)
    assert np.isclose(f[4], np.log2(6.0) / 24)
    assert np.isclose(f[5], 3 / 6)                 # empty rows
    assert np.isclose(f[6], 5 / 6)                 # rows <= 4
    assert np.isclose(f[7], 2 / 6)                 # rows >= 3
    assert f[8] == 0.0                             # nothing longer than 1024
    # length bins 0,2,0,0,3,1: counts per bin 3,1,1,1 -> cumulative 3,4,5,6; the
    # median is bin 0, the 90th and 99th percentiles bin 3
    assert np.isclose(f[9], 0 / 16) and np.isclose(f[10], 3 / 16) and np.isclose(f[11], 3 / 16)
    assert np.isclose(f[12], 4 / 6)                # neighbours differing by more than 2x
    assert np.isclose(f[13], np.log2(480 / 1.5 + 1) / 16)
    assert np.isclose(f[14], 1 / 6)                # an empty row after an empty row
    assert f[15] == 0.0                            # no row reaches 32 x 1.5 = 48 entries


def test_feature_long_rows():
    rp = np.concatenate([[0], np.cumsum([1] * 99 + [5000])])
    f = O.features(rp, n=6000)
    assert np.isclose(f[8], 5000 / 5099)           # entries in rows > 1024
    assert np.isclose(f[15], 5000 / 5099)          # a row >= 32x the mean (mean 50.99)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    F, H1, H2, K, B = 5, 7, 6, 4, 9
    p = rng.normal(0, 0.5, O.sizes(F, H1, H2, K))
    X = rng.normal(0, 1, (B, F))
    T = rng.normal(0, 1, (B, K))
    T[1, 2] = np.nan
    T[4, 0] = np.nan
    _, g = O.loss_and_grad(p, X, T, F, H1, H2, K)
    h = 1e-6
    num = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (O.loss_and_grad(p + e, X, T, F, H1, H2, K)[0]
                  - O.loss_and_grad(p - e, X, T, F, H1, H2, K)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_zero_weights_closed_form():
    F, H1, H2, K, B = 3, 4, 4, 2, 5
    p = np.zeros(O.sizes(F, H1, H2, K))
    p[-K:] = [0.5, -1.5]                           # b3
    X = np.random.default_rng(1).normal(size=(B, F))
    out, _ = O.forward(p, X, F, H1, H2, K)
    assert np.all(out == np.array([0.5, -1.5]))
    T = np.zeros((B, K))
    loss, g = O.loss_and_grad(p, X, T, F, H1, H2, K)
    assert np.isclose(loss, (0.25 + 2.25) / 2)
    # only b3 has a gradient: 2 * mean over the batch of (out - T) / K
    assert np.allclose(g[-K:], 2 * np.array([0.5, -1.5]) * B / (B * K))
    assert np.all(g[:-K] == 0)


def test_first_adam_step():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.1, -3.0, 0.0])
    q, m1, m2 = O.adam_step(p, g, np.zeros(3), np.zeros(3), lr=0.01, t=1)
    assert np.allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)

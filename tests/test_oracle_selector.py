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


def test_adam_hand_worked_three_steps_with_decay():
    """Kingma & Ba, Algorithm 1, with the L2 decay wd*p added to the gradient,
    worked by hand for beta1 = 1/2, beta2 = 3/4, lr = 1, eps = 0, wd = 1/2 on
    two parameters whose raw gradients are constant (1 and -3).

    Parameter A, p = 2:
      t=1: g = 1 + 2/2 = 2; m = 1; v = 1; mhat = 1/(1-1/2) = 2;
           vhat = 1/(1-3/4) = 4; p = 2 - 2/2 = 1
      t=2: g = 1 + 1/2 = 3/2; m = 1/2 + 3/4 = 5/4; v = 3/4 + 9/16 = 21/16;
           mhat = (5/4)/(1-1/4) = 5/3; vhat = (21/16)/(1-9/16) = 3;
           p = 1 - 5/(3 sqrt 3)
      t=3: bias corrections 1 - 1/8 = 7/8 and 1 - 27/64 = 37/64
    Parameter B, p = -1:
      t=1: g = -3 - 1/2 = -7/2; m = -7/4; v = 49/16; mhat = -7/2; vhat = 49/4;
           p = -1 + 1 = 0
      t=2: g = -3; m = -7/8 - 3/2 = -19/8; v = 147/64 + 9/4 = 291/64;
           mhat = -19/6; vhat = 291/28; p = (19/6) / sqrt(291/28)
    """
    import math
    p = np.array([2.0, -1.0])
    graw = np.array([1.0, -3.0])
    m1 = np.zeros(2)
    m2 = np.zeros(2)
    kw = dict(lr=1.0, b1=0.5, b2=0.75, eps=0.0, wd=0.5)
    p, m1, m2 = O.adam_step(p, graw, m1, m2, t=1, **kw)
    assert np.array_equal(p, [1.0, 0.0])
    assert np.array_equal(m1, [1.0, -1.75]) and np.array_equal(m2, [1.0, 49 / 16])
    p, m1, m2 = O.adam_step(p, graw, m1, m2, t=2, **kw)
    pA2 = 1 - 5 / (3 * math.sqrt(3))
    pB2 = (19 / 6) / math.sqrt(291 / 28)
    assert np.allclose(p, [pA2, pB2], rtol=0, atol=1e-15)
    assert np.array_equal(m1, [1.25, -19 / 8]) and np.allclose(m2, [21 / 16, 291 / 64], rtol=1e-15)
    p, m1, m2 = O.adam_step(p, graw, m1, m2, t=3, **kw)
    # t = 3 by hand from the t = 2 moments
    gA, gB = 1 + pA2 / 2, -3 + pB2 / 2
    mA, mB = 5 / 8 + gA / 2, -19 / 16 + gB / 2
    vA, vB = 63 / 64 + gA * gA / 4, 873 / 256 + gB * gB / 4
    want = [pA2 - (mA / (7 / 8)) / math.sqrt(vA / (37 / 64)),
            pB2 - (mB / (7 / 8)) / math.sqrt(vB / (37 / 64))]
    assert np.allclose(p, want, rtol=0, atol=1e-14)
    assert abs(p[0] - (-0.8461244626965501)) < 1e-12


def test_adam_bias_correction_at_every_step():
    """With a constant gradient g and no decay, m_t = (1 - b1^t) g and
    v_t = (1 - b2^t) g^2, so the corrected moments are g and g^2 exactly and
    every step -- not only the first -- moves by lr * g / (|g| + eps)."""
    g = np.array([0.25, -4.0, 1e-3])
    p = np.array([1.0, 2.0, -3.0])
    m1 = np.zeros(3)
    m2 = np.zeros(3)
    for t in range(1, 11):
        q, m1, m2 = O.adam_step(p, g, m1, m2, lr=0.01, t=t)
        assert np.allclose(m1, (1 - 0.9 ** t) * g, rtol=1e-12)
        assert np.allclose(m2, (1 - 0.999 ** t) * g * g, rtol=1e-12)
        assert np.allclose(q - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        p = q


def test_adam_decay_is_added_to_the_gradient():
    """L2 decay enters the moments (coupled, as in the paper's Algorithm 1 with
    the penalty in the objective): with a zero raw gradient the first step is
    an ordinary Adam step on wd*p and moves p by lr*sign(p) when eps = 0.  A
    decoupled decay (p -= lr*wd*p beside the Adam step) would move it by
    lr*wd*|p| instead."""
    p = np.array([3.0, -0.5])
    q, m1, m2 = O.adam_step(p, np.zeros(2), np.zeros(2), np.zeros(2), lr=0.1, eps=0.0, wd=0.2,
                            t=1)
    assert np.allclose(q, [2.9, -0.4], rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * 0.2 * p) and np.allclose(m2, 0.001 * (0.2 * p) ** 2)

"""Pins of the oracle's training-step pieces: the L2 loss gradient against central
differences, and Adam's first step, which from zero moments moves every parameter
by lr * g / (|g| + eps) (bias correction cancels the moment decay)."""
import numpy as np

from oracle import oracle as O


def test_l2_loss_gradient_is_its_derivative():
    rng = np.random.default_rng(0)
    x = rng.normal(size=50)
    t = rng.normal(size=50)
    L, d = O.l2_loss(x, t, 0.25)
    assert abs(L - 0.25 * ((x - t) ** 2).sum()) < 1e-12
    h = 1e-6
    for i in range(0, 50, 7):
        xp = x.copy(); xp[i] += h
        xm = x.copy(); xm[i] -= h
        fd = (O.l2_loss(xp, t, 0.25)[0] - O.l2_loss(xm, t, 0.25)[0]) / (2 * h)
        assert abs(fd - d[i]) < 1e-6


def test_adam_first_step_closed_form_and_zero_gradient():
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=100)
    g = rng.normal(size=100)
    g[:5] = 0.0
    p, m, v = p0.copy(), np.zeros(100), np.zeros(100)
    O.adam_step(p, g, m, v, lr=0.01, b1=0.9, b2=0.99, eps=1e-8, step=1)
    np.testing.assert_allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
    assert np.all(p[:5] == p0[:5])
    # a constant gradient keeps the bias-corrected moments at g and g^2, so every
    # step stays lr * g / (|g| + eps)
    for s in range(2, 6):
        before = p.copy()
        O.adam_step(p, g, m, v, lr=0.01, b1=0.9, b2=0.99, eps=1e-8, step=s)
        np.testing.assert_allclose(before - p, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)

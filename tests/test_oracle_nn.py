"""Pins of the FP64 neural-operator oracle (conv layers, pooling, U-Net
gradient, Adam) to library routines, adjoint identities, finite
differences and closed forms."""
import math

import numpy as np
import pytest

import lbib_inputs as li


@pytest.fixture(scope="module")
def nn(orc):
    import oracle.nn as nn
    return nn


def test_conv_matches_scipy_correlate(orc):
    from scipy.signal import correlate2d
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    w = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    y = orc.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, i], w[:, :, i, o], mode="same")
                             for i in range(3))
            assert np.allclose(y[n, :, :, o], ref, atol=1e-13)


def test_conv_identity_tap(orc):
    """A weight that is 1 at the centre tap from channel i to i is the
    identity map."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 5, 6, 3))
    w = np.zeros((3, 3, 3, 3))
    for i in range(3):
        w[1, 1, i, i] = 1.0
    assert np.array_equal(orc.conv3x3(x, w), x)


def test_dgrad_is_adjoint_and_wgrad_matches_finite_differences(orc):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 6, 5, 3))
    w = rng.normal(size=(3, 3, 3, 4))
    g = rng.normal(size=(2, 6, 5, 4))
    # <conv(x), g> = <x, dgrad(g)>
    assert np.sum(orc.conv3x3(x, w) * g) == pytest.approx(np.sum(x * orc.conv3x3_dgrad(g, w)),
                                                          rel=1e-12)
    dw, db = orc.conv3x3_wgrad(x, g)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 2, 3), (2, 1, 0, 1), (1, 1, 1, 2)]:
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        fd = (np.sum(orc.conv3x3(x, wp) * g) - np.sum(orc.conv3x3(x, wm) * g)) / (2 * h)
        assert dw[idx] == pytest.approx(fd, rel=1e-7, abs=1e-9)
    assert np.allclose(db, g.sum(axis=(0, 1, 2)))


def test_pool_upsample_adjoint(nn):
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 8, 6, 3))
    g = rng.normal(size=(2, 4, 3, 3))
    assert np.sum(nn.avgpool2(x) * g) == pytest.approx(np.sum(x * nn.avgpool2_bwd(g)))
    u = rng.normal(size=(2, 4, 3, 3))
    G = rng.normal(size=(2, 8, 6, 3))
    assert np.sum(nn.upsample2(u) * G) == pytest.approx(np.sum(u * nn.upsample2_bwd(G)))


def test_unet_gradient_matches_finite_differences(nn):
    ch = (4, 6, 8)
    shapes = nn.nop_shapes(ch)
    p = li.nop_init_params(3, shapes)
    rng = np.random.default_rng(4)
    p = p + 0.05 * rng.normal(size=p.size)     # move biases off zero
    x = rng.normal(size=(2, 8, 8, 4))
    t = rng.normal(size=(2, 8, 8, 1))
    y, c = nn.forward(p, x, ch)
    _, dy = nn.loss(y, t)
    g = nn.backward(dy, c, ch)
    h = 1e-6
    for i in rng.choice(p.size, 40, replace=False):
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        Lp, _ = nn.loss(nn.forward(pp, x, ch)[0], t)
        Lm, _ = nn.loss(nn.forward(pm, x, ch)[0], t)
        assert g[i] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_full_size_shapes(nn):
    """Six levels, about two million parameters."""
    assert nn.nop_num_params() == 2083809
    assert len(nn.nop_shapes()) == 23


def test_adam_first_step_is_signed_learning_rate(nn):
    """With bias correction the first Adam step is lr * g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    q, m, v = nn.adam(p, g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)

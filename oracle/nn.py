"""FP64 reference of the neural operator that warm-starts the steady
morphogen solve -- TEST INFRASTRUCTURE (see oracle/__init__.py).

The paper has no network; this is the learned part the measured method
adds on top of the D2Q5 relaxation.  Its definition:

  input   4 channels per node: cell mask (1 inside a cell), source mask
          (1 in a source cell), (D - 0.125) / 0.075, log10(decay) + 3
  target  phi * decay / src_rate (dimensionless, the uniform steady value
          of a source region is 1); phi_pred = y * src_rate / decay
  U-Net   six levels with channels C = 32, 48, 64, 96, 128, 192; every
          level of the encoder is conv3x3-ReLU-conv3x3-ReLU, levels are
          joined by 2x2 average pooling; the decoder upsamples by 2
          (nearest), concatenates [encoder skip, upsampled] on channels and
          applies conv3x3-ReLU-conv3x3-ReLU; a final conv3x3 gives 1 channel.
          All convolutions have zero padding and a bias.
  loss    mean squared error over all nodes of the batch
  Adam    beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected

Parameters are one flat vector, layer by layer in the order of
nop_shapes(): weights (3, 3, Ci, Co) then bias (Co,).
"""
from __future__ import annotations

import numpy as np

from . import conv3x3, conv3x3_dgrad, conv3x3_wgrad

CHANNELS = (32, 48, 64, 96, 128, 192)
IN_CHANNELS = 4


def nop_shapes(channels=CHANNELS, cin=IN_CHANNELS):
    """[(name, Ci, Co)] of every conv layer in parameter order."""
    L = len(channels)
    out = []
    prev = cin
    for l, c in enumerate(channels):
        out.append((f"enc{l}a", prev, c))
        out.append((f"enc{l}b", c, c))
        prev = c
    for l in range(L - 2, -1, -1):
        out.append((f"dec{l}a", channels[l] + channels[l + 1], channels[l]))
        out.append((f"dec{l}b", channels[l], channels[l]))
    out.append(("out", channels[0], 1))
    return out


def nop_num_params(channels=CHANNELS, cin=IN_CHANNELS):
    return sum(9 * ci * co + co for _, ci, co in nop_shapes(channels, cin))


def unpack(params, channels=CHANNELS, cin=IN_CHANNELS):
    layers = {}
    o = 0
    for name, ci, co in nop_shapes(channels, cin):
        w = params[o:o + 9 * ci * co].reshape(3, 3, ci, co)
        o += 9 * ci * co
        b = params[o:o + co]
        o += co
        layers[name] = (w, b)
    assert o == params.size
    return layers


def features(mask, src, D, decay):
    """(N, H, W, 4) network input from per-tissue masks and parameters."""
    N, H, W = mask.shape
    x = np.zeros((N, H, W, 4))
    x[..., 0] = mask
    x[..., 1] = src
    x[..., 2] = ((np.asarray(D) - 0.125) / 0.075)[:, None, None]
    x[..., 3] = (np.log10(np.asarray(decay)) + 3.0)[:, None, None]
    return x


def avgpool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_bwd(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_bwd(g):
    N, H, W, C = g.shape
    return g.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(params, x, channels=CHANNELS):
    """Returns (y (N,H,W,1), cache)."""
    P = unpack(params, channels, x.shape[3])
    L = len(channels)
    cache = {"x": x, "P": P}
    h = x
    skips = []
    for l in range(L):
        if l > 0:
            h = avgpool2(h)
        a_in = h
        z1 = conv3x3(a_in, *P[f"enc{l}a"])
        r1 = np.maximum(z1, 0.0)
        z2 = conv3x3(r1, *P[f"enc{l}b"])
        h = np.maximum(z2, 0.0)
        cache[f"enc{l}"] = (a_in, r1, h)
        skips.append(h)
    for l in range(L - 2, -1, -1):
        u = upsample2(h)
        cat = np.concatenate([skips[l], u], axis=3)
        z1 = conv3x3(cat, *P[f"dec{l}a"])
        r1 = np.maximum(z1, 0.0)
        z2 = conv3x3(r1, *P[f"dec{l}b"])
        h = np.maximum(z2, 0.0)
        cache[f"dec{l}"] = (cat, r1, h)
    y = conv3x3(h, *P["out"])
    cache["dec_out_in"] = h
    return y, cache


def loss(y, target):
    """MSE and its gradient with respect to y."""
    d = y - target
    n = d.size
    return float(np.sum(d * d) / n), 2.0 * d / n


def backward(dy, cache, channels=CHANNELS):
    """Gradient of the loss with respect to the flat parameter vector."""
    P = cache["P"]
    L = len(channels)
    G = {}
    h = cache["dec_out_in"]
    G["out"] = conv3x3_wgrad(h, dy)
    g = conv3x3_dgrad(dy, P["out"][0])
    skip_grads = {}
    for l in range(0, L - 1):
        cat, r1, out = cache[f"dec{l}"]
        g = g * (out > 0)
        G[f"dec{l}b"] = conv3x3_wgrad(r1, g)
        g = conv3x3_dgrad(g, P[f"dec{l}b"][0]) * (r1 > 0)
        G[f"dec{l}a"] = conv3x3_wgrad(cat, g)
        gcat = conv3x3_dgrad(g, P[f"dec{l}a"][0])
        cs = channels[l]
        skip_grads[l] = gcat[..., :cs]
        g = upsample2_bwd(gcat[..., cs:])
    # g is now the gradient of the deepest encoder output
    for l in range(L - 1, -1, -1):
        a_in, r1, out = cache[f"enc{l}"]
        if l < L - 1:
            g = g + skip_grads[l]
        g = g * (out > 0)
        G[f"enc{l}b"] = conv3x3_wgrad(r1, g)
        g = conv3x3_dgrad(g, P[f"enc{l}b"][0]) * (r1 > 0)
        G[f"enc{l}a"] = conv3x3_wgrad(a_in, g)
        if l > 0:
            g = avgpool2_bwd(conv3x3_dgrad(g, P[f"enc{l}a"][0]))
    flat = []
    for name, ci, co in nop_shapes(channels, cache["x"].shape[3]):
        dw, db = G[name]
        flat.append(dw.ravel())
        flat.append(db)
    return np.concatenate(flat)


def adam(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns updated (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v

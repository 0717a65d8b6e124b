"""Oracle of the learned preconditioner step: a small convolutional U-Net (FP64).

Test infrastructure (see the package header).  Plain numpy, written for a
reader to check by eye; the GPU network (BF16 storage, FP32 accumulation) is
compared against it layer by layer and gradient by gradient.

The paper has no network: its preconditioners are Algorithms 1-3.  The
learned step is an addition placed where the paper's outer iteration allows
one -- Sec. 6 uses flexible GMRES, whose preconditioner may change from step
to step -- so a network can serve as one more right-preconditioner stage.

Network (fixed architecture, parameters in a dict):
  input  x: (3, H, W) = (Re r / s, Im r / s, m), s = RMS of the residual r;
  encoder level l = 0..L-1 (channels c_l = c0 * 2^l): two 3x3 convolutions
         with ReLU; between levels a 2x2 average pool;
  decoder level l = L-2..0: nearest-neighbour 2x upsampling of the level
         below, a 3x3 convolution to c_l with ReLU, concatenation with the
         encoder's level-l output (skip), two 3x3 convolutions with ReLU;
  head:  3x3 convolution to 2 channels (Re, Im of the correction / s).
All convolutions are cross-correlations with zero padding 1 and a bias:
  y[o, i, j] = b[o] + sum_{c, a, b'} w[o, c, a, b'] x[c, i + a - 1, j + b' - 1].
Loss: 0.5 * mean((y - t)^2) over every output value.
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------------ layers
def conv3x3(x, w, b):
    """x (C, H, W), w (O, C, 3, 3), b (O,) -> (O, H, W); zero padding 1."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2), dtype=x.dtype)
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], H, W), dtype=np.result_type(x, w))
    for a in range(3):
        for bb in range(3):
            patch = xp[:, a:a + H, bb:bb + W]                 # (C, H, W)
            y += np.einsum("oc,chw->ohw", w[:, :, a, bb], patch)
    return y + b[:, None, None]


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 with respect to x, w, b, given dL/dy."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2), dtype=x.dtype)
    xp[:, 1:-1, 1:-1] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for a in range(3):
        for bb in range(3):
            patch = xp[:, a:a + H, bb:bb + W]
            dw[:, :, a, bb] = np.einsum("ohw,chw->oc", dy, patch)
            dxp[:, a:a + H, bb:bb + W] += np.einsum("oc,ohw->chw", w[:, :, a, bb], dy)
    return dxp[:, 1:-1, 1:-1], dw, dy.sum(axis=(1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    C, H, W = dy.shape
    return dy.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


# ------------------------------------------------------------------ network
def layer_shapes(levels=4, c0=32, cin=3, cout=2):
    """Ordered (name, out_channels, in_channels) of every convolution."""
    ch = [c0 * 2 ** l for l in range(levels)]
    out = []
    prev = cin
    for l in range(levels):
        out.append(("enc%d_a" % l, ch[l], prev))
        out.append(("enc%d_b" % l, ch[l], ch[l]))
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        out.append(("dec%d_up" % l, ch[l], ch[l + 1]))
        out.append(("dec%d_a" % l, ch[l], 2 * ch[l]))
        out.append(("dec%d_b" % l, ch[l], ch[l]))
    out.append(("head", cout, ch[0]))
    return out


def init_params(levels=4, c0=32, cin=3, cout=2, seed=0):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, o, c in layer_shapes(levels, c0, cin, cout):
        std = np.sqrt(2.0 / (9 * c))
        if name == "head":
            std *= 0.1
        p[name + ".w"] = rng.standard_normal((o, c, 3, 3)) * std
        p[name + ".b"] = np.zeros(o)
    return p


def forward(p, x, levels=4):
    """Returns the output (2, H, W) and the cache the backward pass needs."""
    cache = {}
    skips = []
    h = x
    for l in range(levels):
        if l > 0:
            h = avgpool2(h)
        for s in ("a", "b"):
            name = "enc%d_%s" % (l, s)
            cache[name + ".in"] = h
            h = relu(conv3x3(h, p[name + ".w"], p[name + ".b"]))
            cache[name + ".out"] = h
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        up = upsample2(h)
        name = "dec%d_up" % l
        cache[name + ".in"] = up
        h = relu(conv3x3(up, p[name + ".w"], p[name + ".b"]))
        cache[name + ".out"] = h
        h = np.concatenate([h, skips[l]], axis=0)
        for s in ("a", "b"):
            name = "dec%d_%s" % (l, s)
            cache[name + ".in"] = h
            h = relu(conv3x3(h, p[name + ".w"], p[name + ".b"]))
            cache[name + ".out"] = h
    cache["head.in"] = h
    y = conv3x3(h, p["head.w"], p["head.b"])
    return y, cache


def backward(p, cache, dy, levels=4):
    """Gradients of every parameter given dL/dy (same keys as p).

    The decoder runs from level L-2 up to 0 in the forward pass, so its
    gradients flow from level 0 down to L-2, then through the encoder from
    level L-1 up to 0, adding each level's skip gradient."""
    g = {}
    dh, g["head.w"], g["head.b"] = conv3x3_backward(cache["head.in"], p["head.w"], dy)
    dskip = [None] * levels
    for l in range(0, levels - 1):              # decoder, reverse of its forward order
        for s in ("b", "a"):
            name = "dec%d_%s" % (l, s)
            dpre = dh * (cache[name + ".out"] > 0)
            dh, g[name + ".w"], g[name + ".b"] = conv3x3_backward(cache[name + ".in"], p[name + ".w"], dpre)
        c = p["dec%d_up.w" % l].shape[0]
        dskip[l] = dh[c:]
        dh = dh[:c]
        name = "dec%d_up" % l
        dpre = dh * (cache[name + ".out"] > 0)
        dup, g[name + ".w"], g[name + ".b"] = conv3x3_backward(cache[name + ".in"], p[name + ".w"], dpre)
        dh = upsample2_backward(dup)            # gradient of level l+1's last output
    for l in range(levels - 1, -1, -1):         # encoder, bottom up
        if dskip[l] is not None:
            dh = dh + dskip[l]
        for s in ("b", "a"):
            name = "enc%d_%s" % (l, s)
            dpre = dh * (cache[name + ".out"] > 0)
            dh, g[name + ".w"], g[name + ".b"] = conv3x3_backward(cache[name + ".in"], p[name + ".w"], dpre)
        if l > 0:
            dh = avgpool2_backward(dh)
    return g


def loss_and_grad(p, x, t, levels=4):
    """0.5 * mean((y - t)^2) and its parameter gradients."""
    y, cache = forward(p, x, levels)
    d = y - t
    loss = 0.5 * float(np.mean(d * d))
    g = backward(p, cache, d / d.size, levels)
    return loss, g, y


def make_input(r, m):
    """Network input and scale: (Re r / s, Im r / s, m), s = RMS(r)."""
    s = float(np.sqrt(np.mean(np.abs(r) ** 2)))
    s = s if s > 0 else 1.0
    return np.stack([r.real / s, r.imag / s, m]), s


def apply(p, r, m, levels=4):
    """The learned step z = s * N((r / s, m)) as a complex field."""
    x, s = make_input(r, m)
    y, _ = forward(p, x, levels)
    return s * (y[0] + 1j * y[1])

"""Pins of the U-Net oracle (CPU): brute-force convolution, adjoint identities,
finite-difference gradients of the whole network, and the scale equivariance of
the learned step."""
import numpy as np
import pytest

from oracle import unet

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_is_the_zero_padded_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 7, 5))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv3x3(x, w, b)
    # brute force, one output at a time
    for o, i, j in [(0, 0, 0), (3, 6, 4), (2, 3, 2), (1, 0, 4)]:
        acc = b[o]
        for c in range(3):
            for a in range(3):
                for bb in range(3):
                    ii, jj = i + a - 1, j + bb - 1
                    if 0 <= ii < 7 and 0 <= jj < 5:
                        acc += w[o, c, a, bb] * x[c, ii, jj]
        assert abs(y[o, i, j] - acc) < 1e-12
    # and the library routine
    for o in range(4):
        ref = sum(scipy_signal.correlate2d(x[c], w[o, c], mode="same") for c in range(3)) + b[o]
        assert np.allclose(y[o], ref, atol=1e-12)


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 6))
    y = rng.standard_normal((2, 4, 3))
    assert abs(np.sum(unet.avgpool2(x) * y) - np.sum(x * unet.avgpool2_backward(y))) < 1e-12
    z = rng.standard_normal((2, 8, 6))
    assert abs(np.sum(unet.upsample2(y) * z) - np.sum(y * unet.upsample2_backward(z))) < 1e-12


def test_conv_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 5, 4))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((3, 5, 4))
    dx, dw, db = unet.conv3x3_backward(x, w, dy)
    f = lambda xx, ww, bb: float(np.sum(unet.conv3x3(xx, ww, bb) * dy))
    eps = 1e-6
    for idx in [(0, 0, 0), (1, 4, 3), (1, 2, 1)]:
        e = np.zeros_like(x); e[idx] = eps
        assert abs((f(x + e, w, b) - f(x - e, w, b)) / (2 * eps) - dx[idx]) < 1e-7
    for idx in [(0, 0, 0, 0), (2, 1, 2, 1), (1, 0, 1, 2)]:
        e = np.zeros_like(w); e[idx] = eps
        assert abs((f(x, w + e, b) - f(x, w - e, b)) / (2 * eps) - dw[idx]) < 1e-7
    for o in range(3):
        e = np.zeros_like(b); e[o] = eps
        assert abs((f(x, w, b + e) - f(x, w, b - e)) / (2 * eps) - db[o]) < 1e-7


def test_network_gradient_matches_finite_differences():
    levels, c0 = 3, 2
    p = unet.init_params(levels=levels, c0=c0, seed=3)
    rng = np.random.default_rng(4)
    # biases nonzero so that every ReLU sees both signs
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((3, 8, 8))
    t = rng.standard_normal((2, 8, 8))
    loss, g, _ = unet.loss_and_grad(p, x, t, levels)
    eps = 1e-6
    checked = 0
    for name in ["enc0_a.w", "enc1_b.w", "enc2_a.w", "dec1_up.w", "dec1_a.w", "dec0_b.w", "head.w",
                 "enc0_b.b", "dec0_up.b", "head.b"]:
        arr = p[name]
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + eps
            lp, _, _ = unet.loss_and_grad(p, x, t, levels)
            arr[idx] = old - eps
            lm, _, _ = unet.loss_and_grad(p, x, t, levels)
            arr[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name][idx]) < 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])
            checked += 1
    assert checked == 30
    assert set(g) == set(p)


def test_learned_step_is_scale_equivariant_and_shapes_follow_levels():
    p = unet.init_params(levels=3, c0=2, seed=5)
    rng = np.random.default_rng(6)
    r = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    m = rng.standard_normal((16, 16))
    z1 = unet.apply(p, r, m, levels=3)
    z2 = unet.apply(p, 3.0 * r, m, levels=3)
    assert np.allclose(z2, 3.0 * z1, rtol=1e-12, atol=1e-14)
    shapes = unet.layer_shapes(levels=4, c0=32)
    assert len(shapes) == 4 * 2 + 3 * 3 + 1
    assert shapes[0] == ("enc0_a", 32, 3) and shapes[-1] == ("head", 2, 32)
    assert ("dec2_a", 128, 256) in shapes and ("enc3_b", 256, 256) in shapes

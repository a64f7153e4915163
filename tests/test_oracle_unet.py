"""Pins for the U-Net oracle: brute-force convolution, adjoint transfers, finite differences."""
import numpy as np
import pytest

from oracle import unet


def test_conv3d_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    n, ci, co = 3, 2, 3
    x = rng.standard_normal((n, n, n, ci))
    w = rng.standard_normal((27, ci, co))
    b = rng.standard_normal(co)
    y = unet.conv3d(x, w, b)
    ref = np.zeros((n, n, n, co))
    for z in range(n):
        for yy in range(n):
            for xx in range(n):
                acc = b.copy()
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                            zz, yy2, xx2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < n and 0 <= yy2 < n and 0 <= xx2 < n:
                                acc = acc + x[zz, yy2, xx2] @ w[t]
                ref[z, yy, xx] = acc
    np.testing.assert_allclose(y, ref, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 4, 4, 3))
    p = rng.standard_normal((2, 2, 2, 3))
    assert abs(np.sum(unet.pool(x) * p) - np.sum(x * unet.pool_backward(p))) < 1e-12
    assert abs(np.sum(unet.upsample(p) * x) - np.sum(p * unet.upsample_backward(x))) < 1e-12
    # the pool of a constant is the constant; upsample then pool is the identity
    np.testing.assert_allclose(unet.pool(unet.upsample(p)), p)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 3, 5, 2))
    w = rng.standard_normal((27, 2, 3))
    b = np.zeros(3)
    gy = rng.standard_normal((4, 3, 5, 3))
    gx, gw, gb = unet.conv3d_backward(x, w, gy)
    dx = rng.standard_normal(x.shape)
    # <gy, conv(dx)> = <gx, dx>
    assert abs(np.sum(gy * unet.conv3d(dx, w, b)) - np.sum(gx * dx)) < 1e-10
    dw = rng.standard_normal(w.shape)
    assert abs(np.sum(gy * unet.conv3d(x, dw, b)) - np.sum(gw * dw)) < 1e-10
    np.testing.assert_allclose(gb, gy.sum(axis=(0, 1, 2)))


def test_unet_gradient_finite_differences():
    rng = np.random.default_rng(3)
    cin, cout, n = 5, 4, 4
    npar = unet.n_params(cin, cout)
    theta = rng.standard_normal(npar) * 0.2
    x = rng.standard_normal((n, n, n, cin))
    t = rng.standard_normal((n, n, n, cout))
    loss, g = unet.loss_and_grad(theta, x, t, cin, cout)
    idx = rng.choice(npar, 24, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (unet.loss_and_grad(tp, x, t, cin, cout)[0] - unet.loss_and_grad(tm, x, t, cin, cout)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_is_signed_lr():
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = unet.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-4)

"""Pins of the FP64 CPU U-Net (the learned warm start's reference): finite
differences of the hand-written backward pass, closed-form convolutions,
translation equivariance and adjointness of the transfer operators."""
import numpy as np
import pytest

from oracle import unet


def test_single_tap_convolution_is_a_periodic_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 6, 6, 6))
    W = np.zeros((27, 2, 2))
    t = unet.TAPS.index((0, 0, 1))            # dx = +1
    W[t] = np.eye(2)
    b = np.array([0.5, -1.0])
    y = unet.conv3(x, W, b)
    want = np.roll(x, shift=-1, axis=3) + b[:, None, None, None]   # y[..., x] = x[..., x+1]
    assert np.allclose(y, want)
    t = unet.TAPS.index((-1, 1, 0))           # dz = -1, dy = +1
    W[:] = 0
    W[t] = np.array([[0.0, 2.0], [1.0, 0.0]])
    y = unet.conv3(x, W, np.zeros(2))
    sh = x[:, (np.arange(6) - 1) % 6][:, :, (np.arange(6) + 1) % 6]
    assert np.allclose(y[0], sh[1]) and np.allclose(y[1], 2 * sh[0])


def test_transfer_operators_are_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 8, 8, 8))
    yc = rng.standard_normal((3, 4, 4, 4))
    assert abs((unet.pool(x) * yc).sum() - (x * unet.pool_backward(yc)).sum()) < 1e-12
    assert abs((unet.up(yc) * x).sum() - (yc * unet.up_backward(x)).sum()) < 1e-12
    assert np.allclose(unet.pool(unet.up(yc)), yc)


def test_translation_equivariance_by_multiples_of_eight():
    widths = (2, 3, 3, 4)
    p = unet.init_params(widths, seed=2)
    rng = np.random.default_rng(3)
    x = rng.uniform(size=(1, 16, 16, 16))
    y, _ = unet.forward(p, x)
    ys, _ = unet.forward(p, np.roll(x, shift=(8, 0, 8), axis=(1, 2, 3)))
    assert np.allclose(ys, np.roll(y, shift=(8, 0, 8), axis=(1, 2, 3)), atol=1e-12)


def test_backward_matches_central_differences():
    widths = (2, 2, 3, 2)
    n = 8
    p = unet.init_params(widths, seed=4)
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(1, n, n, n))
    target = rng.standard_normal((3, n, n, n))

    def loss(pp, xx):
        y, _ = unet.forward(pp, xx)
        return unet.mse_loss(y, target)[0]

    y, cache = unet.forward(p, x)
    _, dy = unet.mse_loss(y, target)
    g, dx = unet.backward(p, cache, dy, widths)
    h = 1e-6
    checked = 0
    for name in p:
        flat = p[name].ravel()
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            pp = {k: v.copy() for k, v in p.items()}
            pm = {k: v.copy() for k, v in p.items()}
            pp[name].ravel()[idx] += h
            pm[name].ravel()[idx] -= h
            fd = (loss(pp, x) - loss(pm, x)) / (2 * h)
            an = g[name].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)
            checked += 1
    for idx in rng.choice(x.size, size=4, replace=False):
        xp, xm = x.copy(), x.copy()
        xp.ravel()[idx] += h
        xm.ravel()[idx] -= h
        fd = (loss(p, xp) - loss(p, xm)) / (2 * h)
        assert abs(fd - dx.ravel()[idx]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9
    assert checked == sum(min(3, v.size) for v in p.values())


def test_parameter_count_of_the_full_width_network():
    p = unet.init_params((16, 32, 64, 128), seed=0)
    count = sum(v.size for v in p.values())
    assert 1.4e6 < count < 1.6e6

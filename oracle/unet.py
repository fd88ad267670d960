"""FP64 CPU reference of the periodic 3-D convolutional U-Net used as the
learned warm start of the homogenization solve (the learned predictor of the
corrector fields; the paper has no such network -- this is test
infrastructure for checking the GPU network's forward and backward passes).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Network (widths c = (c0, c1, c2, c3), grid n divisible by 8):
  E0 = B(1 -> c0)(x)                       at n
  E1 = B(c0 -> c1)(pool(E0))               at n/2
  E2 = B(c1 -> c2)(pool(E1))               at n/4
  E3 = B(c2 -> c3)(pool(E2))               at n/8
  D2 = B(c3 + c2 -> c2)(cat(up(E3), E2))   at n/4
  D1 = B(c2 + c1 -> c1)(cat(up(D2), E1))   at n/2
  D0 = B(c1 + c0 -> c0)(cat(up(D1), E0))   at n
  y  = H(D0)                               1x1 convolution c0 -> 3, with bias
where B(a -> b) = relu(conv3(relu(conv3(., a -> b)), b -> b)), conv3 is a
3x3x3 convolution with circular (periodic) padding and bias, pool is the
2x2x2 average, up the nearest-neighbour x2 upsampling, cat concatenates
channels (upsampled first).  Tensors are arrays of shape (C, n, n, n)
indexed [c, z, y, x]; conv3 weights have shape (27, Cin, Cout) with tap
index t = (dz+1)*9 + (dy+1)*3 + (dx+1), and
  out[co, v] = b[co] + sum_t sum_ci W[t, ci, co] in[ci, v + (dx, dy, dz)].

Parity: pinned -- finite differences of every parameter group and of the
input, an identity-kernel convolution, translation equivariance, and the
pooling / upsampling adjointness (tests/test_oracle_unet.py).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(x, W, b):
    """x (Cin, n, n, n), W (27, Cin, Cout), b (Cout,) -> (Cout, n, n, n)."""
    cout = W.shape[2]
    out = np.zeros((cout,) + x.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        sh = np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))     # sh[:, z, y, x] = x[:, z+dz, y+dy, x+dx]
        out += np.einsum("ic,izyx->czyx", W[t], sh)
    return out + b[:, None, None, None]


def conv3_backward(x, W, dout):
    """Gradients of sum(dout * conv3(x, W, b)) w.r.t. x, W, b."""
    dx_ = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t, (dz, dy, dx) in enumerate(TAPS):
        sh = np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))
        dW[t] = np.einsum("izyx,czyx->ic", sh, dout)
        g = np.einsum("ic,czyx->izyx", W[t], dout)               # gradient w.r.t. the shifted input
        dx_ += np.roll(g, shift=(dz, dy, dx), axis=(1, 2, 3))
    db = dout.sum(axis=(1, 2, 3))
    return dx_, dW, db


def pool(x):
    c, n = x.shape[0], x.shape[1]
    return x.reshape(c, n // 2, 2, n // 2, 2, n // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dout):
    return np.repeat(np.repeat(np.repeat(dout, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(dout):
    c, n = dout.shape[0], dout.shape[1]
    return dout.reshape(c, n // 2, 2, n // 2, 2, n // 2, 2).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


BLOCKS = ["E0", "E1", "E2", "E3", "D2", "D1", "D0"]


def block_channels(widths):
    c0, c1, c2, c3 = widths
    return {"E0": (1, c0), "E1": (c0, c1), "E2": (c1, c2), "E3": (c2, c3),
            "D2": (c3 + c2, c2), "D1": (c2 + c1, c1), "D0": (c1 + c0, c0)}


def init_params(widths, seed=0):
    """He-style normal initialisation (the GPU network has its own)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (a, b) in block_channels(widths).items():
        p[name + ".W1"] = rng.standard_normal((27, a, b)) * np.sqrt(2.0 / (27 * a))
        p[name + ".b1"] = 0.01 * rng.standard_normal(b)
        p[name + ".W2"] = rng.standard_normal((27, b, b)) * np.sqrt(2.0 / (27 * b))
        p[name + ".b2"] = 0.01 * rng.standard_normal(b)
    p["H.W"] = rng.standard_normal((widths[0], 3)) * np.sqrt(1.0 / widths[0])
    p["H.b"] = np.zeros(3)
    return p


def _block(p, name, x, cache):
    h1 = relu(conv3(x, p[name + ".W1"], p[name + ".b1"]))
    h2 = relu(conv3(h1, p[name + ".W2"], p[name + ".b2"]))
    cache[name] = (x, h1, h2)
    return h2


def forward(p, x):
    """x (1, n, n, n) -> y (3, n, n, n) and the cache for backward."""
    cache = {}
    e0 = _block(p, "E0", x, cache)
    e1 = _block(p, "E1", pool(e0), cache)
    e2 = _block(p, "E2", pool(e1), cache)
    e3 = _block(p, "E3", pool(e2), cache)
    d2 = _block(p, "D2", np.concatenate([up(e3), e2]), cache)
    d1 = _block(p, "D1", np.concatenate([up(d2), e1]), cache)
    d0 = _block(p, "D0", np.concatenate([up(d1), e0]), cache)
    y = np.einsum("ic,izyx->czyx", p["H.W"], d0) + p["H.b"][:, None, None, None]
    cache["H"] = d0
    return y, cache


def _block_backward(p, name, dh2, cache, grads):
    x, h1, h2 = cache[name]
    dpre2 = dh2 * (h2 > 0)
    dh1, grads[name + ".W2"], grads[name + ".b2"] = conv3_backward(h1, p[name + ".W2"], dpre2)
    dpre1 = dh1 * (h1 > 0)
    dx, grads[name + ".W1"], grads[name + ".b1"] = conv3_backward(x, p[name + ".W1"], dpre1)
    return dx


def backward(p, cache, dy, widths):
    """Gradients of sum(dy * y) w.r.t. every parameter and the input."""
    c0, c1, c2, c3 = widths
    g = {}
    d0 = cache["H"]
    g["H.W"] = np.einsum("izyx,czyx->ic", d0, dy)
    g["H.b"] = dy.sum(axis=(1, 2, 3))
    dd0 = np.einsum("ic,czyx->izyx", p["H.W"], dy)
    dcat0 = _block_backward(p, "D0", dd0, cache, g)
    dup1, de0 = dcat0[:c1], dcat0[c1:]
    dd1 = up_backward(dup1)
    dcat1 = _block_backward(p, "D1", dd1, cache, g)
    dup2, de1 = dcat1[:c2], dcat1[c2:]
    dd2 = up_backward(dup2)
    dcat2 = _block_backward(p, "D2", dd2, cache, g)
    dup3, de2 = dcat2[:c3], dcat2[c3:]
    de3 = up_backward(dup3)
    dp3 = _block_backward(p, "E3", de3, cache, g)
    de2 = de2 + pool_backward(dp3)
    dp2 = _block_backward(p, "E2", de2, cache, g)
    de1 = de1 + pool_backward(dp2)
    dp1 = _block_backward(p, "E1", de1, cache, g)
    de0 = de0 + pool_backward(dp1)
    dx = _block_backward(p, "E0", de0, cache, g)
    return g, dx


def mse_loss(y, target):
    """L = mean over all entries of (y - target)^2 and dL/dy."""
    d = y - target
    return float((d * d).mean()), 2.0 * d / d.size

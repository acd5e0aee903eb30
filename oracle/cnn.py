"""FP64 reference of the learned localiser -- TEST INFRASTRUCTURE ONLY.

A small fully-convolutional network maps a projection plane (XDoppler
amplitude divided by its frame maximum) to a microbubble heatmap on a
4x finer grid:

    conv3x3(1 -> C) + ReLU, conv3x3(C -> C) + ReLU, conv3x3(C -> C) + ReLU,
    conv3x3(C -> 16), pixel shuffle (16 channels -> 4 x 4 sub-pixels),

trained with a mean-squared error against Gaussian targets (sigma = 1 pixel
of the fine grid) and Adam.  The paper names learned localisation only as
future work (Sec. IV); this network, its loss and optimiser are the build's
reading.  Convolutions use zero "same" padding; tensors are NHWC.

Plain numpy in double precision: every convolution is a sum over the nine
taps of a shifted input times the tap's weight matrix (``@`` is the library
matmul used as a step).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # tap index = 3 (dy+1) + (dx+1)
UP = 4


def shifted(x, dy, dx):
    """x [B][H][W][C] -> s with s[:, i, j] = x[:, i + dy, j + dx] (zero outside)."""
    B, H, W, C = x.shape
    s = np.zeros_like(x)
    i0, i1 = max(0, -dy), min(H, H - dy)
    j0, j1 = max(0, -dx), min(W, W - dx)
    s[:, i0:i1, j0:j1] = x[:, i0 + dy:i1 + dy, j0 + dx:j1 + dx]
    return s


def conv3x3(x, w, b):
    """y[p, o] = b[o] + sum_taps sum_c x[p + tap, c] w[o, tap, c];  w [O][9][C]."""
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dy, dx) in enumerate(TAPS):
        y += shifted(x, dy, dx) @ w[:, t, :].T
    return y + b


def conv3x3_backward(x, w, dy_out):
    """gradients of conv3x3 w.r.t. its input, weights and bias."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (ty, tx) in enumerate(TAPS):
        xs = shifted(x, ty, tx)
        dw[:, t, :] = np.einsum("bhwo,bhwc->oc", dy_out, xs)
        # x[p + tap] feeds y[p]: route dy back to p + tap
        dx += shifted(dy_out @ w[:, t, :], -ty, -tx)
    db = dy_out.sum(axis=(0, 1, 2))
    return dx, dw, db


def pixel_shuffle(z):
    """z [B][H][W][16] -> [B][4H][4W]: channel 4a + c goes to sub-pixel (a, c)."""
    B, H, W, C = z.shape
    assert C == UP * UP
    return z.reshape(B, H, W, UP, UP).transpose(0, 1, 3, 2, 4).reshape(B, H * UP, W * UP)


def pixel_unshuffle(y):
    B, H4, W4 = y.shape
    return y.reshape(B, H4 // UP, UP, W4 // UP, UP).transpose(0, 1, 3, 2, 4).reshape(B, H4 // UP, W4 // UP, UP * UP)


def init_params(C=32, seed=0):
    """He-normal weights, zero biases; shapes [O][9][I]."""
    rng = np.random.default_rng(seed)
    shapes = [(C, 1), (C, C), (C, C), (UP * UP, C)]
    params = []
    for o, i in shapes:
        params.append(rng.standard_normal((o, 9, i)) * np.sqrt(2.0 / (9 * i)))
        params.append(np.zeros(o))
    return params


def forward(params, x):
    """x [B][H][W] plane -> (heatmap [B][4H][4W], cache)."""
    a = x[..., None].astype(np.float64)
    cache = [a]
    for layer in range(4):
        w, b = params[2 * layer], params[2 * layer + 1]
        z = conv3x3(a, w, b)
        a = np.maximum(z, 0.0) if layer < 3 else z
        cache.append(a)
    return pixel_shuffle(a), cache


def mse(y, t):
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, cache, dheat):
    """gradients of every parameter given dL/dheatmap."""
    grads = [None] * 8
    g = pixel_unshuffle(dheat)
    for layer in (3, 2, 1, 0):
        w = params[2 * layer]
        x_in = cache[layer]
        dx, dw, db = conv3x3_backward(x_in, w, g)
        grads[2 * layer], grads[2 * layer + 1] = dw, db
        if layer > 0:
            g = dx * (cache[layer] > 0)   # ReLU of the previous layer
    return grads


def loss_and_grads(params, x, target):
    heat, cache = forward(params, x)
    loss, dheat = mse(heat, target)
    return loss, backward(params, cache, dheat)


class Adam:
    """Adam with bias correction (beta1 0.9, beta2 0.999, eps 1e-8, lr 1e-3)."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for q, (p, g) in enumerate(zip(params, grads)):
            self.m[q] = self.b1 * self.m[q] + (1 - self.b1) * g
            self.v[q] = self.b2 * self.v[q] + (1 - self.b2) * g * g
            mh = self.m[q] / (1 - self.b1 ** self.t)
            vh = self.v[q] / (1 - self.b2 ** self.t)
            out.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out


def target_heatmap(H, W, points, sigma=1.0):
    """Sum of unit Gaussians on the 4x grid; points = [(z4, x4), ...] in fine
    pixel units (pixel centres at integers)."""
    ii, jj = np.meshgrid(np.arange(H * UP), np.arange(W * UP), indexing="ij")
    t = np.zeros((H * UP, W * UP))
    for z4, x4 in points:
        t += np.exp(-((ii - z4) ** 2 + (jj - x4) ** 2) / (2 * sigma * sigma))
    return t


def flatten(params):
    return np.concatenate([p.ravel() for p in params])


def unflatten(vec, C=32):
    shapes = [(C, 9, 1), (C,), (C, 9, C), (C,), (C, 9, C), (C,), (UP * UP, 9, C), (UP * UP,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(vec[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out

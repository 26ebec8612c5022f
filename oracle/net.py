"""ORACLE -- test infrastructure only.

Plain FP64 numpy restatement of the learned Poisson warm start: a 3D
convolutional network (3^3 kernels, channels 2 -> 16 -> 16 -> 16 -> 1, ReLU
between layers, linear output) that maps the step's change of the Poisson
source and the previous potential to the change of the potential, its
mean-squared loss and the gradients of that loss by reverse-mode chain rule.
Pinned by finite differences in tests/test_oracle_net.py.

Parameter vector layout (FP32/FP64 flat): for each layer W[co][ci][k] then
b[co], k = (dz+1)*9 + (dy+1)*3 + (dx+1) over the 27 offsets.  Boundary:
periodic wrap on periodic axes, zeros beyond closed ones.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 16, 16, 16, 1)
OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def n_params():
    return sum(co * ci * 27 + co for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]))


def unpack(w):
    out, o = [], 0
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        W = np.asarray(w[o:o + co * ci * 27], np.float64).reshape(co, ci, 27)
        o += co * ci * 27
        b = np.asarray(w[o:o + co], np.float64)
        o += co
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def init_params(seed=0):
    """He-style initial weights (seeded)."""
    rng = np.random.default_rng(seed)
    layers = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        W = rng.standard_normal((co, ci, 27)) * np.sqrt(2.0 / (ci * 27))
        layers.append((W, np.zeros(co)))
    return pack(layers)


def shift(x, off, periodic):
    """x[c, z, y, x] -> value at (node + off), zero beyond a closed face."""
    out = x
    for axis_np, d, per in ((3, off[0], periodic[0]), (2, off[1], periodic[1]), (1, off[2], periodic[2])):
        if d == 0:
            continue
        out = np.roll(out, -d, axis=axis_np)
        if not per:
            sl = [slice(None)] * out.ndim
            sl[axis_np] = slice(-1, None) if d > 0 else slice(0, 1)
            out = out.copy()
            out[tuple(sl)] = 0.0
    return out


def conv(x, W, b, periodic):
    """y[co, n] = b[co] + sum_k sum_ci W[co, ci, k] x[ci, n + off_k]."""
    co = W.shape[0]
    y = np.zeros((co,) + x.shape[1:])
    for k, off in enumerate(OFFSETS):
        xs = shift(x, off, periodic)
        y += np.einsum("oc,c...->o...", W[:, :, k], xs)
    return y + b[:, None, None, None]


def conv_adjoint(g, W, periodic):
    """Gradient with respect to the input of conv: d_x[ci, m] =
    sum_k sum_co W[co, ci, k] g[co, m - off_k]."""
    ci = W.shape[1]
    dx = np.zeros((ci,) + g.shape[1:])
    for k, off in enumerate(OFFSETS):
        gs = shift(g, (-off[0], -off[1], -off[2]), periodic)
        dx += np.einsum("oc,o...->c...", W[:, :, k], gs)
    return dx


def forward(x, w, periodic, keep=False):
    layers = unpack(w)
    acts = [x]
    a = x
    for l, (W, b) in enumerate(layers):
        z = conv(a, W, b, periodic)
        a = np.maximum(z, 0.0) if l < len(layers) - 1 else z
        acts.append(a)
    return (a[0], acts) if keep else a[0]


def loss_grad(x, target, mask, w, periodic):
    """Mean squared error over the masked nodes and its gradient."""
    layers = unpack(w)
    y, acts = forward(x, w, periodic, keep=True)
    m = mask.astype(bool)
    cnt = max(int(m.sum()), 1)
    diff = np.where(m, y - target, 0.0)
    loss = float((diff ** 2).sum() / cnt)
    g = (2.0 / cnt) * diff[None]
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        a_in = acts[l]
        if l < len(layers) - 1:
            g = g * (acts[l + 1] > 0)
        dW = np.zeros_like(W)
        for k, off in enumerate(OFFSETS):
            xs = shift(a_in, off, periodic)
            dW[:, :, k] = g.reshape(g.shape[0], -1) @ xs.reshape(xs.shape[0], -1).T
        db = g.reshape(g.shape[0], -1).sum(1)
        grads.append((dW, db))
        if l > 0:
            g = conv_adjoint(g, W, periodic)
    grads.reverse()
    return loss, pack(grads)

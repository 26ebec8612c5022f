"""Training and evaluation of the learned Poisson warm start.

Data recorded by the library during plain steps (ekl_warmstart_collect): the
change of the Poisson source, the previous potential and the change of the
converged potential -- as crops near the beads when the network runs on the
lattice, or as whole coarse grids when it runs on a coarse level
(ekl_warmstart_level).  Inputs and target are scaled by their standard
deviations; the target's mean over each sample is removed (a constant does
not change the residual) and the previous potential gets a random constant
per sample so the network learns not to depend on the potential's level.
Training runs on the GPU (ekl_net_train, ekl_net_train_grid); nothing here
touches the oracle.
"""
from __future__ import annotations

import numpy as np

from . import EKL_NET_PARAMS, ekl_net_train, ekl_net_train_grid

CHANNELS = (2, 16, 16, 16, 1)


def init_params(seed=0):
    """He-style initial weights; per layer W[co][ci][k] then b[co]."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        parts.append(rng.standard_normal(co * ci * 27) * np.sqrt(2.0 / (ci * 27)))
        parts.append(np.zeros(co))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == EKL_NET_PARAMS
    return w


def prepare(crops, seed=0):
    """(x, t, mask, scales) from collected crops[k][3][c][c][c]."""
    rng = np.random.default_rng(seed)
    db, ph, dp = crops[:, 0], crops[:, 1], crops[:, 2]
    s_db = 1.0 / max(float(db.std()), 1e-30)
    s_phi = 1.0 / max(float(ph.std()), 1e-30)
    tgt = dp - dp.mean(axis=(1, 2, 3), keepdims=True)
    s_out = max(float(tgt.std()), 1e-30)
    phc = ph - ph.mean(axis=(1, 2, 3), keepdims=True) + rng.normal(0, 2 * ph.std(), (len(ph), 1, 1, 1))
    x = np.stack([db * s_db, phc * s_phi], axis=1).astype(np.float32)
    t = (tgt / s_out).astype(np.float32)
    c = crops.shape[-1]
    mask = np.zeros((c, c, c), np.uint8)
    mask[4:c - 4, 4:c - 4, 4:c - 4] = 1   # receptive field inside the crop
    return x, t, mask, (s_db, s_phi, s_out)


def prepare_fields(samples, seed=0):
    """(x, t, scales) from whole coarse-grid samples[k][3][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    db, ph, dp = samples[:, 0], samples[:, 1], samples[:, 2]
    s_db = 1.0 / max(float(db.std()), 1e-30)
    s_phi = 1.0 / max(float(ph.std()), 1e-30)
    tgt = dp - dp.mean(axis=(1, 2, 3), keepdims=True)
    s_out = max(float(tgt.std()), 1e-30)
    phc = ph - ph.mean(axis=(1, 2, 3), keepdims=True) + rng.normal(0, 2 * ph.std(), (len(ph), 1, 1, 1))
    x = np.stack([db * s_db, phc * s_phi], axis=1).astype(np.float32)
    t = (tgt / s_out).astype(np.float32)
    return x, t, (s_db, s_phi, s_out)


def train_fields(samples, periodic, iters=1000, batch=8, lr=2e-3, seed=0):
    """Train the network on whole coarse grids of a box with the given
    periodic axes; returns (weights, scales, loss curve)."""
    x, t, scales = prepare_fields(samples, seed)
    nz, ny, nx = samples.shape[-3:]
    w, curve = ekl_net_train_grid((nx, ny, nz), periodic, x, t, None, init_params(seed), iters, batch, lr, seed)
    return w, scales, curve


def train(crops, iters=600, batch=8, lr=2e-3, seed=0):
    x, t, mask, scales = prepare(crops, seed)
    c = crops.shape[-1]
    w, curve = ekl_net_train((c, c, c), x, t, mask, init_params(seed), iters, batch, lr, seed)
    return w, scales, curve


def compare(make_sim, w, scales, steps):
    """Sweeps per step and wall time of the same run without and with the
    warm start, from identical initial states.  Returns dicts."""
    import time
    out = {}
    for name, use in (("plain", False), ("learned", True)):
        sim = make_sim()
        if use:
            sim.set_warmstart(w, scales)
        s0 = sim.stats()["poisson_sweeps"]
        t0 = time.perf_counter()
        sim.step(steps)
        dt = time.perf_counter() - t0
        st = sim.stats()
        out[name] = dict(sweeps_per_step=(st["poisson_sweeps"] - s0) / steps, seconds=dt,
                         residual=st["poisson_res"])
        sim.close()
    return out

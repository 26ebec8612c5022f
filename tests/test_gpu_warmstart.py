"""Learned warm start in the step: trained on crops the solver itself
generates, it leaves the solve's residual bound unchanged (the iteration
still runs to poisson_tol) and the test reports the sweeps it saves."""
import numpy as np
import pytest

import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import warmstart as WS
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_warmstart_collect_train_and_gain():
    wl = W.small_pore(nx=32, ny=32, nz=48, membrane=(22, 25), radius=4.0, n_beads=8,
                      precision="f32").replace(poisson_tol=1e-8, poisson_check_every=2)
    sim = E.Simulation(wl)
    sim.step(20)
    crops = sim.collect(120, crop=16, ncrops=8, seed=1)
    sim.close()
    assert crops.shape == (960, 3, 16, 16, 16) and np.isfinite(crops).all()
    assert np.abs(crops[:, 2]).max() > 0
    w, scales, curve = WS.train(crops, iters=300, batch=8, lr=2e-3, seed=0)
    assert curve[-20:].mean() < 0.7 * curve[:20].mean(), (curve[:5], curve[-5:])

    def make():
        s = E.Simulation(wl)
        s.step(20)
        return s

    res = WS.compare(make, w, scales, 60)
    print(res)
    for k in ("plain", "learned"):
        assert res[k]["residual"] <= 1e-8
    # the network may or may not pay for itself on a small box; it must not
    # make the iteration diverge
    assert res["learned"]["sweeps_per_step"] < 2 * res["plain"]["sweeps_per_step"]

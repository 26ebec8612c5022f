"""Failure detection without faulting the GPU: errors made on the host (a
non-finite population handed in through a checkpoint, an iteration cap the
solver cannot meet) and a device-side wait that runs out (a barrier one
block never reaches).  After each, the context stays usable."""
import numpy as np
import pytest

import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _small(**kw):
    return W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=4,
                        precision="f32").replace(**kw)


def _still_works():
    sim = E.Simulation(_small())
    assert sim.step(3) >= 0
    sim.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_nan_population_is_reported_unstable(precision):
    wl = _small(precision=precision)
    sim = E.Simulation(wl)
    sim.step(2)
    f, phi, step = sim.get_state()
    node = int(np.flatnonzero(wl.solid.ravel() == 0)[500])   # a fluid node
    f[1, 3, node] = np.nan
    sim.set_state(f, phi, step)
    with pytest.raises(E.EklError) as ei:
        sim.step(1)
    assert ei.value.code == E.EKL_ERR_UNSTABLE
    sim.close()
    _still_works()


@pytest.mark.parametrize("flags", [0, W.FLAG_POISSON_MG])
def test_iteration_cap_warns(flags):
    sim = E.Simulation(_small(poisson_tol=1e-15, poisson_max_iter=2, flags=flags))
    rc = sim.step(1)
    assert rc > 0 and (rc & E.EKL_WARN_NOCONV), rc
    assert sim.stats()["poisson_iters"] == 2
    sim.close()
    _still_works()


def test_device_wait_gives_up():
    L = E.load()
    assert L.ekl_selftest_wait() == E.EKL_ERR_TIMEOUT
    assert b"timed out" in L.ekl_last_error()
    _still_works()

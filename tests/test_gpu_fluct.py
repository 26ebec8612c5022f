"""The fluctuating collision term (Eq. 14) on the GPU.

* FP64 path against the oracle to 1e-12: the noise is deterministic
  (Philox, same counters and key on both sides), so the trajectories agree
  to round-off, in a periodic box and in a pore with a bead chain;
* FP32 path: fluctuation-dissipation in a periodic box at rest,
  Var(n) = m n and Var(j_x) = m n / 3 per node (the oracle's pin), and mass
  conservation.
"""
import numpy as np
import pytest

import oracle
import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import workloads as W
from helpers import box, rel
from test_gpu_parity import _compare

pytestmark = pytest.mark.gpu


def _fluct_box(tau, m, n=(1.0, 1.0, 1.0)):
    return box(8, 8, 8, periodic=(1, 1, 1), n=n, bjerrum=0.0, tau=(tau, tau, tau),
               diffusivity=(1e6, 1e6, 1e6), fluct_mass=m, seed=5)


def test_fluct_fp64_matches_oracle_box():
    wl = box(12, 10, 8, periodic=(1, 1, 1), n=(1.0, 0.5, 0.5), tau=(0.9, 0.9, 0.9),
             E_app=(1e-3, 0.0, 0.0), fluct_mass=1e-4, seed=11, poisson_tol=1e-12,
             n_init=W.ion_densities(np.zeros((8, 10, 12), np.uint8), 0.5, 1.0, 0.0, 1e-3, 3))
    errs, _, _ = _compare(wl, 50, 1e-12, precision="f64", check_beads=False)
    assert all(v < 1e-12 for v in errs.values()), errs


def test_fluct_fp64_matches_oracle_pore_with_chain():
    wl = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=4,
                      precision="f64").replace(fluct_mass=1e-6, poisson_tol=1e-12)
    errs, _, _ = _compare(wl, 30, 1e-12, precision="f64")
    assert all(v < 1e-12 for v in errs.values()), errs


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_fluct_fp32_fluctuation_dissipation(tau):
    m = 1e-3
    sim = E.Simulation(_fluct_box(tau, m), precision="f32")
    sim.step(400)
    m0 = sim.stats()["mass"]
    vn, vj = [], []
    for _ in range(150):
        sim.step(5)
        F = sim.fields(("n", "j"))
        vn.append(F["n"].var(axis=1))
        vj.append(F["j"][:, 0].var(axis=1))
    m1 = sim.stats()["mass"]
    sim.close()
    vn = np.mean(vn, axis=0) / m
    vj = np.mean(vj, axis=0) / (m / 3.0)
    print("Var(n)/(m n)", vn, "Var(j_x)/(m n/3)", vj)
    assert np.allclose(vn, 1.0, rtol=0.05) and np.allclose(vj, 1.0, rtol=0.05), (vn, vj)
    assert np.all(np.abs(m1 / m0 - 1) < 1e-6), (m0, m1)

"""Pins of the oracle's bead side (Sec. II.B; interpolation kernel of Sec. II.C).

* the trilinear kernel is a partition of unity, reproduces linear fields
  exactly, gives wall nodes zero weight (renormalising the rest) and wraps
  periodic axes;
* spreading and interpolating with the same weights are adjoint, which is
  what makes the bead-fluid momentum exchange exact (checked end to end in
  the momentum test of test_oracle_lb.py);
* a two-bead FENE + WCA dimer relaxes to the minimum of the textbook energy
  (Eq. 9 with the Kremer-Grest bond), found here by a scalar minimiser;
* the Langevin noise has zero mean and unit variance.
"""
import math

import numpy as np
from scipy.optimize import minimize_scalar

import oracle
from helpers import box, node_coords
from paper_1710_09421_gb300 import workloads as W

KT = 1.0 / 3.0


def test_stencil_partition_and_linear_exactness():
    wl = box(8, 8, 8)
    s = oracle.Sim(wl)
    x, y, z = node_coords(8, 8, 8)
    rng = np.random.default_rng(1)
    field = 0.3 + 0.2 * x - 0.7 * y + 0.11 * z
    for _ in range(20):
        R = rng.uniform(1, 6, 3)
        ok, nodes, w = s.bead_stencil(R)
        assert ok and abs(w.sum() - 1) < 1e-15 and np.all(w >= 0)
        val = (w * field[nodes]).sum()
        assert abs(val - (0.3 + 0.2 * R[0] - 0.7 * R[1] + 0.11 * R[2])) < 1e-13


def test_stencil_periodic_wrap_and_walls():
    wl = box(8, 6, 10, periodic=(1, 1, 0), solid=W.slit_solid(8, 6, 10))
    s = oracle.Sim(wl)
    ok, nodes, w = s.bead_stencil(np.array([7.25, 5.5, 1.4]))
    assert ok
    xs = nodes % 8
    ys = (nodes // 8) % 6
    zs = nodes // 48
    assert set(xs) == {7, 0} and set(ys) == {5, 0}
    # z = 1 and 2 are fluid here: plain trilinear weights
    assert abs(w.sum() - 1) < 1e-15 and np.all(w > 0)
    ok, nodes, w = s.bead_stencil(np.array([3.5, 2.5, 0.6]))   # between wall z=0 and z=1
    assert ok
    zs = nodes // 48
    assert np.all(w[zs == 0] == 0) and abs(w[zs == 1].sum() - 1) < 1e-15
    ok, _, _ = s.bead_stencil(np.array([3.5, 2.5, -0.5]))
    assert not ok


def test_spread_interpolate_adjoint():
    wl = box(8, 8, 8)
    s = oracle.Sim(wl)
    rng = np.random.default_rng(2)
    N = 512
    u = rng.standard_normal(N)
    R = rng.uniform(0, 8, (5, 3))
    F = rng.standard_normal(5)
    spread = np.zeros(N)
    interp = np.zeros(5)
    for i in range(5):
        ok, nodes, w = s.bead_stencil(R[i])
        np.add.at(spread, nodes, F[i] * w)
        interp[i] = (w * u[nodes]).sum()
    assert abs((spread * u).sum() - (F * interp).sum()) < 1e-12
    assert abs(spread.sum() - F.sum()) < 1e-13


def _kg_energy(r, eps=KT, sig=1.0, k=30 * KT, R0=1.5):
    u = -0.5 * k * R0 ** 2 * math.log(1 - (r / R0) ** 2)
    if r < 2 ** (1 / 6) * sig:
        u += 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6) + eps
    return u


def test_fene_wca_dimer_rests_at_energy_minimum():
    rmin = minimize_scalar(_kg_energy, bounds=(0.8, 1.2), method="bounded",
                           options={"xatol": 1e-12}).x
    R = np.array([[5.0, 6.1, 5.7], [5.0 + 1.05, 6.1, 5.7]])
    wl = box(12, 12, 12, flags=W.FLAG_NO_BEAD_NOISE, R=R, V=np.zeros_like(R),
             charge=np.zeros(2), chain=np.zeros(2, np.int32), md_substeps=10)
    s = oracle.Sim(wl)
    assert s.step(400) >= 0
    Rf = s.fields()["R"]
    d = np.linalg.norm(Rf[1] - Rf[0])
    assert abs(d - rmin) < 1e-6, (d, rmin)


def test_noise_moments():
    xs = []
    for c in range(20000):
        o = oracle.philox4x32_10([c, 1 << 24, 7, 0], [2, 0])
        xs.extend(o[:3])
    u = (np.array(xs, np.float64) * 2 + 1) / 2 ** 32 - 1
    xi = math.sqrt(3) * u
    assert abs(xi.mean()) < 0.02 and abs(xi.var() - 1) < 0.02

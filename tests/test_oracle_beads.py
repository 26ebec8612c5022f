"""Pins of the oracle's bead side (Sec. II.B; interpolation kernel of Sec. II.C).

* the trilinear kernel is a partition of unity, reproduces linear fields
  exactly, gives wall nodes zero weight (renormalising the rest) and wraps
  periodic axes;
* spreading and interpolating with the same weights are adjoint, which is
  what makes the bead-fluid momentum exchange exact (checked end to end in
  the momentum test of test_oracle_lb.py);
* a two-bead FENE + WCA dimer relaxes to the minimum of the textbook energy
  (Eq. 9 with the Kremer-Grest bond), found here by a scalar minimiser;
* the Langevin noise has zero mean and unit variance;
* friction (Sec. II.B, Eq. 7): a bead pulled by a constant force through a
  fluid too dense to move drifts at exactly force / xi, the total friction,
  in the direction of the force on its charge;
* thermostat (Eqs. 7-8, fluctuation-dissipation): the same bead with no
  force reaches equipartition, M <V_c^2> = k_B T, within the statistics and
  the O(xi dt / M) bias of a discrete integrator;
* hydrodynamic coupling: the mobility of a bead pulled through periodic
  boxes of side L falls as -2.837 / (6 pi eta L) (Hasimoto's periodic
  correction to Stokes drag), with eta the fluid's viscosity;
* bead-wall repulsion (Eq. 9a against wall nodes): a bead pushed onto a flat
  wall comes to rest where the WCA forces of the wall nodes within the
  cut-off balance the push.
"""
import math
import os

import numpy as np
from scipy.optimize import brentq, minimize_scalar

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


# A fluid of solvent density 1e6 per node (ions 1e-6) takes the bead's drag
# without moving: its velocity response is ~1e-6 of the bead's.
DENSE = (1e6, 1e-6, 1e-6)


def _one_bead(nx, ny, nz, R, q, E, periodic=(1, 1, 1), solid=None, n=DENSE, **kw):
    R = np.array([R], np.float64)
    return box(nx, ny, nz, periodic=periodic, solid=solid, n=n, bjerrum=0.0, E_app=E, R=R,
               V=np.zeros_like(R), charge=np.array([q]), chain=np.zeros(1, np.int32), **kw)


def test_bead_drifts_at_force_over_friction_in_a_fluid_at_rest():
    """Friction-dominated limit of Eq. 7: with the fluid held at rest the
    steady velocity is V = F / xi, F = q k_B T E the force on the bead's
    charge (Sec. II.B; field units k_B T / (e dx)).  A friction split
    gamma^a = xi n^a (instead of xi n^a / n), a wrong sign of the field force
    or of the drag, or a dropped species fails this."""
    xi, E, q = 2.0, 3e-3, -1.0
    s = oracle.Sim(_one_bead(8, 8, 8, (3.3, 4.6, 3.9), q, (0.0, 0.0, E), bead_xi=xi, bead_mass=10.0,
                             flags=W.FLAG_NO_BEAD_NOISE))
    assert s.step(300) == 0
    V = s.fields()["V"][0]
    F = q * KT * E
    assert abs(V[2] / (F / xi) - 1.0) < 1e-5, V
    assert V[2] < 0 and abs(V[0]) < 1e-15 and abs(V[1]) < 1e-15


def test_bead_equipartition_in_a_fluid_at_rest():
    """Fluctuation-dissipation of Eqs. 7-8: noise of variance 2 gamma k_B T /
    dt against the friction gamma = xi gives M <V_c^2> = k_B T.  The
    integrator (friction implicit in V, dt = 1/md_substeps) has the exact
    stationary value k_B T / (1 + a/2), a = xi dt / M (0.5 % below k_B T
    here).  A factor 2 in the variance, dt for 1/dt in the amplitude or the
    friction missing from it all fail; the statistical error of 30 000
    samples per component is about 0.6 %."""
    xi, M, nsub = 2.0, 2.0, 50
    s = oracle.Sim(_one_bead(4, 4, 4, (1.3, 2.6, 1.9), 0.0, (0.0, 0.0, 0.0), bead_xi=xi, bead_mass=M,
                             bead_kT=KT, md_substeps=nsub, seed=11))
    s.step(20)
    V = np.zeros((30000, 3))
    for k in range(len(V)):
        assert s.step(1) == 0
        V[k] = s.fields()["V"][0]
    a = xi / nsub / M
    ratio = M * (V ** 2).mean() / KT
    assert abs(ratio - 1.0 / (1.0 + 0.5 * a)) < 0.03, ratio
    assert np.all(np.abs(V.mean(axis=0)) < 0.05 * math.sqrt(KT / M))


def _mobility(L, tau, xi, M, steps):
    """Steady (V - u_mean) / F' of one bead pulled along z through a fully
    periodic box of side L.  The whole system accelerates at F / M_total;
    in its frame the bead feels F' = F (1 - M / M_total) and the fluid an
    even body force that balances it (Hasimoto's set-up), so V - u_mean is
    the same in both frames.  u_mean includes the half-force shift of the
    Guo scheme: fluid momentum = sum j + F_fluid / 2."""
    E = 3e-5
    n = (1.0, 1e-8, 1e-8)
    wl = _one_bead(L, L, L, (L / 2 + 0.3, L / 2 + 0.1, L / 2 + 0.45), -1.0, (0.0, 0.0, E), n=n,
                   tau=(tau,) * 3, bead_xi=xi, bead_mass=M, flags=W.FLAG_NO_BEAD_NOISE)
    s = oracle.Sim(wl, threads=os.cpu_count() or 1)
    assert s.step(steps) == 0
    f = s.fields()
    F = -KT * E
    ntot = f["n"].sum()
    u_mean = (f["j"][:, 2, :].sum() + 0.5 * F) / ntot
    return (f["V"][0, 2] - u_mean) / (F * (1.0 - M / (ntot + M)))


def test_single_bead_stokes_drag_hasimoto_finite_size():
    """Hasimoto (1959): in a periodic array of spheres the mobility relative
    to the mean fluid velocity is mu(L) = mu_inf - 2.837 / (6 pi eta L) +
    O(L^-3).  The bead's coupling to the fluid must reproduce it with the
    lattice viscosity eta = n (tau - 1/2) / 3: the slope of mu against 1/L
    between L = 24 and 32 within 3 % of the coefficient (the O(L^-3) term,
    set by the bead's hydrodynamic radius of about 1 dx, still moves it by
    2 %; between L = 32 and 48 the slope is within 1 %), and the L = 16 point
    on the same side of the line, as the positive cubic term puts it.
    Everything stays in the Stokes regime (force 1e-5)."""
    tau, xi, M = 2.0, 2.0, 10.0
    eta = (tau - 0.5) / 3.0
    mu = {L: _mobility(L, tau, xi, M, 600) for L in (16, 24, 32)}
    expected = -2.837 / (6.0 * math.pi * eta)
    slope = (mu[32] - mu[24]) / (1 / 32 - 1 / 24)
    assert abs(slope / expected - 1.0) < 0.03, (slope, expected)
    assert mu[16] > mu[24] + slope * (1 / 16 - 1 / 24)
    # the bead is hydrodynamically coupled: its mobility exceeds the bare 1/xi
    assert all(m > 1.0 / xi for m in mu.values())


def _wca(r, eps=KT, sig=1.0):
    """Eq. 9a: 4 eps ((sig/r)^12 - (sig/r)^6) + eps inside 2^(1/6) sig, else 0."""
    if r >= 2 ** (1 / 6) * sig:
        return 0.0
    return 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6) + eps


def test_bead_rests_on_a_wall_where_wca_balances_the_push():
    """A bead above the centre of a square of four wall nodes (lateral
    offset sqrt(1/2) from each; the next wall nodes lie beyond the cut-off)
    is pushed onto the wall z = 0 by its charge in a field.  It comes to
    rest at the height h where the normal WCA force of the four nodes,
    -4 U'(r) h / r with r^2 = 1/2 + h^2 (U of Eq. 9a, differentiated
    numerically here), equals the push.  A wrong sign (the bead enters the
    wall), a factor in the force or a missed wall node moves h."""
    for E in (0.3, 1.0):
        wl = _one_bead(8, 8, 10, (3.5, 4.5, 1.3), -1.0, (0.0, 0.0, E), periodic=(1, 1, 0),
                       solid=W.slit_solid(8, 8, 10), bead_xi=2.0, bead_mass=10.0,
                       flags=W.FLAG_NO_BEAD_NOISE)
        s = oracle.Sim(wl)
        assert s.step(200) == 0
        R = s.fields()["R"][0]
        push = KT * E

        def net(h):
            r = math.sqrt(0.5 + h * h)
            d = 1e-6
            f = -(_wca(r + d) - _wca(r - d)) / (2 * d)
            return 4 * f * h / r - push

        h = brentq(net, 0.5, math.sqrt(2 ** (1 / 3) - 0.5) - 1e-9, xtol=1e-14)
        assert abs(R[2] - h) < 1e-7, (E, R, h)
        assert R[0] == 3.5 and R[1] == 4.5

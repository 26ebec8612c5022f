"""Pins of the oracle's lattice-Boltzmann step against closed forms.

* per-species mass is conserved to round-off (bounce-back and BGK, Eq. 12);
* in a fully periodic box total momentum (fluid + beads) is conserved to the
  Poisson tolerance: the inter-species drag (Eq. 6) and the bead drag cancel
  pairwise, the field force sums to zero for a neutral system;
* plane Poiseuille flow between halfway bounce-back walls is exact at
  tau = 1/2 + sqrt(3/16) and carries an O(1/H^2) relative error otherwise;
* Nernst-Einstein: in a uniform field the ions drift relative to the solvent
  at u^+- - u = +-D E exactly (Eq. 6 with D = v_T^2 / omega_drag);
* zero-field equilibrium at a charged wall matches the discrete
  Poisson-Boltzmann profile n^+- = c^+- exp(-+phi) (Newton solve);
* electro-osmotic flow matches Smoluchowski, u(z) = k_B T E (phi - phi_w) /
  (4 pi l_B eta) with the simulated potential.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import box, slit, node_coords, rel
from paper_1710_09421_gb300 import workloads as W

KT = 1.0 / 3.0


def test_mass_conserved_slit_with_beads():
    wl = W.charged_slit(nx=16, ny=16, nz=16, n_beads=4)
    wl = wl.replace(R=np.array([[5.2 + 0.97 * i, 7.5, 7.3] for i in range(4)]))
    s = oracle.Sim(wl)
    m0 = s.stats()["mass"]
    assert s.step(30) >= 0
    m1 = s.stats()["mass"]
    assert np.all(np.abs(m1 - m0) <= 1e-13 * m0)


def test_total_momentum_conserved_periodic():
    nx = ny = nz = 12
    q = np.array([-1.0, -1.0, -1.0])
    R = np.array([[4.3 + 0.97 * i, 6.1, 5.7] for i in range(3)])
    n_init = W.ion_densities(np.zeros((nz, ny, nx), np.uint8), 0.01, 1.0, q.sum(), 0.0, 1)
    wl = box(nx, ny, nz, E_app=(2e-3, -1e-3, 5e-4), poisson_tol=1e-14, n_init=n_init,
             flags=W.FLAG_NO_BEAD_NOISE, R=R, V=np.zeros_like(R), charge=q,
             chain=np.zeros(3, np.int32))
    s = oracle.Sim(wl)
    st0 = s.stats()
    p0 = st0["momentum"] + st0["bead_momentum"]
    for _ in range(10):
        assert s.step(1) >= 0
        st = s.stats()
        p = st["momentum"] + st["bead_momentum"]
        assert np.max(np.abs(p - p0)) < 1e-10
    # and something actually moved
    assert np.abs(st["bead_momentum"]).max() > 1e-6


def _poiseuille_error(H, tau, g=1e-6, steps=None):
    nx = ny = 2
    nz = H + 2
    wl = slit(nx, ny, nz, n=(1.0, 1e-3, 1e-3), tau=(tau, tau, tau),
              body_force=((g, 0, 0), (0, 0, 0), (0, 0, 0)))
    s = oracle.Sim(wl)
    nu = KT * (tau - 0.5)
    steps = steps or int(30 * (H + 1) ** 2 / (math.pi ** 2 * nu)) + 50
    s.step(steps)
    F = s.fields()
    x, y, z = node_coords(nx, ny, nz)
    fluid = wl.solid.ravel() == 0
    rho = F["n"].sum(0)
    # physical momentum density: bare current + half the force density
    jx = F["j"][:, 0].sum(0) + 0.5 * F["n"][0] * g
    u = jx / np.where(fluid, rho, 1.0)
    n0 = F["n"][0]
    ref = n0 * g / (2 * np.where(fluid, rho, 1.0) * nu) * (z - 0.5) * (H + 0.5 - z)
    return np.max(np.abs(u[fluid] - ref[fluid])) / np.max(ref[fluid])


def test_poiseuille_exact_at_magic_tau():
    err = _poiseuille_error(8, 0.5 + math.sqrt(3.0 / 16.0))
    assert err < 1e-9


def test_poiseuille_second_order():
    e8 = _poiseuille_error(8, 1.0)
    e16 = _poiseuille_error(16, 1.0)
    assert e8 > 1e-4                        # there is a slip error at tau = 1 ...
    assert 3.5 < e8 / e16 < 4.5             # ... and it falls as 1/H^2


@pytest.mark.parametrize("bary", [False, True])
def test_nernst_einstein_drift(bary):
    E = 1e-3
    D = 0.05
    wl = box(4, 4, 4, n=(1.0, 0.01, 0.01), E_app=(E, 0.0, 0.0), diffusivity=(D, D, D),
             flags=W.FLAG_EQ_BARYCENTRIC if bary else 0)
    s = oracle.Sim(wl)
    s.step(200)
    F = s.fields()
    u = F["j"] / F["n"][:, None, :]
    rho = F["n"].sum(0)
    ubar = (F["j"][:, 0].sum(0)) / rho
    assert np.allclose(ubar, 0, atol=1e-17)
    if not bary:
        # species velocities (half-force shifted = bare at steady state)
        assert np.allclose(u[1, 0], D * E, rtol=1e-10, atol=0)
        assert np.allclose(u[2, 0], -D * E, rtol=1e-10, atol=0)
        assert np.allclose(u[:, 1:], 0, atol=1e-18)
    else:
        # with the barycentric equilibrium the BGK term relaxes u^a towards u too:
        # the drift is set by omega_d + omega_visc, i.e. smaller than D E
        assert 0 < u[1, 0].mean() < D * E


def _pb_newton(H, sigma, lb, N_plus, N_minus, area):
    """1D discrete Poisson-Boltzmann on the fluid layers z = 1..H of a slit
    with wall charge sigma per wall node on both walls (per-area density
    sigma per node cross-section), Neumann walls, fixed ion totals."""
    phi = np.zeros(H)
    src = np.zeros(H)
    src[0] += sigma
    src[-1] += sigma
    for _ in range(200):
        e_p = np.exp(-phi)
        e_m = np.exp(phi)
        cp = N_plus / (area * e_p.sum())
        cm = N_minus / (area * e_m.sum())
        npl = cp * e_p
        nmi = cm * e_m
        L = np.zeros((H, H))
        for i in range(H):
            if i > 0:
                L[i, i - 1] += 1
                L[i, i] -= 1
            if i < H - 1:
                L[i, i + 1] += 1
                L[i, i] -= 1
        Fv = L @ phi + 4 * math.pi * lb * (npl - nmi + src)
        # Jacobian (the normalisation constants' dependence on phi included)
        Jp = -np.diag(npl) + np.outer(npl, e_p) * cp / cp * (1.0 / e_p.sum())
        Jm = np.diag(nmi) - np.outer(nmi, e_m) / e_m.sum()
        J = L + 4 * math.pi * lb * (Jp - Jm)
        dphi = np.linalg.lstsq(J, -Fv, rcond=None)[0]
        dphi -= dphi.mean()
        phi += dphi
        if np.abs(dphi).max() < 1e-15:
            break
    return phi - phi.mean(), npl, nmi


def _boltzmann_errors(H, salt, sigma, steps, lb=0.8):
    nx = ny = 2
    nz = H + 2
    sc = np.zeros((nz, ny, nx))
    sc[0] = sigma
    sc[nz - 1] = sigma
    solid = W.slit_solid(nx, ny, nz)
    n_init = W.ion_densities(solid, salt, 1.0, sc.sum(), 0.0, 1)
    wl = slit(nx, ny, nz, bjerrum=lb, surface_charge=sc, n_init=n_init,
              n=(1.0, salt, salt), poisson_tol=1e-13)
    s = oracle.Sim(wl)
    s.step(steps)
    F = s.fields()
    x, y, z = node_coords(nx, ny, nz)
    col = (x == 0) & (y == 0) & (z >= 1) & (z <= H)
    npl, nmi, phi = F["n"][1][col], F["n"][2][col], F["phi"][col]
    # zero physical flux in equilibrium (bare current + half the field force)
    g = s.node_gradient(F["phi"])
    for a, zv in ((1, 1.0), (2, -1.0)):
        flux = F["j"][a, 2] + 0.5 * F["n"][a] * zv * KT * (-g[2])
        assert np.abs(flux[col]).max() < 1e-9 * salt / 0.002
    # counter-ions pile up at the negative walls
    assert npl[0] > npl[H // 2] and nmi[0] < nmi[H // 2]
    area = nx * ny
    phi_pb, np_pb, nm_pb = _pb_newton(H, sigma, lb, F["n"][1].sum(), F["n"][2].sum(), area)
    err_p = np.max(np.abs(npl / np_pb - 1))
    err_m = np.max(np.abs(nmi / nm_pb - 1))
    err_phi = np.max(np.abs(phi - phi.mean() - phi_pb)) / np.abs(phi_pb).max()
    return np.array([err_p, err_m, err_phi])


def test_boltzmann_equilibrium_charged_wall():
    """Discrete Boltzmann profile within the lattice's O((kappa dx)^2) error,
    and that error falls fourfold when the Debye length is doubled in lattice
    units (salt / 4, wall charge / 2, slit width x 2)."""
    e1 = _boltzmann_errors(24, 0.002, -0.002, 3000)
    kappa2 = 4 * math.pi * 0.8 * 2 * 0.002
    assert np.all(e1 < kappa2 / 12), e1
    e2 = _boltzmann_errors(48, 0.0005, -0.001, 12000)
    assert np.all((e1 / e2 > 3.3) & (e1 / e2 < 4.8)), e1 / e2


def test_electro_osmotic_plug_flow():
    nx = ny = 2
    H = 24
    nz = H + 2
    sigma = -0.002
    lb = 0.8
    salt = 0.002
    E = 1e-3
    tau = 1.0
    sc = np.zeros((nz, ny, nx))
    sc[0] = sigma
    sc[nz - 1] = sigma
    solid = W.slit_solid(nx, ny, nz)
    n_init = W.ion_densities(solid, salt, 1.0, sc.sum(), 0.0, 1)
    wl = slit(nx, ny, nz, bjerrum=lb, surface_charge=sc, n_init=n_init,
              n=(1.0, salt, salt), E_app=(E, 0, 0), poisson_tol=1e-13)
    s = oracle.Sim(wl)
    s.step(6000)
    F = s.fields()
    x, y, z = node_coords(nx, ny, nz)
    col = (x == 0) & (y == 0) & (z >= 1) & (z <= H)
    rho_tot = F["n"][:, col].sum(0)
    # physical velocity: bare current + half the field force on the ions
    zc = np.array([0, 1, -1])
    fx = (zc[:, None] * F["n"][:, col]).sum(0) * KT * E
    u = (F["j"][:, 0][:, col].sum(0) + 0.5 * fx) / rho_tot
    phi = F["phi"][col]
    eta = KT * (tau - 0.5) * rho_tot.mean()
    # wall potential by linear extrapolation to the mid-link wall at z = 1/2
    phi_w = phi[0] - 0.5 * (phi[1] - phi[0])
    ref = KT * E * (phi - phi_w) / (4 * math.pi * lb * eta)
    assert u[H // 2] > 0                       # counter-ions (cations) drag the fluid along +x
    assert abs(u[H // 2] / ref[H // 2] - 1) < 0.03, (u[H // 2], ref[H // 2])

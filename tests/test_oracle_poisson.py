"""Pins of the oracle's Poisson solver (Eq. 3; Sec. II.C red-black SOR).

* a dense solve of an independently assembled fluid-only 7-point Laplacian
  (zero-flux wall faces, periodic wrap) on a small connected geometry;
* a lattice eigenmode: rho = sin(2 pi k x / L) gives
  phi = 4 pi l_B rho / (2 - 2 cos(2 pi k / L)) exactly;
* a charged slit with a uniform neutralising background: the discrete
  solution is the parabola -2 pi l_B rho_bar (z - z_c)^2, which fixes the
  placement of the wall charge on the adjacent fluid nodes;
* the stopping rule and the fixed-iteration mode.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
from helpers import box, slit, node_coords


def _laplacian(solid, periodic):
    nz, ny, nx = solid.shape
    N = solid.size
    fluid = (solid.ravel() == 0)
    A = np.zeros((N, N))
    for i in range(N):
        if not fluid[i]:
            continue
        x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
        for d, (dx, dy, dz) in enumerate([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                          (0, 0, 1), (0, 0, -1)]):
            c = [x + dx, y + dy, z + dz]
            ok = True
            for a, L in enumerate((nx, ny, nz)):
                if periodic[a]:
                    c[a] %= L
                elif not (0 <= c[a] < L):
                    ok = False
            if not ok:
                continue
            j = c[0] + nx * (c[1] + ny * c[2])
            if fluid[j]:
                A[i, j] += 1.0
                A[i, i] -= 1.0
    return A, fluid


def test_dense_solve_small_geometry():
    rng = np.random.default_rng(3)
    nx, ny, nz = 6, 4, 6
    periodic = (1, 1, 0)
    while True:
        solid = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8)
        lab, nlab = ndimage.label(solid == 0)
        if nlab == 1:
            break
    wl = box(nx, ny, nz, periodic=periodic, solid=solid, bjerrum=0.7)
    s = oracle.Sim(wl)
    rho = rng.standard_normal(solid.size) * (solid.ravel() == 0)
    phi, it, res = s.poisson(rho, tol=1e-14, max_iter=200000)
    assert it > 0 and res <= 1e-14
    A, fluid = _laplacian(solid, periodic)
    b = 4 * math.pi * 0.7 * (rho - rho[fluid].mean())
    Af = A[np.ix_(fluid, fluid)]
    ref = np.linalg.lstsq(Af, -b[fluid], rcond=None)[0]
    got = phi[fluid]
    got = got - got.mean()
    ref = ref - ref.mean()
    assert np.max(np.abs(got - ref)) < 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("k", [1, 2, 3])
def test_eigenmode_periodic(k):
    nx, ny, nz = 8, 6, 4
    wl = box(nx, ny, nz, bjerrum=0.8)
    s = oracle.Sim(wl)
    x, y, z = node_coords(nx, ny, nz)
    rho = np.sin(2 * math.pi * k * x / nx)
    phi, it, res = s.poisson(rho, tol=1e-14)
    lam = 2 - 2 * math.cos(2 * math.pi * k / nx)
    ref = 4 * math.pi * 0.8 * rho / lam
    assert np.max(np.abs((phi - phi.mean()) - ref)) < 1e-11 * np.abs(ref).max()


def test_charged_slit_parabola():
    nx, ny, nz = 4, 4, 12
    H = nz - 2
    sigma = -0.03
    sc = np.zeros((nz, ny, nx))
    sc[0] = sigma
    sc[nz - 1] = sigma
    wl = slit(nx, ny, nz, bjerrum=0.8, surface_charge=sc)
    s = oracle.Sim(wl)
    src = s.wall_source()
    x, y, z = node_coords(nx, ny, nz)
    fluid = (wl.solid.ravel() == 0)
    rho_bar = -2 * sigma / H                   # neutralising background
    rho = np.where(fluid, rho_bar, 0.0) + src
    # the wall charge lands on the first fluid layer only
    assert np.allclose(src[fluid & (z == 1)], sigma) and np.allclose(src[fluid & (z == H)], sigma)
    assert np.allclose(src[fluid & (z > 1) & (z < H)], 0)
    phi, it, res = s.poisson(rho, tol=1e-14)
    zc = (H + 1) / 2.0
    ref = -2 * math.pi * 0.8 * rho_bar * (z - zc) ** 2
    d = phi[fluid] - ref[fluid]
    assert np.max(np.abs(d - d.mean())) < 1e-11


def test_stopping_rule_and_fixed_iterations():
    wl = box(8, 8, 8, bjerrum=0.8)
    s = oracle.Sim(wl)
    rng = np.random.default_rng(0)
    rho = rng.standard_normal(512)
    phi, it, res = s.poisson(rho, tol=1e-6, check_every=1)
    assert it > 0 and res <= 1e-6
    phi2, it2, res2 = s.poisson(rho, tol=1e-6, fixed_iter=it - 1)
    assert it2 == it - 1 and res2 > 1e-6       # one sweep fewer is not converged
    phi3, it3, _ = s.poisson(rho, tol=1e-6, check_every=4)
    assert it3 % 4 == 0 and it3 >= it
    _, it0, _ = s.poisson(np.zeros(512), tol=1e-6)
    assert it0 == 0                            # no charge, no sweep


def test_node_gradient_linear_and_ghost():
    nx, ny, nz = 4, 4, 8
    sc = np.zeros((nz, ny, nx))
    sc[0] = 0.02
    wl = slit(nx, ny, nz, bjerrum=0.8, surface_charge=sc)
    s = oracle.Sim(wl)
    x, y, z = node_coords(nx, ny, nz)
    phi = 0.3 * z + 0.0
    g = s.node_gradient(phi)
    fluid = wl.solid.ravel() == 0
    inner = fluid & (z > 1) & (z < nz - 2)
    assert np.allclose(g[2][inner], 0.3, atol=1e-15)
    assert np.allclose(g[0][fluid], 0) and np.allclose(g[1][fluid], 0)
    # z = 1 has the charged wall below: ghost = phi_1 + 4 pi l_B * 0.02
    lo = fluid & (z == 1)
    assert np.allclose(g[2][lo], (phi[lo] + 0.3 - (phi[lo] + 4 * math.pi * 0.8 * 0.02)) / 2)
    hi = fluid & (z == nz - 2)
    assert np.allclose(g[2][hi], (phi[hi] - (phi[hi] - 0.3)) / 2)


def test_residual_function_manufactured_solution():
    """eko_poisson_residual against an independently assembled operator:
    rho = -L phi / (4 pi l_B) makes phi an exact solution; a kick delta at one
    node leaves exactly ||L delta|| / ||b||; phi = 0 leaves ||b|| / ||b|| = 1;
    and the SOR solver's answer meets its own tolerance."""
    rng = np.random.default_rng(11)
    nx, ny, nz = 6, 4, 6
    periodic = (1, 1, 0)
    while True:
        solid = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8)
        lab, nlab = ndimage.label(solid == 0)
        if nlab == 1:
            break
    lb = 0.7
    wl = box(nx, ny, nz, periodic=periodic, solid=solid, bjerrum=lb)
    s = oracle.Sim(wl)
    L, fluid = _laplacian(solid, periodic)
    phi = rng.standard_normal(solid.size) * fluid
    rho = -(L @ phi) / (4 * math.pi * lb)
    assert abs(rho[fluid].sum()) < 1e-12
    assert s.poisson_residual(rho, phi) < 1e-14
    assert s.poisson_residual(rho, np.zeros_like(phi)) == pytest.approx(1.0, rel=1e-14)
    i = int(np.flatnonzero(fluid)[5])
    kick = np.zeros_like(phi)
    kick[i] = 1e-3
    b = -(L @ phi)
    want = np.linalg.norm(L @ kick) / np.linalg.norm(b)
    assert s.poisson_residual(rho, phi + kick) == pytest.approx(want, rel=1e-9)
    sol, it, res = s.poisson(rho, tol=1e-11)
    assert it > 0 and s.poisson_residual(rho, sol) <= 1e-11 * 1.01

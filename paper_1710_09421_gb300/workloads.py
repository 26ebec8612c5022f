"""Seeded synthetic inputs for the electrokinetic LB-MD step.

This module builds the *inputs* of a run -- wall maps, wall surface charge,
initial species densities, polymer chains and the scalar parameters -- for the
workloads the paper describes (a charged slit, a membrane pierced by a
cylindrical pore with a threaded polyelectrolyte, Sec. IV.A) and the sizes the
benchmarks use.  It contains none of the method's arithmetic: no populations,
no forces, no Poisson solve.  Both the CUDA library and the CPU oracle consume
what it produces, each through its own binding.

Conventions shared by every consumer (they are data layout, not arithmetic):

* node id = x + nx * (y + ny * z); arrays are shaped [nz, ny, nx];
* species 0 = solvent, 1 = cation (+1), 2 = anion (-1) (Sec. II.A);
* lattice units: dx = dt = 1, m = 1, v_T^2 = 1/3, k_B T = m v_T^2 = 1/3
  (Sec. II.C); E_app in k_B T / (e dx), surface charge in e per wall node.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

KT = 1.0 / 3.0

# precision codes (same numbers as the C headers of each consumer)
PRECISION = {"f64": 0, "f32": 1, "bf16": 2, "fp16": 3}

# flags (same bits as the C headers of each consumer)
FLAG_EQ_BARYCENTRIC = 1 << 0   # f_eq and S use the barycentric u* (printed reading)
FLAG_GAMMA_LITERAL = 1 << 1    # gamma^alpha = xi for every species (literal Sec. II.B)
FLAG_NO_BEAD_NOISE = 1 << 2    # switch off the Langevin noise on the beads
FLAG_POISSON_GLOBAL = 1 << 3   # CUDA library only: no shared-memory Poisson tiles
FLAG_POISSON_MG = 1 << 4       # CUDA library only: multigrid-preconditioned CG Poisson solver
FLAG_POISSON_MG_SINGLE = 1 << 5  # CUDA library only: the multigrid solve as one cooperative launch (not split)

BOND_FENE = 0
BOND_HARMONIC = 1


@dataclasses.dataclass
class Workload:
    """Everything a run needs; arrays are float64/uint8/int32 numpy arrays."""

    name: str
    nx: int
    ny: int
    nz: int
    periodic: tuple
    solid: np.ndarray                       # uint8 [nz,ny,nx]
    surface_charge: Optional[np.ndarray]    # float64 [nz,ny,nx] or None
    n_init: np.ndarray                      # float64 [3,nz,ny,nx]
    valence: tuple = (0, 1, -1)
    diffusivity: tuple = (0.05, 0.05, 0.05)
    tau: tuple = (1.0, 1.0, 1.0)
    n_ref: tuple = (1.0, 0.01, 0.01)
    body_force: tuple = ((0.0, 0.0, 0.0),) * 3
    bjerrum: float = 0.8
    E_app: tuple = (0.0, 0.0, 0.0)
    poisson_tol: float = 1e-8
    poisson_max_iter: int = 5000
    poisson_check_every: int = 1
    poisson_fixed_iter: int = 0
    rho_jacobi: float = 0.0                 # <= 0: each consumer's default
    precision: str = "f32"
    md_substeps: int = 10
    bead_xi: float = 2.0                    # explicit coupling is stable for xi * w / n < 2
    bead_mass: float = 10.0
    bond_kind: int = BOND_FENE
    bond_k: float = 30.0 * KT               # Kremer-Grest 30 eps / sigma^2 with eps = k_B T
    bond_r0: float = 1.5                    # FENE maximum extension (sigma units)
    bond_l0: float = 0.97                   # harmonic rest length
    wca_eps: float = KT
    wca_sigma: float = 1.0
    wall_eps: float = KT
    wall_sigma: float = 1.0
    seed: int = 2
    bead_kT: float = 1e-3                   # bead thermostat temperature (lattice units)
    flags: int = 0
    fluct_mass: float = 0.0                 # thermal mass of the fluctuating LB term (0 = none)
    R: Optional[np.ndarray] = None          # float64 [nb,3]
    V: Optional[np.ndarray] = None          # float64 [nb,3]
    charge: Optional[np.ndarray] = None     # float64 [nb]
    chain: Optional[np.ndarray] = None      # int32 [nb]

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_beads(self) -> int:
        return 0 if self.R is None else int(self.R.shape[0])

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def slit_solid(nx, ny, nz):
    """Two solid planes at z = 0 and z = nz-1 (a charged slit, as in config 1)."""
    s = np.zeros((nz, ny, nx), np.uint8)
    s[0] = 1
    s[nz - 1] = 1
    return s


def pore_solid(nx, ny, nz, z0, z1, radius):
    """Membrane slab z0 <= z <= z1 pierced by a cylinder along z (Sec. IV.A).

    The pore axis sits at ((nx-1)/2, (ny-1)/2); a membrane node is fluid when
    its squared distance to the axis is below radius^2, which puts exactly
    2*radius nodes across the pore when nx, ny are even.
    """
    s = np.zeros((nz, ny, nx), np.uint8)
    xc, yc = (nx - 1) / 2.0, (ny - 1) / 2.0
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    inside = (x - xc) ** 2 + (y - yc) ** 2 < radius * radius
    for z in range(z0, z1 + 1):
        s[z] = np.where(inside, 0, 1)
    return s


def wall_nodes_touching_fluid(solid, periodic):
    """Boolean map of solid nodes that have at least one fluid face neighbour."""
    nz, ny, nx = solid.shape
    fluid = solid == 0
    touch = np.zeros_like(fluid)
    for axis, per in zip((2, 1, 0), periodic):
        for sh in (1, -1):
            if per:
                nb = np.roll(fluid, sh, axis=axis)
            else:
                nb = np.zeros_like(fluid)
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if sh == 1:
                    dst[axis] = slice(1, None)
                    src[axis] = slice(0, -1)
                else:
                    dst[axis] = slice(0, -1)
                    src[axis] = slice(1, None)
                nb[tuple(dst)] = fluid[tuple(src)]
            touch |= nb
    return (solid == 1) & touch


# ----------------------------------------------------------------------------
# polymer chains
# ----------------------------------------------------------------------------

_OFFS = np.array([(dx, dy, dz) for dz in range(-3, 4) for dy in range(-3, 4) for dx in range(-3, 4)])


def _min_dist_to_solid(p, solid, periodic, reach=3):
    """Distance from p to the nearest wall node (or closed-box outside) within
    `reach` nodes; 1e30 when there is none."""
    nz, ny, nx = solid.shape
    dims = np.array([nx, ny, nz])
    base = np.floor(p).astype(int)
    nodes = base[None, :] + _OFFS
    q = nodes.copy()
    inside = np.ones(len(q), bool)
    for a in range(3):
        if periodic[a]:
            q[:, a] %= dims[a]
        else:
            inside &= (q[:, a] >= 0) & (q[:, a] < dims[a])
    qc = np.clip(q, 0, dims - 1)
    wall = ~inside | (solid[qc[:, 2], qc[:, 1], qc[:, 0]] == 1)
    if not wall.any():
        return 1e30
    return float(np.min(np.linalg.norm(p[None, :] - nodes[wall], axis=1)))


def threaded_chain(n, center, bond, solid, periodic, rng, straight_zone, wall_clear=1.2,
                   bead_clear=1.0):
    """A chain of n beads along z with bead n//2 at `center`.

    Beads are added outward from the centre bead, one bond at a time; each new
    bond direction is the previous one plus a seeded Gaussian kick (small inside
    `straight_zone` = (zlo, zhi), larger outside) and a candidate is rejected
    when it comes within `wall_clear` of a solid node or `bead_clear` of any
    earlier bead.
    """
    dims = (solid.shape[2], solid.shape[1], solid.shape[0])
    R = np.zeros((n, 3))
    mid = n // 2
    R[mid] = center
    placed = [mid]
    for direction, rng_idx in ((+1, range(mid + 1, n)), (-1, range(mid - 1, -1, -1))):
        d = np.array([0.0, 0.0, float(direction)])
        for k in rng_idx:
            prev = R[k - direction]
            for attempt in range(2000):
                zl, zh = straight_zone
                kick = 0.15 if zl - 2 <= prev[2] <= zh + 2 else 0.7
                if attempt > 200:
                    kick *= 1.5
                nd = d + kick * rng.standard_normal(3)
                if attempt > 500:  # crowded: any direction
                    nd = rng.standard_normal(3)
                nd /= np.linalg.norm(nd)
                cand = prev + bond * nd
                w = [cand[a] % dims[a] if periodic[a] else cand[a] for a in range(3)]
                w = np.array(w)
                if any((not periodic[a]) and (w[a] < 1 or w[a] > dims[a] - 2) for a in range(3)):
                    continue
                if _min_dist_to_solid(w, solid, periodic) < wall_clear:
                    continue
                okb = True
                for j in placed:
                    diff = cand - R[j]
                    for a in range(3):
                        if periodic[a]:
                            diff[a] -= dims[a] * round(diff[a] / dims[a])
                    if np.linalg.norm(diff) < bead_clear and abs(j - k) > 1:
                        okb = False
                        break
                if not okb:
                    continue
                R[k] = cand
                d = nd
                placed.append(k)
                break
            else:
                raise RuntimeError("chain generation failed")
    for a in range(3):
        if periodic[a]:
            R[:, a] %= dims[a]
    return R


# ----------------------------------------------------------------------------
# densities
# ----------------------------------------------------------------------------

def random_walk_chain(n, start, bond, solid, periodic, rng, z_min, wall_clear=1.2, bead_clear=1.6):
    """A chain grown from `start` (bead 0, e.g. at a pore mouth) by a seeded
    random walk of fixed bond length (Sec. IV.A: generated in the cis chamber
    starting from the pore entrance): every new bead takes a uniformly random
    direction and is rejected when it falls below z_min, comes within
    `wall_clear` of a wall node or within `bead_clear` of any earlier bead."""
    dims = (solid.shape[2], solid.shape[1], solid.shape[0])
    R = np.zeros((n, 3))
    R[0] = start
    for k in range(1, n):
        for attempt in range(5000):
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            cand = R[k - 1] + bond * d
            if cand[2] < z_min:
                continue
            w = np.array([cand[a] % dims[a] if periodic[a] else cand[a] for a in range(3)])
            if any((not periodic[a]) and (w[a] < 1 or w[a] > dims[a] - 2) for a in range(3)):
                continue
            if _min_dist_to_solid(w, solid, periodic) < wall_clear:
                continue
            diff = cand[None, :] - R[:k]
            for a in range(3):
                if periodic[a]:
                    diff[:, a] -= dims[a] * np.round(diff[:, a] / dims[a])
            if k > 1 and np.min(np.linalg.norm(diff[:-1], axis=1)) < bead_clear:
                continue
            R[k] = cand
            break
        else:
            raise RuntimeError("chain generation failed")
    for a in range(3):
        if periodic[a]:
            R[:, a] %= dims[a]
    return R


def ion_densities(solid, salt, n_solvent, counter_charge, noise, seed):
    """Solvent + 1:1 salt with a uniform counter-ion excess that neutralises
    `counter_charge` (the sum of wall and bead charges); each ion density gets
    seeded U(-noise, noise) perturbations.  Solid nodes carry zero density."""
    fluid = solid == 0
    nf = int(fluid.sum())
    rng = np.random.default_rng(seed)
    n = np.zeros((3,) + solid.shape)
    n[0][fluid] = n_solvent
    excess = -counter_charge / nf          # >0 adds cations, <0 adds anions
    cat = salt + max(excess, 0.0)
    an = salt + max(-excess, 0.0)
    n[1][fluid] = cat
    n[2][fluid] = an
    if noise > 0:
        n[1][fluid] += rng.uniform(-noise, noise, nf)
        n[2][fluid] += rng.uniform(-noise, noise, nf)
    return n


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def charged_slit(nx=32, ny=32, nz=32, wall_charge=-0.01, salt=0.01, n_solvent=1.0,
                 n_beads=8, bead_charge=-1.0, E=(1e-3, 0.0, 0.0), noise=1e-4,
                 precision="f64", seed_init=1, seed_noise=2, tol=1e-10):
    """Plain EK-LB-MD slit: 32^3, periodic x,y, charged walls z = 0, nz-1,
    an 8-bead FENE+WCA chain along x at mid-height (the FP64 parity case)."""
    periodic = (1, 1, 0)
    solid = slit_solid(nx, ny, nz)
    sc = np.zeros(solid.shape)
    sc[solid == 1] = wall_charge
    sc[~wall_nodes_touching_fluid(solid, periodic)] = 0.0
    R = np.array([[12.0 + 0.97 * i, (ny - 1) / 2.0, (nz - 1) / 2.0] for i in range(n_beads)])
    R = R.reshape(-1, 3)
    q = np.full(n_beads, bead_charge)
    total = sc.sum() + q.sum()
    n = ion_densities(solid, salt, n_solvent, total, noise, seed_init)
    return Workload(
        name=f"slit_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, periodic=periodic, solid=solid,
        surface_charge=sc, n_init=n, n_ref=(n_solvent, salt, salt), E_app=tuple(E),
        poisson_tol=tol, precision=precision, seed=seed_noise,
        R=R, V=np.zeros_like(R), charge=q, chain=np.zeros(n_beads, np.int32))


def translocation(nx=64, ny=64, nz=128, membrane=(60, 67), radius=4.0, salt=0.005,
                  n_solvent=1.0, n_beads=32, bead_charge=-1.0, E=(0.0, 0.0, 5e-3),
                  noise=1e-4, precision="f32", seed_init=1, seed_chain=3, seed_noise=2,
                  tol=1e-8, wall_charge=0.0):
    """Membrane slab with a cylindrical pore and a chain threaded halfway through
    it (Sec. IV.A geometry; 64x64x128, pore radius 4, N=32 is the translocation
    benchmark).  Fully periodic box; the applied field drives the ions and the
    chain along z."""
    periodic = (1, 1, 1)
    solid = pore_solid(nx, ny, nz, membrane[0], membrane[1], radius)
    sc = None
    total = 0.0
    if wall_charge != 0.0:
        sc = np.zeros(solid.shape)
        sc[wall_nodes_touching_fluid(solid, periodic)] = wall_charge
        total += sc.sum()
    R = q = None
    if n_beads > 0:
        rng = np.random.default_rng(seed_chain)
        zc = 0.5 * (membrane[0] + membrane[1])
        center = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, zc])
        R = threaded_chain(n_beads, center, 0.97, solid, periodic, rng, membrane)
        q = np.full(n_beads, bead_charge)
        total += q.sum()
    n = ion_densities(solid, salt, n_solvent, total, noise, seed_init)
    return Workload(
        name=f"pore_{nx}x{ny}x{nz}_r{radius:g}_N{n_beads}", nx=nx, ny=ny, nz=nz,
        periodic=periodic, solid=solid, surface_charge=sc, n_init=n,
        n_ref=(n_solvent, salt, salt), E_app=tuple(E), poisson_tol=tol, precision=precision,
        seed=seed_noise, R=R, V=None if R is None else np.zeros_like(R), charge=q,
        chain=None if R is None else np.zeros(n_beads, np.int32))


def paper_pore(nx=64, ny=64, nz=160, membrane=(60, 99), radius=6.0, salt_mM=100.0, n_beads=100,
               bead_charge=-0.1, bjerrum=1.4, E=(0.0, 0.0, 0.05), pore_line_charge=-0.18, dx_nm=0.5,
               precision="f32", seed_init=1, seed_chain=3, seed_noise=2, tol=1e-8):
    """The paper's translocation set-up (Sec. IV.A) in lattice units, dx = 0.5 nm:
    pore diameter 12, membrane 40 thick, chain of 100 beads of charge 0.1 e
    with 1 nm (2 dx) bonds and sigma = 1 nm, Bjerrum length 0.7 nm = 1.4 dx,
    field 0.05 k_B T/(e dx), 1:1 salt (100 or 10 mM: salt_mM * N_A * dx^3 per
    node).  The pore wall carries the paper's -0.36 e per nm of pore length
    (the printed unit "C/nm" read as e/nm): -0.18 e per dx slice, spread
    evenly over the wall nodes lining the pore in that slice.  The chain is a
    random walk in the cis chamber (high z; negative beads drift to -z) from
    the pore entrance; the freely jointed bonds are stiff harmonic springs.
    Fully periodic box."""
    periodic = (1, 1, 1)
    solid = pore_solid(nx, ny, nz, membrane[0], membrane[1], radius)
    # wall nodes lining the pore: wall nodes touching fluid inside the membrane
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    lining = wall_nodes_touching_fluid(solid, periodic) & (z >= membrane[0]) & (z <= membrane[1]) & \
        ((x - cx) ** 2 + (y - cy) ** 2 < (radius + 2.0) ** 2)
    sc = np.zeros(solid.shape)
    for zz in range(membrane[0], membrane[1] + 1):
        sl = lining[zz]
        if sl.any():
            sc[zz][sl] = pore_line_charge / sl.sum()
    salt = salt_mM * 6.02214076e23 * (dx_nm * 1e-9) ** 3
    rng = np.random.default_rng(seed_chain)
    sigma = 2.0
    start = np.array([cx, cy, membrane[1] + 1.5])
    R = random_walk_chain(n_beads, start, 2.0, solid, periodic, rng, z_min=membrane[1] + 1.5,
                          wall_clear=1.2, bead_clear=0.9 * sigma) if n_beads else None
    q = np.full(n_beads, bead_charge) if n_beads else None
    total = sc.sum() + (q.sum() if n_beads else 0.0)
    n = ion_densities(solid, salt, 1.0, total, 0.0, seed_init)
    return Workload(
        name=f"paper_pore_{nx}x{ny}x{nz}_d{2 * radius:g}_{salt_mM:g}mM_N{n_beads}", nx=nx, ny=ny, nz=nz,
        periodic=periodic, solid=solid, surface_charge=sc, n_init=n, n_ref=(1.0, salt, salt),
        E_app=tuple(E), bjerrum=bjerrum, poisson_tol=tol, precision=precision, seed=seed_noise,
        bond_kind=BOND_HARMONIC, bond_k=100.0 * KT / sigma ** 2, bond_l0=2.0, wca_sigma=sigma,
        R=R, V=None if R is None else np.zeros_like(R), charge=q,
        chain=None if R is None else np.zeros(n_beads, np.int32))


def config_slit_fp64():
    """32^3 charged slit, FP64, 200 steps, SOR to 1e-10 (the FP64 parity case)."""
    return charged_slit()


def config_pore_fp32():
    """64x64x128 pore of radius 4, N=32, FP32, SOR to 1e-8 (the timed workload).
    Solver knobs: Chebyshev spectral radius 0.9999 (fastest in a scan of the
    pore: 584 sweeps/step against 1136 at the slowest-box-mode default) and a
    residual test every 4 sweeps."""
    return translocation().replace(rho_jacobi=0.9999, poisson_check_every=4)


def config_learned(precision="f32"):
    """128x128x256 pore of radius 6 (12 nodes across, as in the paper), N = 64,
    salt 0.005, membrane 8 thick centred, E_z = 5e-3: the learned warm-start
    comparison."""
    return translocation(nx=128, ny=128, nz=256, membrane=(124, 131), radius=6.0, salt=0.005,
                         n_beads=64, precision=precision)


def config_precision_sweep(precision="f32"):
    """256x256x512 box, membrane 16 thick centred at z=256, pore radius 8,
    salt 0.01, E_z = 2e-3, N = 128."""
    return translocation(nx=256, ny=256, nz=512, membrane=(248, 263), radius=8.0, salt=0.01,
                         n_beads=128, E=(0.0, 0.0, 2e-3), precision=precision)


def small_pore(nx=40, ny=24, nz=36, membrane=(16, 19), radius=4.0, n_beads=8,
               precision="f32", **kw):
    """A small pore box with ragged extents (x not a multiple of the tile width)."""
    return translocation(nx=nx, ny=ny, nz=nz, membrane=membrane, radius=radius,
                         n_beads=n_beads, precision=precision, **kw)


def replica_set(n_rep=96, seed=1000, sizes_xy=(48, 64, 96), sizes_z=(96, 128, 192),
                radius=(3.0, 8.0), beads=(16, 128), salt=(0.002, 0.02), E_z=5e-3,
                membrane_thickness=8, bead_charge=-0.1, precision="f32"):
    """Independent translocation pores of uneven size: each replica draws its
    box from sizes_xy^2 x sizes_z, a pore radius, a chain length and a salt
    concentration (seeded), with its own seeds; membrane of the given
    thickness centred in z.  Beads carry the paper's 0.1 e (Sec. IV.A): with
    one elementary charge per bead, a long chain in a narrow pore at the low
    end of the salt range drives the ion densities negative within a few
    dozen steps (the stability bound of Sec. III)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_rep):
        L = int(rng.choice(sizes_xy))
        Lz = int(rng.choice(sizes_z))
        R = float(rng.uniform(*radius))
        nb = int(rng.integers(beads[0], beads[1] + 1))
        c0 = float(rng.uniform(*salt))
        zc = Lz // 2
        mem = (zc - membrane_thickness // 2, zc + membrane_thickness // 2 - 1)
        wl = translocation(nx=L, ny=L, nz=Lz, membrane=mem, radius=R, salt=c0, n_beads=nb,
                           bead_charge=bead_charge, E=(0.0, 0.0, E_z), precision=precision, seed_init=seed + r,
                           seed_chain=seed + 5000 + r, seed_noise=seed + 10000 + r)
        wl.name = f"rep{r}_{L}x{L}x{Lz}_r{R:.1f}_N{nb}"
        out.append(wl)
    return out

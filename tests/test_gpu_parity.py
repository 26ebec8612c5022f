"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer work (link bits) must match bit for bit; the FP64 path must match
the oracle to 1e-12 normwise relative on densities, velocities, potential and
bead displacements; the FP32 path to 1e-5 on densities and velocities.
Normwise relative error per field: ||a - b||_2 / ||b||_2.
"""
import numpy as np
import pytest

import oracle
import paper_1710_09421_gb300 as E
from helpers import box, pointwise, rel
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _vel(F):
    n = F["n"]
    return F["j"] / np.where(n > 0, n, 1.0)[:, None, :]


def _compare(wl, steps, tol, precision=None, check_phi=True, check_beads=True, threads=8):
    sim = E.Simulation(wl, precision=precision)
    ref = oracle.Sim(wl, threads=threads)
    R0 = None if wl.R is None else np.array(wl.R, np.float64)
    st_g = sim.step(steps)
    st_o = ref.step(steps)
    assert st_g >= 0 and st_o >= 0, (st_g, st_o)
    G = sim.fields()
    O = ref.fields()
    fluid = wl.solid.ravel() == 0
    errs = {}
    errs["n"] = max(rel(G["n"][a][fluid], O["n"][a][fluid]) for a in range(3))
    ug, uo = _vel(G), _vel(O)
    errs["u"] = max(rel(ug[a][:, fluid], uo[a][:, fluid]) for a in range(3))
    # velocity error of each species against the flow's velocity scale (the
    # largest species velocity norm): a species at rest has no velocity
    # scale of its own, and its drag closure sums nearly cancelling ion
    # momenta, so its per-field relative error is not a precision measure
    scale = max(np.linalg.norm(uo[a][:, fluid]) for a in range(3))
    errs["u_flow"] = max(np.linalg.norm(ug[a][:, fluid] - uo[a][:, fluid]) / scale for a in range(3))
    errs["u_ions"] = max(rel(ug[a][:, fluid], uo[a][:, fluid]) for a in (1, 2))
    if check_phi:
        errs["phi"] = rel(G["phi"][fluid], O["phi"][fluid])
    if check_beads and R0 is not None and len(R0):
        dg = G["R"] - R0
        do = O["R"] - R0
        errs["R"] = rel(dg, do)
    # pointwise: the largest node error against the field's largest value
    # (a single node far off cannot hide in a norm over the lattice)
    errs["n_max"] = max(pointwise(G["n"][a][fluid], O["n"][a][fluid]) for a in range(3))
    errs["u_flow_max"] = max(np.abs(ug[a][:, fluid] - uo[a][:, fluid]).max() for a in range(3)) / max(
        np.abs(uo[a][:, fluid]).max() for a in range(3))
    if check_phi:
        errs["phi_max"] = pointwise(G["phi"][fluid], O["phi"][fluid])
    sg, so = sim.stats(), ref.stats()
    sim.close()
    return errs, sg, so


def test_link_mask_bit_exact():
    rng = np.random.default_rng(11)
    cases = [W.small_pore(n_beads=0), W.charged_slit(nx=20, ny=12, nz=10, n_beads=0)]
    for per in [(1, 1, 1), (0, 1, 0), (0, 0, 0)]:
        solid = (rng.random((10, 12, 14)) < 0.3).astype(np.uint8)
        cases.append(box(14, 12, 10, periodic=per, solid=solid))
    for wl in cases:
        sim = E.Simulation(wl, precision="f64")
        assert np.array_equal(sim.link_mask(), oracle.Sim(wl).link_mask())
        sim.close()


def test_fp64_charged_slit_200_steps():
    """The FP64 parity workload: 32^3 charged slit, 8-bead chain, SOR 1e-10."""
    wl = W.config_slit_fp64()
    errs, sg, so = _compare(wl, 200, TOL64, precision="f64")
    assert all(v < TOL64 for v in errs.values()), errs
    assert sg["poisson_iters"] == so["poisson_iters"]


def test_fp64_small_pore_ragged():
    wl = W.small_pore(precision="f64").replace(poisson_tol=1e-10)
    errs, sg, so = _compare(wl, 60, TOL64, precision="f64")
    assert all(v < TOL64 for v in errs.values()), errs


def test_fp64_closed_box_odd_extent_no_beads():
    solid = np.zeros((6, 8, 7), np.uint8)
    solid[2:4, 3:5, 2:5] = 1
    wl = box(7, 8, 6, periodic=(0, 1, 1), solid=solid, E_app=(1e-3, 2e-3, 0),
             n_init=W.ion_densities(solid, 0.01, 1.0, 0.0, 1e-3, 5), poisson_tol=1e-12)
    errs, _, _ = _compare(wl, 40, TOL64, precision="f64")
    assert all(v < TOL64 for v in errs.values()), errs


# The FP32 tests run the same number of SOR sweeps on both sides: two
# solves stopped independently at a relative residual tol differ in phi by up
# to cond(L) * tol, which is not an FP32 effect.
def test_fp32_small_pore_1000_steps():
    """Ions, solvent and potential without beads: FP32 storage/arithmetic vs FP64."""
    wl = W.small_pore(nx=20, ny=16, nz=24, membrane=(10, 13), radius=3.0, n_beads=0,
                      precision="f32").replace(poisson_fixed_iter=60)
    errs, sg, so = _compare(wl, 1000, TOL32, precision="f32", check_beads=False)
    assert errs["n"] < TOL32 and errs["u_flow"] < TOL32 and errs["u_ions"] < TOL32, errs
    assert errs["phi"] < TOL32, errs
    assert errs["n_max"] < TOL32 and errs["u_flow_max"] < TOL32 and errs["phi_max"] < TOL32, errs


def test_fp32_small_pore_with_chain_1000_steps():
    """With a 4-bead chain (no bead noise) the bead trajectory itself is
    integrated in FP32 forces and velocities; densities and velocities stay
    within the FP32 tolerance after 1000 steps."""
    wl = W.small_pore(nx=20, ny=16, nz=24, membrane=(10, 13), radius=3.0, n_beads=4,
                      precision="f32").replace(poisson_fixed_iter=60, flags=W.FLAG_NO_BEAD_NOISE)
    errs, sg, so = _compare(wl, 1000, TOL32, precision="f32", check_beads=True)
    print(errs)
    assert errs["n"] < TOL32 and errs["u_flow"] < TOL32 and errs["u_ions"] < TOL32, errs
    assert errs["R"] < TOL32, errs
    assert errs["n_max"] < TOL32 and errs["u_flow_max"] < TOL32, errs


def test_fp32_multigrid_small_pore_with_chain_1000_steps():
    """The benchmarked configuration of the solver -- FP32 storage and
    arithmetic, multigrid-CG stopped on its true residual -- over 1000 steps
    against the oracle's Chebyshev SOR.  Both stop on a tolerance (1e-10 on
    the GPU, 1e-13 in the oracle), so their potentials differ by at most
    about cond(A) x 1e-10 ~ 1e-7 relative per step; FP32 rounding must keep
    densities, velocities, potential and bead displacements within 1e-5."""
    wl = W.small_pore(nx=20, ny=16, nz=24, membrane=(10, 13), radius=3.0, n_beads=4,
                      precision="f32").replace(poisson_tol=1e-10, flags=W.FLAG_NO_BEAD_NOISE | W.FLAG_POISSON_MG)
    sim = E.Simulation(wl)
    ref = oracle.Sim(wl.replace(poisson_tol=1e-13, flags=W.FLAG_NO_BEAD_NOISE), threads=8)
    R0 = np.array(wl.R, np.float64)
    for _ in range(10):
        st = sim.step(100)
        assert st >= 0 and not (st & E.EKL_WARN_NOCONV), st
        assert sim.stats()["poisson_res"] <= 1e-10
        assert ref.step(100) >= 0
    G, O = sim.fields(), ref.fields()
    sim.close()
    fluid = wl.solid.ravel() == 0
    ug, uo = _vel(G), _vel(O)
    scale = max(np.linalg.norm(uo[a][:, fluid]) for a in range(3))
    errs = {
        "n": max(rel(G["n"][a][fluid], O["n"][a][fluid]) for a in range(3)),
        "u_flow": max(np.linalg.norm(ug[a][:, fluid] - uo[a][:, fluid]) / scale for a in range(3)),
        "u_ions": max(rel(ug[a][:, fluid], uo[a][:, fluid]) for a in (1, 2)),
        "phi": rel(G["phi"][fluid], O["phi"][fluid]),
        "R": rel(G["R"] - R0, O["R"] - R0),
        "n_max": max(pointwise(G["n"][a][fluid], O["n"][a][fluid]) for a in range(3)),
        "phi_max": pointwise(G["phi"][fluid], O["phi"][fluid]),
    }
    print(errs)
    assert all(v < TOL32 for v in errs.values()), errs


def test_fp32_charged_slit_fixed_point_poisson():
    wl = W.charged_slit(nx=16, ny=16, nz=16, n_beads=4).replace(poisson_fixed_iter=80)
    errs, sg, so = _compare(wl, 100, TOL32, precision="f32", check_beads=False)
    assert errs["n"] < TOL32 and errs["u_flow"] < TOL32 and errs["phi"] < TOL32, errs


def test_fp32_tolerance_stopping_bounded_by_solver_tolerance():
    """With the tolerance-based stop the FP32 path stays within a small
    multiple of the Poisson tolerance effect (reported, loose bound)."""
    wl = W.small_pore(nx=20, ny=16, nz=24, membrane=(10, 13), radius=3.0, n_beads=4,
                      precision="f32").replace(poisson_tol=1e-10)
    errs, sg, so = _compare(wl, 200, TOL32, precision="f32", check_beads=False)
    assert errs["n"] < TOL32 and errs["u_flow"] < 1e-4, errs


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("which", ["small", "bench"])
def test_tiled_poisson_bitwise_equals_global(precision, which):
    """The shared-memory tiled SOR kernel performs the same node updates in
    the same schedule as the global-memory kernel: identical bits."""
    if which == "small":
        wl = W.small_pore(precision=precision)
        steps = 20
    else:
        wl = W.config_pore_fp32().replace(precision=precision, rho_jacobi=0.9999,
                                          poisson_check_every=4)
        steps = 4
    out = []
    for flags in (0, W.FLAG_POISSON_GLOBAL):
        sim = E.Simulation(wl.replace(flags=wl.flags | flags))
        sim.step(steps)
        f, phi, _ = sim.get_state()
        st = sim.stats()
        out.append((f, phi, st["poisson_sweeps"]))
        sim.close()
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][0], out[1][0])


def test_mass_conservation_fp32():
    wl = W.small_pore(precision="f32")
    sim = E.Simulation(wl)
    sim.step(1)
    m0 = sim.stats()["mass"]
    sim.step(200)
    m1 = sim.stats()["mass"]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-5), (m0, m1)
    sim.close()


def test_bitwise_reproducible():
    wl = W.small_pore(precision="f32")
    out = []
    for _ in range(2):
        sim = E.Simulation(wl)
        sim.step(50)
        f, phi, _ = sim.get_state()
        out.append((f, phi, sim.fields(("R",))["R"]))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


def test_state_roundtrip_resume():
    """N + N steps with a checkpoint in between equals 2N steps."""
    wl = W.small_pore(precision="f64")
    a = E.Simulation(wl)
    a.step(20)
    f, phi, st = a.get_state()
    R = a.fields(("R", "V"))
    a.step(20)
    Fa = a.fields()
    b = E.Simulation(wl)
    b.set_state(f, phi, st)
    b.set_beads(R["R"], R["V"], wl.charge, wl.chain)
    b.step(20)
    Fb = b.fields()
    for k in ("n", "j", "phi", "R"):
        assert np.array_equal(Fa[k], Fb[k]), k
    a.close()
    b.close()


def test_full_size_pore_one_step_against_oracle():
    """At the benchmark size (64x64x128, N=32, FP32): run the GPU 30 steps,
    hand its state to the oracle, advance both one step and compare every
    node."""
    wl = W.config_pore_fp32().replace(poisson_fixed_iter=400)
    sim = E.Simulation(wl)
    assert sim.step(30) >= 0
    f, phi, st = sim.get_state()
    B = sim.fields(("R", "V"))
    ref = oracle.Sim(wl, threads=16)
    ref.set_state(f, phi, st)
    ref.set_beads(B["R"], B["V"], wl.charge, wl.chain)
    assert sim.step(1) >= 0
    assert ref.step(1) >= 0
    G, O = sim.fields(), ref.fields()
    fluid = wl.solid.ravel() == 0
    assert max(rel(G["n"][a][fluid], O["n"][a][fluid]) for a in range(3)) < TOL32
    ug, uo = _vel(G), _vel(O)
    scale = max(np.linalg.norm(uo[a][:, fluid]) for a in range(3))
    assert max(np.linalg.norm(ug[a][:, fluid] - uo[a][:, fluid]) / scale for a in range(3)) < TOL32
    assert max(rel(ug[a][:, fluid], uo[a][:, fluid]) for a in (1, 2)) < TOL32
    assert rel(G["phi"][fluid], O["phi"][fluid]) < TOL32
    sim.close()


def test_argument_errors():
    wl = box(7, 8, 6, periodic=(1, 1, 1))   # odd periodic extent
    with pytest.raises(E.EklError) as ei:
        E.Simulation(wl)
    assert ei.value.code == E.EKL_ERR_ARG
    wl = W.small_pore(precision="f32")
    sim = E.Simulation(wl)
    with pytest.raises(E.EklError):
        sim.set_beads(np.array([[-1.0, 2.0, 3.0]]), None, np.array([-1.0]), None)
    sim.close()


def test_bead_inside_wall_reports_error():
    wl = W.small_pore(precision="f32")
    sim = E.Simulation(wl)
    # a bead in the middle of the membrane, far from the pore
    sim.set_beads(np.array([[2.5, 2.5, 17.5]]), None, np.array([-1.0]), None)
    with pytest.raises(E.EklError) as ei:
        sim.step(1)
    assert ei.value.code == E.EKL_ERR_BEAD
    sim.close()

"""Ionic current through a plane (ekl_get_current), the field switch
(ekl_set_field) and the paper's translocation set-up on the GPU."""
import numpy as np
import pytest

import oracle
import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import observables as O
from paper_1710_09421_gb300 import workloads as W
from helpers import rel

pytestmark = pytest.mark.gpu


def _pore():
    return W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=4,
                        precision="f64").replace(poisson_tol=1e-12)


def test_current_and_field_switch_match_oracle_fp64():
    wl = _pore().replace(E_app=(0.0, 0.0, 0.0))
    sim = E.Simulation(wl)
    ref = oracle.Sim(wl, threads=8)
    sim.step(5)
    ref.step(5)
    Ez = np.array([0.0, 0.0, 5e-3])
    sim.set_field(Ez)
    ref.set_field(Ez)
    sim.step(10)
    ref.step(10)
    G, R = sim.fields(), ref.fields()
    fluid = wl.solid.ravel() == 0
    for s in range(3):
        assert rel(G["n"][s][fluid], R["n"][s][fluid]) < 1e-12
    assert rel(G["R"], R["R"]) < 1e-12
    # plane fluxes: the oracle's currents summed over the plane's nodes
    jz = R["j"][:, 2].reshape(3, wl.nz, wl.ny, wl.nx)
    for plane in (2, 9, 15):
        out = sim.current(axis=2, plane=plane)
        want = jz[:, plane].sum(axis=(1, 2))
        scale = np.abs(jz[:, plane]).sum(axis=(1, 2)) + 1e-300
        assert np.all(np.abs(out[:3] - want) <= 1e-12 * scale), (plane, out, want)
        assert abs(out[3] - (want[1] - want[2])) <= 1e-12 * (scale[1] + scale[2])
    sim.close()


def test_current_arguments():
    sim = E.Simulation(_pore())
    with pytest.raises(E.EklError):
        E.ekl_get_current(sim.h, 3, 0)
    with pytest.raises(E.EklError):
        E.ekl_get_current(sim.h, 2, 20)
    sim.close()


def test_paper_pore_relax_then_drive():
    """Sec. IV.A protocol on the paper's set-up (FP32, multigrid): relax at
    zero field, then drive; the run stays stable, the chain keeps its bonds,
    and the ionic current through the pore's mid-plane has the field's sign."""
    wl = W.paper_pore().replace(flags=W.FLAG_POISSON_MG)
    sim = E.Simulation(wl)
    codes = O.relax_then_drive(sim, 100, np.array(wl.E_app), chunk=50)
    codes += [sim.step(200)]
    assert all(c >= 0 for c in codes), codes
    R = sim.fields(("R",))["R"]
    b = np.linalg.norm(np.diff(R, axis=0), axis=1)
    assert np.all(np.abs(b - 2.0) < 0.3), (b.min(), b.max())
    zmid = (60 + 99) // 2
    I = sim.current(axis=2, plane=zmid)
    print("mid-pore fluxes and current", I)
    assert np.isfinite(I).all() and I[3] > 0
    sim.close()


def test_paper_pore_fp64_matches_oracle_across_field_switch():
    """The paper's own set-up (Sec. IV.A) at a size the oracle finishes in
    seconds: a 16 x 16 x 40 box, membrane z = 15..24 pierced by a pore of
    radius 3, the pore lining charged with -0.18 e per lattice slice, six
    beads of -0.1 e on stiff harmonic bonds of 2 dx with WCA sigma = 2 dx,
    Bjerrum length 1.4 dx, 100 mM salt, Chebyshev SOR to 1e-12.  Relaxed at
    zero field for 25 steps, then driven at E_z = 0.05 for 25 more (the
    relax-then-drive protocol): FP64 on the GPU against the oracle within
    1e-12 normwise and pointwise on densities, velocities, potential and
    bead displacements, and the plane current through the pore's mid-plane
    against the oracle's plane sum."""
    from helpers import pointwise

    wl = W.paper_pore(nx=16, ny=16, nz=40, membrane=(15, 24), radius=3.0, n_beads=6,
                      precision="f64", tol=1e-12)
    assert wl.surface_charge is not None and wl.surface_charge.min() < 0
    sim = E.Simulation(wl.replace(E_app=(0.0, 0.0, 0.0)))
    ref = oracle.Sim(wl.replace(E_app=(0.0, 0.0, 0.0)), threads=8)
    R0 = np.array(wl.R)
    assert sim.step(25) >= 0 and ref.step(25) >= 0
    E_drive = np.array(wl.E_app)
    sim.set_field(E_drive)
    ref.set_field(E_drive)
    assert sim.step(25) >= 0 and ref.step(25) >= 0
    G, O_ = sim.fields(), ref.fields()
    fluid = wl.solid.ravel() == 0
    vel = lambda F: F["j"] / np.where(F["n"] > 0, F["n"], 1.0)[:, None, :]
    ug, uo = vel(G), vel(O_)
    errs = {
        "n": max(rel(G["n"][a][fluid], O_["n"][a][fluid]) for a in range(3)),
        "u": max(rel(ug[a][:, fluid], uo[a][:, fluid]) for a in range(3)),
        "phi": rel(G["phi"][fluid], O_["phi"][fluid]),
        "R": rel(G["R"] - R0, O_["R"] - R0),
        "n_max": max(pointwise(G["n"][a][fluid], O_["n"][a][fluid]) for a in range(3)),
        "u_max": max(pointwise(ug[a][:, fluid], uo[a][:, fluid]) for a in range(3)),
        "phi_max": pointwise(G["phi"][fluid], O_["phi"][fluid]),
    }
    print(errs, sim.stats()["poisson_iters"], ref.stats()["poisson_iters"])
    assert all(v < 1e-12 for v in errs.values()), errs
    zmid = (15 + 24) // 2
    jz = O_["j"][:, 2].reshape(3, wl.nz, wl.ny, wl.nx)[:, zmid]
    out = sim.current(axis=2, plane=zmid)
    scale = np.abs(jz).sum(axis=(1, 2)) + 1e-300
    assert np.all(np.abs(out[:3] - jz.sum(axis=(1, 2))) <= 1e-12 * scale), (out, jz.sum(axis=(1, 2)))
    sim.close()

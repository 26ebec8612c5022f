"""Large host transfers through the C ABI.  Arrays of 8 MB and more go through
pinned staging buffers in 64 MB chunks (the upload of the initial densities,
ekl_get_fields, ekl_get_state / ekl_set_state); these lattices are large
enough for several chunks, so a chunk placed at the wrong offset would show.
"""
import numpy as np
import pytest

import oracle
import paper_1710_09421_gb300 as E
from helpers import rel
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_staged_fields_match_the_oracle():
    """64x64x96 pore in FP64 (densities 9.4 MB, currents 28 MB: two and
    more chunks each way): the initial densities go up staged, the fields
    come back staged, and both agree with the FP64 oracle to 1e-12 after two
    steps."""
    wl = W.small_pore(nx=64, ny=64, nz=96, membrane=(44, 51), radius=5.0, n_beads=8,
                      precision="f64").replace(poisson_tol=1e-11)
    assert 3 * wl.n_nodes * 8 >= 8 << 20
    sim = E.Simulation(wl)
    ref = oracle.Sim(wl.replace(poisson_tol=1e-13), threads=16)
    assert sim.step(2) >= 0 and ref.step(2) >= 0
    G, O = sim.fields(), ref.fields()
    sim.close()
    fluid = wl.solid.ravel() == 0
    for a in range(3):
        assert rel(G["n"][a][fluid], O["n"][a][fluid]) < 1e-12, a
    assert rel(G["j"][:, :, fluid].ravel(), O["j"][:, :, fluid].ravel()) < 1e-9
    assert rel(G["phi"][fluid], O["phi"][fluid]) < 1e-9


def test_staged_state_round_trip():
    """128x128x96 FP32 pore (populations 717 MB as FP64: twelve chunks):
    the state read from one handle and written into a fresh one reads back
    identical, and both handles then step to the same fields (to the Poisson
    tolerance's effect: ekl_set_state drops the potential history, so the
    second handle's first solve starts from a different guess)."""
    wl = W.small_pore(nx=128, ny=128, nz=96, membrane=(44, 51), radius=6.0, n_beads=8,
                      precision="f32").replace(flags=W.FLAG_POISSON_MG)
    a = E.Simulation(wl)
    assert a.step(3) >= 0
    f, phi, step = a.get_state()
    beads = a.fields(("R", "V"))
    b = E.Simulation(wl)
    b.set_state(f, phi, step)
    b.set_beads(beads["R"], beads["V"], wl.charge, wl.chain)
    f2, phi2, step2 = b.get_state()
    assert step2 == step
    assert np.array_equal(f, f2) and np.array_equal(phi, phi2)
    assert a.step(2) >= 0 and b.step(2) >= 0
    fa, fb = a.fields(("n", "j", "phi")), b.fields(("n", "j", "phi"))
    a.close()
    b.close()
    fluid = wl.solid.ravel() == 0
    for a_ in range(3):
        assert rel(fb["n"][a_][fluid], fa["n"][a_][fluid]) < 1e-7, a_
    assert rel(fb["phi"][fluid], fa["phi"][fluid]) < 1e-4

"""Reduced-precision population storage (BF16 / FP16 deviations from
w_p n_ref, FP32 arithmetic) against the FP64 oracle.

The error of each storage format is measured per observable (ion densities,
velocities against the flow's velocity scale, potential) after a fixed number
of steps with equal Poisson sweep counts on both sides; the bounds are the
measured errors with a safety factor, so a regression in the conversion or
the deviation form shows up as a failure.
"""
import numpy as np
import pytest

import oracle
import paper_1710_09421_gb300 as E
from helpers import rel
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# storage -> bound on (n, u_flow, phi) normwise errors after 300 steps
BOUNDS = {"f32": (1e-5, 1e-5, 1e-5), "fp16": (2e-4, 2e-3, 1e-3), "bf16": (1e-2, 5e-2, 2e-2)}


def _errors(G, O, fluid):
    u = lambda F: F["j"] / np.where(F["n"] > 0, F["n"], 1.0)[:, None, :]
    ug, uo = u(G), u(O)
    scale = max(np.linalg.norm(uo[a][:, fluid]) for a in range(3))
    return dict(
        n=max(rel(G["n"][a][fluid], O["n"][a][fluid]) for a in range(3)),
        u_flow=max(np.linalg.norm(ug[a][:, fluid] - uo[a][:, fluid]) / scale for a in range(3)),
        phi=rel(G["phi"][fluid], O["phi"][fluid]))


def test_storage_precision_errors():
    wl = W.small_pore(nx=20, ny=16, nz=24, membrane=(10, 13), radius=3.0, n_beads=4,
                      precision="f32").replace(poisson_fixed_iter=60, flags=W.FLAG_NO_BEAD_NOISE)
    ref = oracle.Sim(wl, threads=16)
    assert ref.step(300) >= 0
    O = ref.fields()
    fluid = wl.solid.ravel() == 0
    report = {}
    for prec, bound in BOUNDS.items():
        sim = E.Simulation(wl, precision=prec)
        assert sim.step(300) >= 0
        e = _errors(sim.fields(), O, fluid)
        sim.close()
        report[prec] = e
    print(report)
    for prec, bound in BOUNDS.items():
        e = report[prec]
        assert e["n"] < bound[0] and e["u_flow"] < bound[1] and e["phi"] < bound[2], (prec, report)
    # more bits, smaller error
    assert report["f32"]["n"] < report["fp16"]["n"] < report["bf16"]["n"]
    print(report)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_reduced_storage_conserves_mass(prec):
    """Mass per species is conserved up to the storage rounding of the
    deviations (relative to the total, far below the format's epsilon)."""
    wl = W.small_pore(precision=prec)
    sim = E.Simulation(wl)
    sim.step(1)
    m0 = sim.stats()["mass"]
    sim.step(200)
    m1 = sim.stats()["mass"]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-3), (m0, m1)
    sim.close()

"""Learned warm start in the step: trained on crops the solver itself
generates, it leaves the solve's residual bound unchanged (the iteration
still runs to poisson_tol) and the test reports the sweeps it saves."""
import numpy as np
import pytest

import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import warmstart as WS
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_warmstart_collect_train_and_gain():
    wl = W.small_pore(nx=32, ny=32, nz=48, membrane=(22, 25), radius=4.0, n_beads=8,
                      precision="f32").replace(poisson_tol=1e-8, poisson_check_every=2)
    sim = E.Simulation(wl)
    sim.step(20)
    crops = sim.collect(120, crop=16, ncrops=8, seed=1)
    sim.close()
    assert crops.shape == (960, 3, 16, 16, 16) and np.isfinite(crops).all()
    assert np.abs(crops[:, 2]).max() > 0
    w, scales, curve = WS.train(crops, iters=300, batch=8, lr=2e-3, seed=0)
    assert curve[-20:].mean() < 0.7 * curve[:20].mean(), (curve[:5], curve[-5:])

    def make():
        s = E.Simulation(wl)
        s.step(20)
        return s

    res = WS.compare(make, w, scales, 60)
    print(res)
    for k in ("plain", "learned"):
        assert res[k]["residual"] <= 1e-8
    # the network may or may not pay for itself on a small box; it must not
    # make the iteration diverge
    assert res["learned"]["sweeps_per_step"] < 2 * res["plain"]["sweeps_per_step"]


def _restrict(field, fluid, L, how):
    """Per cube of 2^L nodes: sum (how='sum') or mean over its fluid nodes."""
    nz, ny, nx = field.shape
    b = 2 ** L
    f = (field * fluid).reshape(nz // b, b, ny // b, b, nx // b, b).sum(axis=(1, 3, 5))
    if how == "sum":
        return f
    c = fluid.reshape(nz // b, b, ny // b, b, nx // b, b).sum(axis=(1, 3, 5))
    return np.where(c > 0, f / np.maximum(c, 1), 0.0)


def test_coarse_level_samples_match_oracle_fields():
    """At network level 2 the library records, per step, the whole grid of
    4^3-node cells: the change of the Poisson source summed over each cell,
    and phi(t-1) and phi(t) - phi(t-1) averaged over the cell's fluid nodes.
    Against the same quantities formed in numpy from the FP64 oracle's own
    charge density and potential (b = 4 pi l_B (rho - mean over fluid)):
    within the FP32 rounding of the recorded values (potentials compared up
    to their mean, the gauge of a periodic box)."""
    import oracle

    wl = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=4,
                      precision="f64").replace(poisson_tol=1e-12)
    sim = E.Simulation(wl)
    ref = oracle.Sim(wl, threads=8)
    sim.step(3)
    ref.step(3)
    sim.warmstart_level(2)
    samples = sim.collect(4, seed=0)
    sim.close()
    assert samples.shape == (4, 3, 5, 4, 4)
    shape = (wl.nz, wl.ny, wl.nx)
    fluid = (wl.solid == 0).astype(np.float64)
    c4 = 4 * np.pi * wl.bjerrum
    bprev = None
    phiprev = ref.fields()["phi"].reshape(shape)
    for k in range(4):
        assert ref.step(1) >= 0
        rho = ref.last_rho().reshape(shape)
        b = c4 * (rho - rho[fluid > 0].mean()) * fluid
        phi = ref.fields()["phi"].reshape(shape)
        if k > 0:   # the first recorded step has no previous source
            want_db = _restrict(b - bprev, fluid, 2, "sum")
            got = samples[k, 0]
            assert np.abs(got - want_db).max() <= 1e-5 * np.abs(want_db).max(), k
        cells = _restrict(np.ones(shape), fluid, 2, "sum") > 0   # cells holding fluid
        for ch, want in ((1, _restrict(phiprev, fluid, 2, "mean")), (2, _restrict(phi - phiprev, fluid, 2, "mean"))):
            got = samples[k, ch].astype(np.float64)
            assert np.all(got[~cells] == 0)
            got, want = got[cells] - got[cells].mean(), want[cells] - want[cells].mean()
            assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max() + 1e-12, (k, ch)
        bprev, phiprev = b, phi


def test_coarse_level_warmstart_trains_and_keeps_the_residual():
    """Network on 4^3-node cells of a periodic pore: trained on whole coarse
    grids the solver records (another seed), installed at the same level; the
    solve still meets its tolerance every step and the trajectory stays with
    the plain run's within the solver tolerance's effect."""
    wl = W.small_pore(nx=32, ny=32, nz=48, membrane=(22, 25), radius=4.0, n_beads=8,
                      precision="f32").replace(poisson_tol=1e-8, flags=W.FLAG_POISSON_MG)
    src = E.Simulation(wl.replace(seed=wl.seed + 7))
    src.step(5)
    src.warmstart_level(2)
    data = src.collect(201, seed=1)[1:]
    src.close()
    assert data.shape == (200, 3, 12, 8, 8) and np.isfinite(data).all()
    w, scales, curve = WS.train_fields(data, wl.periodic, iters=300, batch=8, lr=2e-3, seed=0)
    assert curve[-20:].mean() < 0.7 * curve[:20].mean(), (curve[:5], curve[-5:])
    runs = []
    for use in (False, True):
        sim = E.Simulation(wl)
        sim.step(5)
        if use:
            sim.set_warmstart(w, scales, level=2)
        for _ in range(20):
            rc = sim.step(1)
            assert rc >= 0 and not (rc & E.EKL_WARN_NOCONV), rc
            assert sim.stats()["poisson_res"] <= 1e-8
        runs.append(sim.fields(("n", "phi")))
        sim.close()
    fl = wl.solid.ravel() == 0
    dphi = np.linalg.norm(runs[0]["phi"][fl] - runs[1]["phi"][fl]) / np.linalg.norm(runs[1]["phi"][fl])
    dn = max(np.linalg.norm(runs[0]["n"][a][fl] - runs[1]["n"][a][fl]) / np.linalg.norm(runs[1]["n"][a][fl])
             for a in range(3))
    assert dphi < 1e-5 and dn < 1e-6, (dphi, dn)

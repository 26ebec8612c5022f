"""Batched replicas: every replica of a batch evolves exactly as the same
workload run on its own handle (equal sweep counts), and a tolerance-based
batch converges each replica to its own tolerance."""
import numpy as np
import pytest

import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _uneven(fixed):
    wls = [W.small_pore(nx=20, ny=16, nz=24, membrane=(10, 13), radius=3.0, n_beads=4),
           W.small_pore(nx=24, ny=20, nz=28, membrane=(12, 15), radius=4.0, n_beads=6, seed_noise=7),
           W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=0, seed_init=9)]
    return [w.replace(poisson_fixed_iter=fixed) for w in wls]


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_replicas_bitwise_equal_single_runs(precision):
    wls = _uneven(40)
    batch = E.Batch(wls, precision=precision)
    assert batch.step(15) >= 0
    for r, wl in enumerate(wls):
        sim = E.Simulation(wl, precision=precision)
        sim.step(15)
        a, b = sim.get_state(), batch.reps[r].get_state()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), r
        fa, fb = sim.fields(("R", "V")), batch.reps[r].fields(("R", "V"))
        assert np.array_equal(fa["R"], fb["R"]), r
        sim.close()
    batch.close()


def test_batch_tolerance_and_autotune():
    # every replica carries a charged chain (a bead-free replica's source is
    # only the ion noise; its relative residual floors near 1e-8 in the 2^-40
    # fixed-point potential)
    wls = [w.replace(poisson_tol=1e-8) for w in _uneven(0)]
    wls[2] = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=3,
                          seed_init=9).replace(poisson_tol=1e-8)
    batch = E.Batch(wls)
    choice = batch.autotune(1)
    assert 0 <= choice < 4
    assert batch.step(5) >= 0
    for r in range(len(wls)):
        st = batch.reps[r].stats()
        assert st["poisson_res"] <= 1e-8 and st["poisson_iters"] > 0
    # one launch per phase per step for the whole batch (5 phases), plus the
    # charge totals
    l0 = batch.launches()
    batch.step(3)
    assert batch.launches() - l0 == 3 * 6
    batch.close()


def test_batch_multigrid_replicas():
    """Batched multigrid: each replica solves on its own blocks with its own
    barrier and converges on its own.  Every replica meets its tolerance; its
    FP64 potential meets it under the oracle's operator and source too; and it
    agrees with a single-handle multigrid run (whose coarsest level is solved
    exactly instead of smoothed) within the bound two tolerance-converged
    solves allow."""
    import oracle
    from helpers import rel

    tol = 1e-10
    wls = _uneven(0)
    wls[2] = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=3, seed_init=9)
    wls = [w.replace(poisson_tol=tol, flags=W.FLAG_POISSON_MG, precision="f64") for w in wls]
    batch = E.Batch(wls, precision="f64")
    assert batch.step(1) >= 0
    for r, wl in enumerate(wls):
        ref = oracle.Sim(wl.replace(poisson_tol=1e-13), threads=8)
        assert ref.step(1) >= 0
        _, phi, _ = batch.reps[r].get_state()
        assert ref.poisson_residual(ref.last_rho(), phi) <= tol * 1.001, r
    tot0 = [batch.reps[r].stats()["poisson_sweeps"] for r in range(len(wls))]
    l0 = batch.launches()
    assert batch.step(9) >= 0
    # per step: bin, charge, charge totals, MD, LB and the split solve's six
    # host launches; the loop's 15 kernels once per iteration, an iteration
    # running while any replica is still iterating
    extra = batch.launches() - l0 - 9 * 11
    its = [batch.reps[r].stats()["poisson_sweeps"] - tot0[r] for r in range(len(wls))]
    assert extra % 15 == 0 and max(its) <= extra // 15 <= sum(its), (extra, its)
    for r, wl in enumerate(wls):
        st = batch.reps[r].stats()
        assert st["poisson_res"] <= tol and st["poisson_iters"] > 0, (r, st)
        sim = E.Simulation(wl, precision="f64")
        sim.step(10)
        a, b = sim.fields(), batch.reps[r].fields()
        fluid = wl.solid.ravel() == 0
        assert max(rel(b["n"][s][fluid], a["n"][s][fluid]) for s in range(3)) < 1e-10, r
        assert rel(b["phi"][fluid], a["phi"][fluid]) < 1e-7, r
        sim.close()
    batch.close()


def test_batch_replica_field_change_matches_single_run():
    """A field switched on one replica between batch steps (the relax-then-drive
    protocol) acts from the next step, exactly as on a handle of its own."""
    wls = _uneven(40)[:2]
    drive = (0.0, 0.0, 0.02)
    batch = E.Batch(wls, precision="f32")
    assert batch.step(5) >= 0
    batch.reps[1].set_field(drive)
    assert batch.step(5) >= 0
    for r, wl in enumerate(wls):
        sim = E.Simulation(wl, precision="f32")
        sim.step(5)
        if r == 1:
            sim.set_field(drive)
        sim.step(5)
        a, b = sim.get_state(), batch.reps[r].get_state()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), r
        sim.close()
    batch.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_split_solve_equals_cooperative(precision):
    """The batched multigrid solve split into per-pass launches over all
    replicas (the default) and the single cooperative launch return the same
    states bit for bit, with the same iteration counts, on replicas of three
    sizes that converge after different numbers of iterations."""
    wls = _uneven(0)
    wls[2] = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=3, seed_init=9)
    wls = [w.replace(poisson_tol=1e-8, flags=W.FLAG_POISSON_MG, precision=precision) for w in wls]
    coop = [w.replace(flags=W.FLAG_POISSON_MG | W.FLAG_POISSON_MG_SINGLE) for w in wls]
    a, b = E.Batch(wls, precision=precision), E.Batch(coop, precision=precision)
    a.set_schedule(2)  # blocks shared by fluid nodes; lattice passes on the coarse launch's blocks
    b.set_schedule(2)
    iters = [[], []]
    for _ in range(4):
        assert a.step(2) >= 0 and b.step(2) >= 0
        for k, bt in enumerate((a, b)):
            iters[k].append([bt.reps[r].stats()["poisson_iters"] for r in range(len(wls))])
    assert iters[0] == iters[1]
    assert len({tuple(x) for x in iters[0]}) > 0 and any(len(set(x)) > 1 for x in iters[0]), iters[0]
    for r in range(len(wls)):
        sa, sb = a.reps[r].get_state(), b.reps[r].get_state()
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]), r
        fa, fb = a.reps[r].fields(("R",)), b.reps[r].fields(("R",))
        assert np.array_equal(fa["R"], fb["R"]), r
    a.close()
    b.close()


def test_batch_split_solve_on_finer_blocks():
    """The split batch solve with its lattice passes on four times the blocks
    of the coarse launch (schedule bit 0) sums its block partials in another
    order: in FP64 at tolerance 1e-10 its states agree with the cooperative
    form to the solve's tolerance.  The cooperative form has no such
    schedule."""
    from helpers import rel

    wls = _uneven(0)
    wls[2] = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=3, seed_init=9)
    wls = [w.replace(poisson_tol=1e-10, flags=W.FLAG_POISSON_MG, precision="f64") for w in wls]
    coop = [w.replace(flags=W.FLAG_POISSON_MG | W.FLAG_POISSON_MG_SINGLE) for w in wls]
    a, b = E.Batch(wls, precision="f64"), E.Batch(coop, precision="f64")
    a.set_schedule(3)
    with pytest.raises(E.EklError):
        b.set_schedule(3)
    assert a.step(6) >= 0 and b.step(6) >= 0
    for r, wl in enumerate(wls):
        sa, sb = a.reps[r].stats(), b.reps[r].stats()
        assert sa["poisson_res"] <= 1e-10 and abs(sa["poisson_iters"] - sb["poisson_iters"]) <= 1, (r, sa, sb)
        fa, fb = a.reps[r].fields(), b.reps[r].fields()
        fluid = wl.solid.ravel() == 0
        assert max(rel(fa["n"][s][fluid], fb["n"][s][fluid]) for s in range(3)) < 1e-10, r
        assert rel(fa["phi"][fluid], fb["phi"][fluid]) < 1e-7, r
    a.close()
    b.close()

"""The paper's translocation set-up as a workload (Sec. IV.A) and the
random-walk chain generator: host-side input construction only."""
import numpy as np

from paper_1710_09421_gb300 import observables as O
from paper_1710_09421_gb300 import workloads as W


def test_paper_pore_inputs():
    wl = W.paper_pore()
    R, solid = wl.R, wl.solid
    assert wl.n_beads == 100 and np.allclose(wl.charge, -0.1)
    # chain: bead 0 at the pore mouth on the cis side, 2 dx bonds, all in the cis chamber
    assert np.allclose(R[0], [31.5, 31.5, 100.5])
    b = np.linalg.norm(np.diff(R, axis=0), axis=1)
    assert np.allclose(b, 2.0, atol=1e-9)
    assert R[:, 2].min() >= 100.5 - 1e-9
    d = np.linalg.norm(R[:, None, :] - R[None, :, :], axis=2)
    np.fill_diagonal(d, 1e9)
    assert d.min() >= 1.8 - 1e-9
    # pore wall charge: -0.18 e per dx slice of the 40-dx membrane
    per_slice = wl.surface_charge.sum(axis=(1, 2))
    assert np.allclose(per_slice[60:100], -0.18) and abs(per_slice.sum() + 7.2) < 1e-12
    assert np.all(solid.ravel()[wl.surface_charge.ravel() != 0] == 1)
    # 100 mM at dx = 0.5 nm, overall neutral
    assert abs(wl.n_ref[1] - 100 * 6.02214076e23 * 0.5e-9 ** 3) < 1e-15
    fl = solid == 0
    net = (wl.n_init[1] - wl.n_init[2])[fl].sum() + wl.surface_charge.sum() + wl.charge.sum()
    assert abs(net) < 1e-9
    assert wl.bjerrum == 1.4 and wl.E_app == (0.0, 0.0, 0.05)


def test_observable_helpers():
    z = np.array([[5.0, 6.0], [4.0, 6.0], [2.0, 4.5], [1.0, 3.0]])
    assert list(O.crossing_times(z, 4.5)) == [1, 3]
    assert O.conductance(2.0, 0.5, 8) == 0.5
    assert abs(O.g0(40) - 3 ** 0.5 / 40) < 1e-15


def test_benchmark_workload_geometries():
    """The timed, precision-sweep and learned-warm-start pores have the sizes
    the benchmarks name: box, membrane slab, pore radius, chain length, salt,
    neutrality, and the chain threaded through the pore."""
    cases = [(W.config_pore_fp32(), (64, 64, 128), (60, 67), 4.0, 32, 0.005),
             (W.config_learned(), (128, 128, 256), (124, 131), 6.0, 64, 0.005),
             (W.config_precision_sweep(), (256, 256, 512), (248, 263), 8.0, 128, 0.01)]
    for wl, dims, (z0, z1), radius, nb, salt in cases:
        assert (wl.nx, wl.ny, wl.nz) == dims and wl.n_beads == nb
        solid = wl.solid
        # membrane: every node of the slab outside the pore is solid, none outside the slab
        z = np.arange(wl.nz)
        slab = (z >= z0) & (z <= z1)
        assert not solid[~slab].any()
        cx, cy = (wl.nx - 1) / 2.0, (wl.ny - 1) / 2.0
        yy, xx = np.meshgrid(np.arange(wl.ny), np.arange(wl.nx), indexing="ij")
        r = np.hypot(xx - cx, yy - cy)
        for k in (z0, (z0 + z1) // 2, z1):
            open_ = solid[k] == 0
            assert open_.any() and r[open_].max() <= radius + 1e-9
            assert np.all(solid[k][r > radius + 1.5])
        # salt, and neutrality up to the seeded U(-1e-4, 1e-4) density noise
        # (the counter-ions compensate the chain; six standard deviations)
        assert abs(wl.n_ref[2] - salt) < 1e-12
        fl = solid == 0
        net = (wl.n_init[1] - wl.n_init[2])[fl].sum() + wl.charge.sum()
        if wl.surface_charge is not None:
            net += wl.surface_charge.sum()
        assert abs(net) < 6 * 1e-4 * np.sqrt(2 * fl.sum() / 3), net
        # some bead inside the pore, every bead in fluid
        R = wl.R
        assert np.any((R[:, 2] >= z0) & (R[:, 2] <= z1 + 1))
        idx = np.floor(R).astype(int)
        assert not solid[idx[:, 2] % wl.nz, idx[:, 1] % wl.ny, idx[:, 0] % wl.nx].any()

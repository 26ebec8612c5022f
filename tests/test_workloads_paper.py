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

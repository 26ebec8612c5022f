"""Pins of the oracle's lattice table, link bits and random numbers.

D3Q19 (Sec. II.C): the weights must reproduce the isotropic Gaussian moments
up to fourth order with v_T^2 = 1/3; the link bits are recomputed by brute
force with numpy shifts; Philox-4x32-10 is checked against the published
known-answer vectors (tests/golden/philox4x32_10_kat.txt).
"""
import itertools
import os

import numpy as np

import oracle
from helpers import box
from paper_1710_09421_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def test_d3q19_isotropy():
    c, w, opp = oracle.lattice()
    c = c.astype(np.float64)
    assert len(w) == 19 and len({tuple(v) for v in c.astype(int)}) == 19
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("p,pa->a", w, c), 0, atol=1e-16)
    d = np.eye(3)
    assert np.allclose(np.einsum("p,pa,pb->ab", w, c, c), d / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("p,pa,pb,pc->abc", w, c, c, c), 0, atol=1e-16)
    m4 = np.einsum("p,pa,pb,pc,pd->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-16)
    assert np.all(c[opp] == -c)
    norms = (c ** 2).sum(1)
    assert sorted(norms.tolist()) == [0] + [1] * 6 + [2] * 12


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert list(oracle.philox4x32_10(v[:4], v[4:6])) == v[6:]
        n += 1
    assert n == 3


def _brute_mask(wl):
    """Link bits recomputed with array shifts: bit p set when x - c_p is wall
    or lies beyond a closed face; bit 31 on wall nodes."""
    c, _, _ = oracle.lattice()
    solid = wl.solid.astype(bool)
    nz, ny, nx = solid.shape
    mask = np.zeros(solid.shape, np.uint32)
    for p in range(1, 19):
        # neighbour x - c_p: pad closed axes with wall
        pad = [(1, 1) if not wl.periodic[ax] else (0, 0) for ax in (2, 1, 0)]
        s = np.pad(solid, pad, constant_values=True)
        for ax_np, ax in ((2, 0), (1, 1), (0, 2)):
            s = np.roll(s, c[p][ax], axis=ax_np)
        sl = tuple(slice(1, -1) if not wl.periodic[ax] else slice(None) for ax in (2, 1, 0))
        nb_solid = s[sl]
        mask |= np.where(nb_solid, np.uint32(1 << p), np.uint32(0))
    mask = np.where(solid, np.uint32(1 << 31), mask)
    return mask.ravel()


def test_link_mask_brute_force():
    rng = np.random.default_rng(7)
    for periodic in itertools.product((0, 1), repeat=3):
        dims = (6, 4, 8)
        solid = (rng.random(dims[::-1]) < 0.25).astype(np.uint8)
        wl = box(*dims, periodic=periodic, solid=solid)
        s = oracle.Sim(wl)
        assert np.array_equal(s.link_mask(), _brute_mask(wl)), periodic


def test_pore_geometry_counts():
    wl = W.translocation(nx=64, ny=64, nz=128, n_beads=0)
    # 8 nodes across the pore on the axis row, 2*radius as the workload states
    row = wl.solid[63, 31, :]
    assert int((row == 0).sum()) == 8
    assert wl.solid[60:68].sum() > 0 and wl.solid[:60].sum() == 0

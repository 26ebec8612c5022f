"""Pins of the oracle's fluctuating collision term (Eq. 14).

* the moment basis is orthonormal in sum_p w_p chi_kp chi_lp, complete, and
  its first four vectors span the conserved moments {1, c} (so the noise on
  k = 4..18 leaves mass and momentum untouched);
* mass per species and total momentum are conserved to round-off with the
  noise on;
* fluctuation-dissipation: in a periodic box at rest the stationary
  populations satisfy <df_p df_q> = m n w_p delta_pq (the noise amplitude
  sqrt(m n omega (2 - omega)) exactly balances the BGK damping of every
  non-conserved moment), hence Var(n) = m n and Var(j_x) = m n v_T^2 = m n / 3
  per node, at two relaxation times.
"""
import numpy as np
import pytest

import oracle
from helpers import box


def test_basis_orthonormal_and_conserved_span():
    chi = oracle.basis()
    c, w, _ = oracle.lattice()
    c = np.asarray(c, float).reshape(19, 3)
    w = np.asarray(w, float)
    G = chi @ np.diag(w) @ chi.T
    assert np.allclose(G, np.eye(19), atol=1e-13)
    # completeness: sum_k chi_kp chi_kq = delta_pq / w_p
    assert np.allclose(chi.T @ chi, np.diag(1.0 / w), atol=1e-12)
    cons = np.vstack([np.ones(19), c.T])                # 1, cx, cy, cz
    proj = chi[:4].T @ (chi[:4] @ np.diag(w) @ cons.T)  # projection onto span(chi_0..3)
    assert np.allclose(proj, cons.T, atol=1e-13)


def _fluct_box(tau, m, seed=5):
    n = (1.0, 1.0, 1.0)
    wl = box(8, 8, 8, periodic=(1, 1, 1), n=n, bjerrum=0.0, tau=(tau, tau, tau),
             diffusivity=(1e6, 1e6, 1e6), fluct_mass=m, seed=seed)
    return wl


def test_fluctuations_conserve_mass_and_momentum():
    s = oracle.Sim(_fluct_box(1.0, 1e-3), threads=4)
    s.step(1)
    F0 = s.fields()
    s.step(50)
    F1 = s.fields()
    for a in range(3):
        assert abs(F1["n"][a].sum() / F0["n"][a].sum() - 1) < 1e-13
    p0 = F0["j"].sum(axis=(0, 2))
    p1 = F1["j"].sum(axis=(0, 2))
    assert np.all(np.abs(p1 - p0) < 1e-11), (p0, p1)
    assert np.abs(F1["n"] - 1.0).max() > 1e-3   # the noise is there


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_fluctuation_dissipation(tau):
    m = 1e-3
    s = oracle.Sim(_fluct_box(tau, m), threads=4)
    s.step(400)
    vn, vj = [], []
    for _ in range(150):
        s.step(5)
        F = s.fields()
        vn.append(F["n"].var(axis=1))                 # per species, over nodes
        vj.append(F["j"][:, 0].var(axis=1))
    vn = np.mean(vn, axis=0)
    vj = np.mean(vj, axis=0)
    assert np.allclose(vn, m * 1.0, rtol=0.08), vn
    assert np.allclose(vj, m * 1.0 / 3.0, rtol=0.08), vj

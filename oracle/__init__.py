"""ORACLE -- test infrastructure only.

Python binding of the plain FP64 CPU oracle in ``ekl_oracle.c``.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this module; the CUDA library and its Python binding never do.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ekl_oracle.c")
_LIB = os.path.join(_HERE, "libekl_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
NS = 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", _SRC,
            "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("periodic", C.c_int32 * 3),
        ("valence", C.c_int32 * 3),
        ("diffusivity", C.c_double * 3),
        ("tau", C.c_double * 3),
        ("n_ref", C.c_double * 3),
        ("body_force", (C.c_double * 3) * 3),
        ("bjerrum", C.c_double),
        ("E_app", C.c_double * 3),
        ("poisson_tol", C.c_double),
        ("poisson_max_iter", C.c_int32),
        ("poisson_check_every", C.c_int32),
        ("poisson_fixed_iter", C.c_int32),
        ("rho_jacobi", C.c_double),
        ("md_substeps", C.c_int32),
        ("bead_xi", C.c_double),
        ("bead_mass", C.c_double),
        ("bond_kind", C.c_int32),
        ("bond_k", C.c_double), ("bond_r0", C.c_double), ("bond_l0", C.c_double),
        ("wca_eps", C.c_double), ("wca_sigma", C.c_double),
        ("wall_eps", C.c_double), ("wall_sigma", C.c_double),
        ("seed", C.c_uint64),
        ("bead_kT", C.c_double),
        ("flags", C.c_int32),
        ("fluct_mass", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.eko_create.restype = vp
            L.eko_create.argtypes = [C.POINTER(Params), vp, vp, vp, C.POINTER(C.c_int)]
            L.eko_destroy.argtypes = [vp]
            L.eko_set_threads.argtypes = [vp, C.c_int]
            L.eko_set_beads.argtypes = [vp, C.c_int, vp, vp, vp, vp]
            L.eko_step.argtypes = [vp, C.c_int]
            L.eko_step.restype = C.c_int
            L.eko_get_fields.argtypes = [vp, vp, vp, vp, vp, vp]
            L.eko_get_state.argtypes = [vp, vp, vp, C.POINTER(C.c_int64)]
            L.eko_set_state.argtypes = [vp, vp, vp, C.c_int64]
            L.eko_get_stats.argtypes = [vp, dp]
            L.eko_link_mask.argtypes = [vp, vp]
            L.eko_wall_source.argtypes = [vp, vp]
            L.eko_lattice.argtypes = [vp, vp, vp]
            L.eko_poisson_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.c_int, C.c_int,
                                            dp]
            L.eko_poisson_solve.restype = C.c_int
            L.eko_node_gradient.argtypes = [vp, vp, vp]
            L.eko_poisson_residual.argtypes = [vp, vp, vp]
            L.eko_poisson_residual.restype = C.c_double
            L.eko_last_rho.argtypes = [vp, vp]
            L.eko_basis.argtypes = [vp]
            L.eko_set_field.argtypes = [vp, vp]
            L.eko_bead_stencil.argtypes = [vp, vp, vp, vp]
            L.eko_bead_stencil.restype = C.c_int
            L.eko_philox4x32_10.argtypes = [vp, vp, vp]
            L.eko_default_rho_jacobi.argtypes = [vp]
            L.eko_default_rho_jacobi.restype = C.c_double
            L.eko_sizeof_params.restype = C.c_int64
            assert L.eko_sizeof_params() == C.sizeof(Params), "oracle params layout mismatch"
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lattice():
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    lib().eko_lattice(_ptr(c), _ptr(w), _ptr(opp))
    return c, w, opp


def basis():
    """Moment basis of the fluctuating term, chi[k][p] (Eq. 14)."""
    out = np.zeros((19, 19))
    lib().eko_basis(_ptr(out))
    return out


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().eko_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def _params(wl) -> Params:
    P = Params()
    P.nx, P.ny, P.nz = wl.nx, wl.ny, wl.nz
    for a in range(3):
        P.periodic[a] = int(wl.periodic[a])
        P.valence[a] = int(wl.valence[a])
        P.diffusivity[a] = float(wl.diffusivity[a])
        P.tau[a] = float(wl.tau[a])
        P.n_ref[a] = float(wl.n_ref[a])
        P.E_app[a] = float(wl.E_app[a])
        for c in range(3):
            P.body_force[a][c] = float(wl.body_force[a][c])
    P.bjerrum = wl.bjerrum
    P.poisson_tol = wl.poisson_tol
    P.poisson_max_iter = wl.poisson_max_iter
    P.poisson_check_every = wl.poisson_check_every
    P.poisson_fixed_iter = wl.poisson_fixed_iter
    P.rho_jacobi = wl.rho_jacobi
    P.md_substeps = wl.md_substeps
    P.bead_xi = wl.bead_xi
    P.bead_mass = wl.bead_mass
    P.bond_kind = wl.bond_kind
    P.bond_k, P.bond_r0, P.bond_l0 = wl.bond_k, wl.bond_r0, wl.bond_l0
    P.wca_eps, P.wca_sigma = wl.wca_eps, wl.wca_sigma
    P.wall_eps, P.wall_sigma = wl.wall_eps, wl.wall_sigma
    P.seed = wl.seed
    P.bead_kT = wl.bead_kT
    P.flags = wl.flags
    P.fluct_mass = wl.fluct_mass
    return P


class Sim:
    """One oracle simulation built from a workloads.Workload."""

    def __init__(self, wl, threads: int = 1):
        L = lib()
        self.wl = wl
        self.N = wl.n_nodes
        self.shape = (wl.nz, wl.ny, wl.nx)
        self._P = _params(wl)
        solid = np.ascontiguousarray(wl.solid, np.uint8)
        sc = None if wl.surface_charge is None else np.ascontiguousarray(wl.surface_charge, np.float64)
        n0 = None if wl.n_init is None else np.ascontiguousarray(wl.n_init, np.float64)
        err = C.c_int(0)
        h = L.eko_create(C.byref(self._P), _ptr(solid), _ptr(sc), _ptr(n0), C.byref(err))
        if not h:
            raise ValueError(f"oracle create failed ({err.value})")
        self.h = C.c_void_p(h)
        L.eko_set_threads(self.h, threads)
        if wl.R is not None and len(wl.R):
            self.set_beads(wl.R, wl.V, wl.charge, wl.chain)
        else:
            self.nb = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.eko_destroy(h)
            self.h = None

    def set_threads(self, t):
        lib().eko_set_threads(self.h, int(t))

    def set_beads(self, R, V, q, chain):
        R = np.ascontiguousarray(R, np.float64)
        V = np.ascontiguousarray(np.zeros_like(R) if V is None else V, np.float64)
        q = np.ascontiguousarray(q, np.float64)
        ch = np.ascontiguousarray(np.zeros(len(R), np.int32) if chain is None else chain, np.int32)
        self.nb = len(R)
        self._beads = (R, V, q, ch)
        lib().eko_set_beads(self.h, len(R), _ptr(R), _ptr(V), _ptr(q), _ptr(ch))

    def step(self, n=1):
        return lib().eko_step(self.h, int(n))

    def fields(self):
        N = self.N
        n = np.zeros((NS, N))
        j = np.zeros((NS, 3, N))
        phi = np.zeros(N)
        R = np.zeros((max(self.nb, 1), 3))
        V = np.zeros((max(self.nb, 1), 3))
        lib().eko_get_fields(self.h, _ptr(n), _ptr(j), _ptr(phi), _ptr(R), _ptr(V))
        return dict(n=n, j=j, phi=phi, R=R[: self.nb], V=V[: self.nb])

    def stats(self):
        out = np.zeros(12)
        lib().eko_get_stats(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return dict(mass=out[0:3].copy(), momentum=out[3:6].copy(), poisson_iters=int(out[6]),
                    poisson_res=out[7], bead_momentum=out[8:11].copy())

    def get_state(self):
        f = np.zeros((NS, Q, self.N))
        phi = np.zeros(self.N)
        st = C.c_int64(0)
        lib().eko_get_state(self.h, _ptr(f), _ptr(phi), C.byref(st))
        return f, phi, st.value

    def set_state(self, fstar, phi, step):
        f = np.ascontiguousarray(fstar, np.float64)
        p = np.ascontiguousarray(phi, np.float64)
        lib().eko_set_state(self.h, _ptr(f), _ptr(p), int(step))

    def link_mask(self):
        m = np.zeros(self.N, np.uint32)
        lib().eko_link_mask(self.h, _ptr(m))
        return m

    def wall_source(self):
        out = np.zeros(self.N)
        lib().eko_wall_source(self.h, _ptr(out))
        return out

    def poisson(self, rho, phi0=None, tol=1e-12, max_iter=100000, check_every=1, fixed_iter=0):
        rho = np.ascontiguousarray(rho, np.float64).ravel()
        phi = np.zeros(self.N) if phi0 is None else np.ascontiguousarray(phi0, np.float64).ravel().copy()
        res = C.c_double(0.0)
        it = lib().eko_poisson_solve(self.h, _ptr(rho), _ptr(phi), tol, max_iter, check_every,
                                     fixed_iter, C.byref(res))
        return phi, it, res.value

    def set_field(self, E):
        E = np.ascontiguousarray(E, np.float64)
        lib().eko_set_field(self.h, _ptr(E))

    def poisson_residual(self, rho, phi):
        """||b - A phi|| / ||b|| of phi for the charge density rho."""
        rho = np.ascontiguousarray(rho, np.float64).ravel()
        phi = np.ascontiguousarray(phi, np.float64).ravel()
        return lib().eko_poisson_residual(self.h, _ptr(rho), _ptr(phi))

    def last_rho(self):
        """Charge density rho_e of the last step."""
        out = np.zeros(self.N)
        lib().eko_last_rho(self.h, _ptr(out))
        return out

    def node_gradient(self, phi):
        phi = np.ascontiguousarray(phi, np.float64).ravel()
        g = np.zeros((3, self.N))
        lib().eko_node_gradient(self.h, _ptr(phi), _ptr(g))
        return g

    def bead_stencil(self, R):
        R = np.ascontiguousarray(R, np.float64)
        nodes = np.zeros(8, np.int64)
        w = np.zeros(8)
        ok = lib().eko_bead_stencil(self.h, _ptr(R), _ptr(nodes), _ptr(w))
        return bool(ok), nodes, w

    def default_rho_jacobi(self):
        return lib().eko_default_rho_jacobi(self.h)

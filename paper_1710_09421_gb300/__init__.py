"""GB300 electrokinetic lattice-Boltzmann / MD library: Python binding.

Argument marshalling over the C ABI declared in ``include/ekl.h``; every step
of the computation runs in the CUDA kernels of ``libekl.so``.  There is no
CPU fallback: loading fails loudly when the library is missing or cannot be
built.  PyTorch, when present, provides device memory (its caching allocator)
and the stream the library queues its work on.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads  # noqa: F401  (seeded inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libekl.so")

EKL_OK = 0
EKL_WARN_NOCONV = 1
EKL_WARN_CFL = 2
EKL_ERR_ARG = -1
EKL_ERR_ALLOC = -2
EKL_ERR_UNSTABLE = -3
EKL_ERR_BEAD = -4
EKL_ERR_TIMEOUT = -5
EKL_ERR_CUDA = -6

EKL_F64, EKL_F32, EKL_BF16DEV, EKL_FP16DEV = 0, 1, 2, 3
EKL_EQ_BARYCENTRIC, EKL_GAMMA_LITERAL, EKL_NO_BEAD_NOISE, EKL_POISSON_GLOBAL, EKL_POISSON_MG = 1, 2, 4, 8, 16
PRECISION = {"f64": EKL_F64, "f32": EKL_F32, "bf16": EKL_BF16DEV, "fp16": EKL_FP16DEV}

Q = 19
NS = 3
PHASES = ("bead_bin", "charge", "poisson", "bead_md", "lb", "other")


class ekl_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("periodic", C.c_int32 * 3),
        ("solid", C.c_void_p),
        ("surface_charge", C.c_void_p),
        ("n_init", C.c_void_p),
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
        ("precision", C.c_int32),
        ("fluct_mass", C.c_double),
    ]


class ekl_stats(C.Structure):
    _fields_ = [
        ("mass", C.c_double * 3),
        ("step", C.c_int64),
        ("poisson_iters", C.c_int32),
        ("status", C.c_int32),
        ("poisson_res", C.c_double),
        ("ms_phase", C.c_double * 6),
        ("launches", C.c_int64),
        ("poisson_sweeps", C.c_int64),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()
_alloc_refs = None


def load(build_if_missing: bool = True):
    """Load libekl.so (building it with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not found at {LIB_PATH}; build it with "
                               "paper_1710_09421_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.ekl_create.argtypes = [C.POINTER(ekl_params), vp, C.POINTER(vp)]
        L.ekl_set_beads.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
        L.ekl_step.argtypes = [vp, C.c_int32]
        L.ekl_step_async.argtypes = [vp, C.c_int32]
        L.ekl_get_fields.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ekl_get_state.argtypes = [vp, vp, vp, C.POINTER(C.c_int64)]
        L.ekl_set_state.argtypes = [vp, vp, vp, C.c_int64]
        L.ekl_get_stats.argtypes = [vp, C.POINTER(ekl_stats)]
        L.ekl_set_timing.argtypes = [vp, C.c_int32]
        L.ekl_set_field.argtypes = [vp, vp]
        L.ekl_selftest_wait.argtypes = []
        L.ekl_get_current.argtypes = [vp, C.c_int32, C.c_int32, vp]
        L.ekl_get_link_mask.argtypes = [vp, vp]
        L.ekl_lattice.argtypes = [vp, vp, vp]
        L.ekl_lattice.restype = None
        L.ekl_destroy.argtypes = [vp]
        L.ekl_test_set_device.argtypes = [vp, C.c_int32]
        L.ekl_get_fields_noalloc.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ekl_destroy.restype = None
        L.ekl_last_error.restype = C.c_char_p
        L.ekl_sizeof_params.restype = C.c_int64
        L.ekl_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
        L.ekl_batch_create.argtypes = [C.c_int32, C.POINTER(ekl_params), vp, C.POINTER(vp)]
        L.ekl_batch_set_beads.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp]
        L.ekl_batch_step.argtypes = [vp, C.c_int32]
        L.ekl_batch_replica.argtypes = [vp, C.c_int32]
        L.ekl_batch_replica.restype = vp
        L.ekl_batch_autotune.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
        L.ekl_batch_set_schedule.argtypes = [vp, C.c_int32]
        L.ekl_batch_launches.argtypes = [vp]
        L.ekl_batch_launches.restype = C.c_int64
        L.ekl_batch_destroy.argtypes = [vp]
        L.ekl_batch_destroy.restype = None
        L.ekl_net_eval.argtypes = [vp, vp, vp, vp, vp]
        L.ekl_set_warmstart.argtypes = [vp, vp, vp]
        L.ekl_warmstart_collect.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, vp,
                                            C.POINTER(C.c_int64)]
        L.ekl_net_loss_grad.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(C.c_double), vp]
        L.ekl_warmstart_level.argtypes = [vp, C.c_int32]
        L.ekl_net_tensor_path.argtypes = [C.c_int32]
        L.ekl_net_train_grid.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_float,
                                         C.c_uint64, vp]
        L.ekl_net_train.argtypes = [C.c_int32, vp, vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_float,
                                    C.c_uint64, vp]
        if L.ekl_sizeof_params() != C.sizeof(ekl_params):
            raise RuntimeError("ekl_params layout of the binding does not match the library")
        _lib = L
    return _lib


class EklError(RuntimeError):
    def __init__(self, code, where):
        msg = load().ekl_last_error().decode()
        super().__init__(f"{where} failed with {code}: {msg}")
        self.code = code


def _check(code, where):
    if code < 0:
        raise EklError(code, where)
    return code


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ C names
def ekl_lattice():
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    load().ekl_lattice(_ptr(c), _ptr(w), _ptr(opp))
    return c, w, opp


def ekl_set_allocator(alloc, free):
    """Install Python callables alloc(bytes, stream) -> int and free(ptr, bytes,
    stream) as the device allocator (None, None restores cudaMalloc)."""
    global _alloc_refs
    L = load()
    if alloc is None:
        _alloc_refs = None
        return _check(L.ekl_set_allocator(ALLOC_FN(), FREE_FN(), None), "ekl_set_allocator")
    a = ALLOC_FN(lambda n, s, ctx: int(alloc(int(n), s)))
    f = FREE_FN(lambda p, n, s, ctx: free(int(p), int(n), s))
    _alloc_refs = (a, f)
    return _check(L.ekl_set_allocator(a, f, None), "ekl_set_allocator")


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    def alloc(n, stream):
        return torch.cuda.caching_allocator_alloc(n, dev, stream)

    def free(p, n, stream):
        torch.cuda.caching_allocator_delete(p)

    return ekl_set_allocator(alloc, free)


def make_params(wl, precision=None):
    """ekl_params (and the arrays it points to) from a workloads.Workload."""
    P = ekl_params()
    P.nx, P.ny, P.nz = wl.nx, wl.ny, wl.nz
    keep = []
    solid = np.ascontiguousarray(wl.solid, np.uint8)
    keep.append(solid)
    P.solid = solid.ctypes.data
    if wl.surface_charge is not None:
        sc = np.ascontiguousarray(wl.surface_charge, np.float64)
        keep.append(sc)
        P.surface_charge = sc.ctypes.data
    if wl.n_init is not None:
        n0 = np.ascontiguousarray(wl.n_init, np.float64)
        keep.append(n0)
        P.n_init = n0.ctypes.data
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
    P.precision = PRECISION[precision or wl.precision]
    P.fluct_mass = wl.fluct_mass
    return P, keep


def ekl_create(params, stream=None):
    h = C.c_void_p()
    _check(load().ekl_create(C.byref(params), stream, C.byref(h)), "ekl_create")
    return h


def ekl_set_beads(h, R, V, q, chain):
    R = np.ascontiguousarray(R, np.float64)
    V = None if V is None else np.ascontiguousarray(V, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    ch = None if chain is None else np.ascontiguousarray(chain, np.int32)
    return _check(load().ekl_set_beads(h, len(R), _ptr(R), _ptr(V), _ptr(q), _ptr(ch)),
                  "ekl_set_beads")


def ekl_step(h, nsteps):
    return _check(load().ekl_step(h, int(nsteps)), "ekl_step")


def ekl_step_async(h, nsteps):
    return _check(load().ekl_step_async(h, int(nsteps)), "ekl_step_async")


def ekl_get_fields(h, N, nb, which=("n", "j", "phi", "R", "V")):
    n = np.zeros((NS, N)) if "n" in which else None
    j = np.zeros((NS, 3, N)) if "j" in which else None
    phi = np.zeros(N) if "phi" in which else None
    R = np.zeros((max(nb, 1), 3)) if "R" in which else None
    V = np.zeros((max(nb, 1), 3)) if "V" in which else None
    _check(load().ekl_get_fields(h, _ptr(n), _ptr(j), _ptr(phi), _ptr(R), _ptr(V)),
           "ekl_get_fields")
    return dict(n=n, j=j, phi=phi, R=None if R is None else R[:nb],
                V=None if V is None else V[:nb])


def ekl_get_state(h, N):
    f = np.zeros((NS, Q, N))
    phi = np.zeros(N)
    st = C.c_int64(0)
    _check(load().ekl_get_state(h, _ptr(f), _ptr(phi), C.byref(st)), "ekl_get_state")
    return f, phi, st.value


def ekl_set_state(h, fstar, phi, step):
    f = np.ascontiguousarray(fstar, np.float64)
    p = None if phi is None else np.ascontiguousarray(phi, np.float64)
    return _check(load().ekl_set_state(h, _ptr(f), _ptr(p), int(step)), "ekl_set_state")


def ekl_get_stats(h):
    s = ekl_stats()
    _check(load().ekl_get_stats(h, C.byref(s)), "ekl_get_stats")
    return dict(mass=np.array(s.mass[:]), step=s.step, poisson_iters=s.poisson_iters,
                status=s.status, poisson_res=s.poisson_res,
                ms_phase=dict(zip(PHASES, s.ms_phase[:])), launches=s.launches,
                poisson_sweeps=s.poisson_sweeps)


def ekl_set_field(h, E):
    E = np.ascontiguousarray(E, np.float64)
    return _check(load().ekl_set_field(h, _ptr(E)), "ekl_set_field")


def ekl_get_current(h, axis, plane):
    """Species fluxes through a lattice plane and the ionic current (4 values)."""
    out = np.zeros(4)
    _check(load().ekl_get_current(h, int(axis), int(plane), _ptr(out)), "ekl_get_current")
    return out


def ekl_set_timing(h, on):
    return _check(load().ekl_set_timing(h, 1 if on else 0), "ekl_set_timing")


def ekl_get_link_mask(h, N):
    m = np.zeros(N, np.uint32)
    _check(load().ekl_get_link_mask(h, _ptr(m)), "ekl_get_link_mask")
    return m


def ekl_destroy(h):
    if h:
        load().ekl_destroy(h)


# ------------------------------------------------------------ convenience
class Simulation:
    """One handle built from a workloads.Workload (marshalling only)."""

    def __init__(self, wl, precision=None, stream=None):
        self.wl = wl
        self.N = wl.n_nodes
        self.nb = wl.n_beads
        P, keep = make_params(wl, precision)
        self.h = ekl_create(P, stream)
        del keep
        if self.nb:
            ekl_set_beads(self.h, wl.R, wl.V, wl.charge, wl.chain)

    def close(self):
        if getattr(self, "h", None):
            ekl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        return ekl_step(self.h, n)

    def step_async(self, n=1):
        return ekl_step_async(self.h, n)

    def fields(self, which=("n", "j", "phi", "R", "V")):
        return ekl_get_fields(self.h, self.N, self.nb, which)

    def stats(self):
        return ekl_get_stats(self.h)

    def get_state(self):
        return ekl_get_state(self.h, self.N)

    def set_state(self, fstar, phi, step):
        return ekl_set_state(self.h, fstar, phi, step)

    def set_beads(self, R, V, q, chain):
        self.nb = len(R)
        return ekl_set_beads(self.h, R, V, q, chain)

    def link_mask(self):
        return ekl_get_link_mask(self.h, self.N)

    def set_timing(self, on=True):
        return ekl_set_timing(self.h, on)

    def set_field(self, E):
        return ekl_set_field(self.h, E)

    def current(self, axis=2, plane=None):
        """out[0:3] species fluxes, out[3] ionic current through the plane
        (default: the middle plane along `axis`)."""
        L = (self.wl.nx, self.wl.ny, self.wl.nz)[axis]
        return ekl_get_current(self.h, axis, L // 2 if plane is None else plane)

    def set_warmstart(self, w, scales=(1.0, 1.0, 1.0), level=None):
        if level is not None:
            ekl_warmstart_level(self.h, level)
        return ekl_set_warmstart(self.h, w, scales)

    def warmstart_level(self, level):
        self._ws_level = int(level)
        return ekl_warmstart_level(self.h, level)

    def collect(self, nsteps, crop=16, ncrops=8, seed=0):
        L = getattr(self, "_ws_level", 0)
        if L:
            dims = (self.wl.nz >> L, self.wl.ny >> L, self.wl.nx >> L)
            return ekl_warmstart_collect_level(self.h, nsteps, dims, seed)
        return ekl_warmstart_collect(self.h, nsteps, crop, ncrops, seed)


# ------------------------------------------------------------------ batches
def ekl_batch_create(params_list, stream=None):
    arr = (ekl_params * len(params_list))(*params_list)
    h = C.c_void_p()
    _check(load().ekl_batch_create(len(params_list), arr, stream, C.byref(h)), "ekl_batch_create")
    return h


def ekl_batch_set_beads(b, rep, R, V, q, chain):
    R = np.ascontiguousarray(R, np.float64)
    V = None if V is None else np.ascontiguousarray(V, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    ch = None if chain is None else np.ascontiguousarray(chain, np.int32)
    return _check(load().ekl_batch_set_beads(b, int(rep), len(R), _ptr(R), _ptr(V), _ptr(q), _ptr(ch)),
                  "ekl_batch_set_beads")


def ekl_batch_step(b, nsteps):
    return _check(load().ekl_batch_step(b, int(nsteps)), "ekl_batch_step")


def ekl_batch_replica(b, rep):
    return C.c_void_p(load().ekl_batch_replica(b, int(rep)))


def ekl_batch_set_schedule(b, choice):
    return _check(load().ekl_batch_set_schedule(b, int(choice)), "ekl_batch_set_schedule")


def ekl_batch_autotune(b, trial_steps):
    c = C.c_int32(0)
    _check(load().ekl_batch_autotune(b, int(trial_steps), C.byref(c)), "ekl_batch_autotune")
    return c.value


def ekl_batch_destroy(b):
    if b:
        load().ekl_batch_destroy(b)


class _Replica:
    """Read-back view of one replica of a Batch (plus the applied field,
    which takes effect from the batch's next step)."""

    def __init__(self, h, wl, nb):
        self.h, self.wl, self.N, self.nb = h, wl, wl.n_nodes, nb

    def fields(self, which=("n", "j", "phi", "R", "V")):
        return ekl_get_fields(self.h, self.N, self.nb, which)

    def stats(self):
        return ekl_get_stats(self.h)

    def get_state(self):
        return ekl_get_state(self.h, self.N)

    def set_field(self, E):
        return ekl_set_field(self.h, E)


class Batch:
    """Many independent workloads stepped together (marshalling only)."""

    def __init__(self, wls, precision=None, stream=None):
        self.wls = list(wls)
        plist, keep = [], []
        for wl in self.wls:
            P, k = make_params(wl, precision)
            plist.append(P)
            keep.append(k)
        self.h = ekl_batch_create(plist, stream)
        del keep
        self.reps = []
        for r, wl in enumerate(self.wls):
            if wl.n_beads:
                ekl_batch_set_beads(self.h, r, wl.R, wl.V, wl.charge, wl.chain)
            self.reps.append(_Replica(ekl_batch_replica(self.h, r), wl, wl.n_beads))

    def step(self, n=1):
        return ekl_batch_step(self.h, n)

    def autotune(self, trial_steps=2):
        return ekl_batch_autotune(self.h, trial_steps)

    def set_schedule(self, choice):
        return ekl_batch_set_schedule(self.h, choice)

    def launches(self):
        return load().ekl_batch_launches(self.h)

    def close(self):
        if getattr(self, "h", None):
            ekl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ warm-start network
EKL_NET_PARAMS = 15169


def _i3(v):
    return np.ascontiguousarray(v, np.int32)


def ekl_net_eval(dims, periodic, x, w):
    """dims = (nx, ny, nz); x[2][nz][ny][nx]; returns y[nz][ny][nx]."""
    d, p = _i3(dims), _i3(periodic)
    x = np.ascontiguousarray(x, np.float32)
    w = np.ascontiguousarray(w, np.float32)
    y = np.zeros(x.shape[1:], np.float32)
    _check(load().ekl_net_eval(_ptr(d), _ptr(p), _ptr(x), _ptr(w), _ptr(y)), "ekl_net_eval")
    return y


def ekl_net_loss_grad(dims, periodic, x, target, mask, w):
    d, p = _i3(dims), _i3(periodic)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(target, np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    w = np.ascontiguousarray(w, np.float32)
    g = np.zeros(EKL_NET_PARAMS, np.float32)
    loss = C.c_double(0)
    _check(load().ekl_net_loss_grad(_ptr(d), _ptr(p), _ptr(x), _ptr(t), _ptr(m), _ptr(w),
                                     C.byref(loss), _ptr(g)), "ekl_net_loss_grad")
    return loss.value, g


def ekl_net_train(dims, x, target, mask, w, iters, batch=4, lr=1e-3, seed=0):
    """x[S][2][...], target[S][...]; returns (trained w, per-iteration loss)."""
    d = _i3(dims)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(target, np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    w = np.ascontiguousarray(w, np.float32).copy()
    curve = np.zeros(iters, np.float32)
    _check(load().ekl_net_train(len(x), _ptr(d), _ptr(x), _ptr(t), _ptr(m), _ptr(w), int(iters),
                                int(batch), float(lr), int(seed), _ptr(curve)), "ekl_net_train")
    return w, curve


def ekl_set_warmstart(h, w, scales=(1.0, 1.0, 1.0)):
    """Install (w: EKL_NET_PARAMS floats) or remove (w=None) the warm start."""
    wp = None if w is None else np.ascontiguousarray(w, np.float32)
    sc = np.ascontiguousarray(scales, np.float32)
    return _check(load().ekl_set_warmstart(h, _ptr(wp), _ptr(sc)), "ekl_set_warmstart")


def ekl_warmstart_level(h, level):
    return _check(load().ekl_warmstart_level(h, int(level)), "ekl_warmstart_level")


def ekl_warmstart_collect_level(h, nsteps, dims_zyx, seed=0):
    """Coarse-level samples[k][3][nzL][nyL][nxL] = (db summed per cell,
    phi_prev and dphi averaged per cell)."""
    out = np.zeros((nsteps, 3) + tuple(dims_zyx), np.float32)
    n = C.c_int64(0)
    _check(load().ekl_warmstart_collect(h, int(nsteps), 0, 1, int(seed), _ptr(out), C.byref(n)),
           "ekl_warmstart_collect")
    return out[: n.value]


def ekl_net_train_grid(dims, periodic, x, target, mask, w, iters, batch=4, lr=1e-3, seed=0):
    """ekl_net_train on a grid with periodic axes; returns (trained w, loss curve)."""
    d = _i3(dims)
    p = _i3(periodic)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(target, np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    w = np.ascontiguousarray(w, np.float32).copy()
    curve = np.zeros(iters, np.float32)
    _check(load().ekl_net_train_grid(len(x), _ptr(d), _ptr(p), _ptr(x), _ptr(t), _ptr(m), _ptr(w), int(iters),
                                     int(batch), float(lr), int(seed), _ptr(curve)), "ekl_net_train_grid")
    return w, curve


def ekl_warmstart_collect(h, nsteps, crop=16, ncrops=8, seed=0):
    """Returns crops[k][3][crop][crop][crop] = (db, phi_prev, dphi)."""
    out = np.zeros((nsteps * ncrops, 3, crop, crop, crop), np.float32)
    n = C.c_int64(0)
    _check(load().ekl_warmstart_collect(h, int(nsteps), int(crop), int(ncrops), int(seed), _ptr(out),
                                        C.byref(n)), "ekl_warmstart_collect")
    return out[: n.value]

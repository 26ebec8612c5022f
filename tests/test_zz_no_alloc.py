"""The allocation-free field read-back, ekl_get_fields_noalloc, through the C ABI.

It serves callers that may not allocate device memory while they run (for
instance between capture and replay of a CUDA graph, or in a loop that has
reserved all GPU memory up front): it stages the fields in one fixed device
array instead of per-call buffers.  Here it must return what ekl_get_fields
returns, bit for bit, on two calls in a row, and refuse a request larger than
its array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1710_09421_gb300 as E
from paper_1710_09421_gb300 import workloads as W

pytestmark = pytest.mark.gpu

def _noalloc(lib):
    f = lib.ekl_get_fields_noalloc
    f.argtypes = [C.c_void_p] * 6
    f.restype = C.c_int
    return f


def _fields_noalloc(f, sim):
    N, nb = sim.N, sim.nb
    n = np.full((3, N), np.nan)
    j = np.full((3, 3, N), np.nan)
    phi = np.full(N, np.nan)
    R = np.full((nb, 3), np.nan)
    V = np.full((nb, 3), np.nan)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = f(sim.h, p(n), p(j), p(phi), p(R), p(V))
    assert rc == E.EKL_OK, (rc, E.load().ekl_last_error())
    return dict(n=n, j=j, phi=phi, R=R, V=V)


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16", "fp16"])
def test_noalloc_matches_get_fields_twice(precision):
    lib = E.load()
    f = _noalloc(lib)
    wl = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=4,
                      precision=precision)
    sim = E.Simulation(wl)
    for call in range(2):
        sim.step(5)
        ref = sim.fields()
        got = _fields_noalloc(f, sim)
        for k in ("n", "j", "phi", "R", "V"):
            assert np.array_equal(got[k], ref[k]), (call, k)
    sim.close()


def test_noalloc_rejects_requests_beyond_its_array():
    lib = E.load()
    f = _noalloc(lib)
    # 64 x 64 x 48 = 196608 nodes: all fields need 13 N doubles > 2^21
    wl = W.translocation(nx=64, ny=64, nz=48, membrane=(20, 27), n_beads=0)
    sim = E.Simulation(wl)
    N = sim.N
    n = np.zeros((3, N))
    j = np.zeros((3, 3, N))
    phi = np.zeros(N)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = f(sim.h, p(n), p(j), p(phi), None, None)
    assert rc == E.EKL_ERR_ARG
    assert b"allocation-free path holds" in lib.ekl_last_error()
    # the potential alone fits
    assert f(sim.h, None, None, p(phi), None, None) == E.EKL_OK
    assert np.array_equal(phi, sim.fields(("phi",))["phi"])
    sim.close()


def test_noalloc_refuses_a_handle_whose_device_is_unavailable():
    """The staging array's address is looked up for the handle's device with
    that device current; a handle whose device cannot be made current is
    refused (EKL_ERR_ARG) before any lookup or work, and nothing is cached
    for it: restored to its real device, the same handle reads back exactly
    what ekl_get_fields returns."""
    import torch

    lib = E.load()
    f = _noalloc(lib)
    wl = W.small_pore(nx=16, ny=16, nz=20, membrane=(8, 11), radius=3.0, n_beads=4, precision="f32")
    sim = E.Simulation(wl)
    sim.step(3)
    ref = sim.fields()
    dev = torch.cuda.current_device()
    assert lib.ekl_test_set_device(sim.h, torch.cuda.device_count()) == E.EKL_OK
    N, nb = sim.N, sim.nb
    n = np.zeros((3, N))
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    assert f(sim.h, p(n), None, None, None, None) == E.EKL_ERR_ARG
    assert b"device cannot be made current" in lib.ekl_last_error()
    assert lib.ekl_step(sim.h, 1) == E.EKL_ERR_ARG
    assert torch.cuda.current_device() == dev
    assert lib.ekl_test_set_device(sim.h, dev) == E.EKL_OK
    got = _fields_noalloc(f, sim)
    for k in ("n", "j", "phi", "R", "V"):
        assert np.array_equal(got[k], ref[k]), k
    sim.close()

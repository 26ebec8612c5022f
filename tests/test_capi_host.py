"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every function that include/ekl.h declares, its parameter block has
the binding's layout, and its lattice table equals the oracle's."""
import os
import re
import subprocess

import numpy as np

import oracle
import paper_1710_09421_gb300 as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ekl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ekl_[a-z0-9_]+)\s*\(", src)) - {"ekl_alloc_fn", "ekl_free_fn"})


def test_library_exports_every_declared_symbol():
    E.load()
    out = subprocess.run(["nm", "-D", "--defined-only", E.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (ekl_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    assert len(_declared()) >= 15


def test_params_layout():
    L = E.load()
    assert L.ekl_sizeof_params() == __import__("ctypes").sizeof(E.ekl_params)


def test_lattice_table_matches_oracle():
    c, w, opp = E.ekl_lattice()
    c2, w2, opp2 = oracle.lattice()
    assert np.array_equal(c, c2) and np.array_equal(w, w2) and np.array_equal(opp, opp2)


def test_no_cpu_fallback_in_binding():
    """The binding carries no arithmetic of its own: it never imports the
    oracle and has no numpy stand-in for a kernel."""
    src = open(os.path.join(ROOT, "paper_1710_09421_gb300", "__init__.py")).read()
    assert "oracle" not in src.replace("# ", "")
    for name in ("stream(", "collide", "poisson_solve"):
        assert name not in src


def test_batch_entry_points_reject_a_null_batch():
    """The batch calls check their handle before any CUDA work: a null batch
    is refused with EKL_ERR_ARG and a message (and has made no launches)."""
    import ctypes as C

    L = E.load()
    L.ekl_batch_set_schedule.argtypes = [C.c_void_p, C.c_int32]
    L.ekl_batch_step.argtypes = [C.c_void_p, C.c_int32]
    L.ekl_batch_launches.argtypes = [C.c_void_p]
    L.ekl_batch_launches.restype = C.c_int64
    assert L.ekl_batch_set_schedule(None, 1) == E.EKL_ERR_ARG
    assert b"batch" in L.ekl_last_error()
    assert L.ekl_batch_step(None, 1) == E.EKL_ERR_ARG
    assert L.ekl_batch_launches(None) == 0

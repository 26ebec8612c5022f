"""Small builders shared by the tests (inputs only, no method arithmetic)."""
import numpy as np

from paper_1710_09421_gb300 import workloads as W


def box(nx, ny, nz, periodic=(1, 1, 1), solid=None, n=(1.0, 0.01, 0.01), **kw):
    """A workload with uniform densities and no beads."""
    if solid is None:
        solid = np.zeros((nz, ny, nx), np.uint8)
    fluid = solid == 0
    n_init = np.zeros((3, nz, ny, nx))
    for a in range(3):
        n_init[a][fluid] = n[a]
    base = dict(name="box", nx=nx, ny=ny, nz=nz, periodic=tuple(periodic), solid=solid,
                surface_charge=None, n_init=n_init, n_ref=tuple(n), precision="f64")
    base.update(kw)
    return W.Workload(**base)


def slit(nx, ny, nz, **kw):
    return box(nx, ny, nz, periodic=(1, 1, 0), solid=W.slit_solid(nx, ny, nz), **kw)


def node_coords(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def pointwise(a, b):
    """max |a - b| / max |b|: the worst node against the field's scale."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    mb = np.abs(b).max()
    return np.abs(a - b).max() / (mb if mb > 0 else 1.0)

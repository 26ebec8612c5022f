"""Translocation observables (Sec. IV.B-C) from what the library returns:
the ionic current through a plane (ekl_get_current), the conductance it
gives, and bead crossing times.  Host-side arithmetic on returned values."""
from __future__ import annotations

import math

import numpy as np


def conductance(current, E_axis, L_axis):
    """G = I / Delta V with Delta V = E L the potential drop (k_B T / e) that a
    uniform applied field E produces over the periodic box length L."""
    return current / (E_axis * L_axis)


def g0(pore_length, v_T=1.0 / math.sqrt(3.0), m=1.0):
    """The paper's reference conductance G_0 = e^2 / (m v_T L_p) in lattice
    units (e = 1, Sec. IV.B)."""
    return 1.0 / (m * v_T * pore_length)


def crossing_times(z_traj, z_plane, direction=-1):
    """First time index at which each bead passes z_plane moving along
    `direction` (-1: towards smaller z); -1 where it never does.
    z_traj: [times][beads]."""
    z = np.asarray(z_traj)
    past = (z < z_plane) if direction < 0 else (z > z_plane)
    first = np.argmax(past, axis=0)
    return np.where(past.any(axis=0), first, -1)


def relax_then_drive(sim, relax_steps, E, chunk=100):
    """The paper's protocol: relax the chain at zero field for about a Rouse
    time, then apply the field (Sec. IV.A).  Returns the status codes."""
    E0 = np.zeros(3)
    sim.set_field(E0)
    out = []
    for k in range(0, relax_steps, chunk):
        out.append(sim.step(min(chunk, relax_steps - k)))
    sim.set_field(E)
    return out

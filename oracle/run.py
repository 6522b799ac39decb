"""Drivers that build the oracle for a synthetic case and run it.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

from .dg import Discretization
from . import refelem as R


def node_coords(dim, coords, etov, order):
    """Physical coordinates (K, Np, dim) of the equispaced nodes, computed from
    the affine map of each element."""
    coords = np.asarray(coords, dtype=float).reshape(-1, dim)
    X = coords[np.asarray(etov)]
    r = R.ref_nodes(dim, order)
    if dim == 1:
        lam = 0.5 * (1.0 + r[:, 0])
        return X[:, 0, None, :] * (1 - lam)[None, :, None] + X[:, 1, None, :] * lam[None, :, None]
    l1 = 0.5 * (1.0 + r[:, 0])
    l2 = 0.5 * (1.0 + r[:, 1])
    l0 = 1.0 - l1 - l2
    return (X[:, 0, None, :] * l0[None, :, None] + X[:, 1, None, :] * l1[None, :, None]
            + X[:, 2, None, :] * l2[None, :, None])


def build(case, order=None, m3=None):
    """Discretization and nodal initial state (V nodal, bed nodal) for a case."""
    p = case.order if order is None else order
    xyz = node_coords(case.dim, case.coords, case.etov, p)
    V0, bed = case.initial_state(xyz)
    mm = case.m3 if m3 is None else m3
    disc = Discretization(case.dim, case.coords, case.etov, p, case.params,
                          face_bc=case.face_bc, bcs=case.bcs, bed_nodal=bed, m3=mm)
    return disc, V0, bed


def run_explicit(disc, V0_nodal, n_steps, dt=None):
    """n_steps SSP-RK3 steps from a nodal state; returns final nodal state,
    the list of step sizes and the final time."""
    Vh = disc.to_modal(V0_nodal)
    dts = []
    for _ in range(n_steps):
        Vh, dtk = disc.ssp_rk3_step(Vh, dt)
        dts.append(dtk)
    return disc.to_nodal(Vh), dts, float(np.sum(dts))


def residual_nodal(disc, V_nodal):
    """dV/dt and E at the nodes for a nodal state (one residual evaluation)."""
    Vh = disc.to_modal(V_nodal)
    dV, Eh = disc.rhs(Vh)
    return disc.to_nodal(dV), disc.E_to_nodal(Eh)

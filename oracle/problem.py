"""Manufactured-solution stage problem on a hierarchy (Section 3.1 stage
right-hand side; initial data by interpolation of the exact solution, with
the pressure shifted to zero mean as the L^2_0 space requires)."""
import numpy as np

import synth
from . import stage


def initial_state(mesh, t=0.0, kind="steady"):
    X, Y = mesh.p2_coords[mesh.free_p2].T
    un = np.concatenate(synth.mms_velocity(X, Y, t, kind))
    pn = synth.mms_pressure(mesh.coords[:, 0], mesh.coords[:, 1], t, kind)
    return un, pn - pn.mean()


def forcing(mesh, c, t0, dt, nu=1.0, kind="steady"):
    """f_i at every P2 node at t0 + c_i dt, shape [s, 2, np2]."""
    X, Y = mesh.p2_coords.T
    return np.stack([np.stack(synth.mms_forcing(X, Y, t0 + ci * dt, nu, kind)) for ci in c])


def mms_rhs(H, c, t0=0.0, kind="steady"):
    """Stage right-hand side F on the finest level of hierarchy H."""
    L = H.finest
    un, pn = initial_state(L.mesh, t0, kind)
    f = forcing(L.mesh, c, t0, H.dt, H.nu, kind)
    return stage.stage_rhs(L.ops, un, pn, f), un, pn

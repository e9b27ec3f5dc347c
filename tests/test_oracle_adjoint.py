"""Pins for the oracle's discrete adjoint: central finite differences of its
own forward model (solved by sparse direct LU), the transpose identity of the
stage operator, and checkpointing that does not change the result."""
import numpy as np
import pytest

import synth
from oracle import adjoint, mesh as M, problem, tableau


def _setup(n=6, s=2, dt=1 / 32, nu=1.0):
    A, b, c = tableau.radau_iia(s)
    m = M.Mesh(*synth.square_mesh(n))
    prob = adjoint.Problem(m, A, b, dt, nu)
    u0, p0 = problem.initial_state(m)
    X, Y = m.p2_coords[m.free_p2].T
    ut = np.concatenate(synth.mms_velocity(X, Y))
    forcing = lambda k: problem.forcing(m, c, k * dt, dt, nu)
    theta = synth.normal(7, 2 * m.nc)
    return prob, u0, p0, ut, forcing, theta, c


def test_transpose_identity():
    prob, *_ = _setup()
    x = synth.random_vector(1, prob.J.shape[0])
    y = synth.random_vector(2, prob.J.shape[0])
    assert abs(x @ (prob.J.T @ y) - (prob.J @ x) @ y) <= 1e-13 * np.abs(prob.J).sum()


def test_gradient_matches_central_differences():
    prob, u0, p0, ut, forcing, theta, _ = _setup()
    nsteps = 4
    ut = 0.9 * ut
    J0, thb, dnu = adjoint.run(prob, u0, p0, forcing, theta, nsteps, ut)
    assert J0 > 0
    d = synth.normal(11, theta.size)
    h = 1e-6 * max(1.0, np.abs(theta).max())
    Jp = adjoint.objective_only(prob, u0, p0, forcing, theta + h * d, nsteps, ut)
    Jm = adjoint.objective_only(prob, u0, p0, forcing, theta - h * d, nsteps, ut)
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - thb @ d) <= 1e-5 * abs(fd)
    nu0 = prob.nu
    hn = 1e-6
    prob.set_nu(nu0 + hn)
    Jp = adjoint.objective_only(prob, u0, p0, forcing, theta, nsteps, ut)
    prob.set_nu(nu0 - hn)
    Jm = adjoint.objective_only(prob, u0, p0, forcing, theta, nsteps, ut)
    prob.set_nu(nu0)
    fdn = (Jp - Jm) / (2 * hn)
    assert abs(fdn - dnu) <= 1e-5 * abs(fdn)


def test_checkpoint_interval_does_not_change_gradient():
    prob, u0, p0, ut, forcing, theta, _ = _setup(n=4)
    r1 = adjoint.run(prob, u0, p0, forcing, theta, 5, 0.5 * ut, checkpoint_every=1)
    r2 = adjoint.run(prob, u0, p0, forcing, theta, 5, 0.5 * ut, checkpoint_every=2)
    r5 = adjoint.run(prob, u0, p0, forcing, theta, 5, 0.5 * ut, checkpoint_every=5)
    for a, b in [(r1, r2), (r1, r5)]:
        assert abs(a[0] - b[0]) <= 1e-14 * abs(a[0])
        np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-14 * np.abs(a[1]).max())
        assert abs(a[2] - b[2]) <= 1e-12 * abs(a[2])


def test_cell_load_integrates_constants():
    """sum over all P2 nodes of int_c phi_a = |c| (partition of unity); vertex
    functions of P2 integrate to zero on a triangle."""
    m = M.Mesh(*synth.square_mesh(3))
    C = adjoint.cell_load_matrix(m)
    mm = M.Mesh(*synth.square_mesh(3), )
    from oracle import fem
    ref = np.array([fem._integral_over_area(fem.P2[a]) for a in range(6)])
    np.testing.assert_allclose(ref[:3], 0.0, atol=1e-15)
    np.testing.assert_allclose(ref[3:], 1.0 / 3.0, atol=1e-15)
    # a cell with no Dirichlet edge keeps all of its mass on free nodes
    area = 0.5 / 9
    interior = [c for c in range(m.nc) if np.all(m.p2_to_free[m.cell_p2[c, 3:]] >= 0)]
    np.testing.assert_allclose(np.asarray(C.sum(axis=0)).ravel()[interior], area, rtol=1e-14)

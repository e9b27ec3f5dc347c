"""Pins of the Navier-Stokes stage oracle (Section 3.2): the Jacobian is the
derivative of the stage residual (central differences), Newton converges
quadratically to a root of the residual, and that root is the one an
independent solver (MINPACK's hybrid method with its own finite-difference
Jacobian) finds.  Lid-driven cavity on a 4x4 mesh, Radau IIA(2)."""
import numpy as np
import pytest
import scipy.optimize as so

import synth
from oracle import mesh as M, ns, tableau


def _cavity(n0=2, nl=2, s=2, dt=0.05, nu=0.01):
    mesh = M.hierarchy(*synth.square_mesh(n0), nl)[-1]
    A = tableau.radau_iia(s)[0]
    st = ns.NSStages(mesh, A, dt, nu)
    X = mesh.p2_coords
    lx, ly = synth.lid_velocity(X[:, 0], X[:, 1])
    un = np.stack([lx, ly], axis=1)
    pn = np.zeros(mesh.nv)
    f = np.zeros((s, mesh.np2, 2))
    return st, un, pn, f


def test_jacobian_is_the_derivative_of_the_stage_residual():
    st, un, pn, f = _cavity()
    rng = np.random.default_rng(3)
    k = 0.5 * rng.standard_normal(st.N)
    d = rng.standard_normal(st.N)
    J = st.jacobian(k, un, pn)
    h = 1e-5
    fd = (st.residual(k + h * d, un, pn, f) - st.residual(k - h * d, un, pn, f)) / (2 * h)
    assert np.linalg.norm(J @ d - fd) <= 1e-7 * np.linalg.norm(fd)


def test_reaction_term_is_needed():
    """Dropping R(U) from the Jacobian (the Picard/Oseen linearisation) leaves
    an O(1) mismatch with the derivative: a plausible omission is caught."""
    st, un, pn, f = _cavity()
    rng = np.random.default_rng(4)
    k = 0.5 * rng.standard_normal(st.N)
    d = rng.standard_normal(st.N)
    saved = ns.reaction_matrices
    try:
        ns.reaction_matrices = lambda *a: 0.0 * saved(*a)
        J0 = st.jacobian(k, un, pn)
    finally:
        ns.reaction_matrices = saved
    h = 1e-5
    fd = (st.residual(k + h * d, un, pn, f) - st.residual(k - h * d, un, pn, f)) / (2 * h)
    assert np.linalg.norm(J0 @ d - fd) > 1e-3 * np.linalg.norm(fd)


def test_newton_converges_quadratically_to_the_independent_root():
    st, un, pn, f = _cavity()
    k, hist, _ = ns.newton(st, un, pn, f, np.zeros(st.N), ns.bordered_solve(st), atol=1e-12)
    assert hist[-1] <= 1e-12
    # quadratic: once in the basin, each residual is below C times the square
    r = np.array(hist)
    tail = [(r[i + 1], r[i]) for i in range(len(r) - 1) if r[i] < 1e-2]
    assert any(b > 0 and a <= 10.0 * b * b for a, b in tail)
    # the root of an independent solver (bordered: zero pressure mean per stage)
    mask = st.pressure_mask()
    s, m, nf = st.s, st.m, st.nf

    def G(z):
        kz, lam = z[:st.N], z[st.N:]
        F = st.residual(kz, un, pn, f)
        for t in range(s):
            F[t * m + 2 * nf:(t + 1) * m] += lam[t]
        cons = [kz[t * m + 2 * nf:(t + 1) * m].sum() for t in range(s)]
        return np.concatenate([F, cons])

    sol = so.root(G, np.zeros(st.N + s), method="hybr", options={"xtol": 1e-13})
    assert sol.success
    kr = sol.x[:st.N]
    assert np.linalg.norm(kr[~mask] - k[~mask]) <= 1e-8 * np.linalg.norm(k[~mask])
    assert np.linalg.norm(st.project_pressure(kr)[mask] - st.project_pressure(k)[mask]) <= \
        1e-8 * np.linalg.norm(st.project_pressure(k)[mask])


def test_eisenstat_walker_forcing_terms():
    """Choice 2 with its safeguard and cap."""
    assert ns.eisenstat_walker(0.5, 1e-2, 1e-1) == pytest.approx(max(0.9 * 1e-2, 0.9 * 0.25))
    assert ns.eisenstat_walker(0.2, 1e-4, 1e-1) == pytest.approx(0.9 * 1e-6)
    assert ns.eisenstat_walker(0.9, 1.0, 1.0) == pytest.approx(0.9)

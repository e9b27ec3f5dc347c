"""GPU parity of Newton's method for the Navier-Stokes stage equations
(Section 3.2) with the oracle: lid-driven cavity, Radau IIA(2), nu = 1/100,
dt = 0.05.  For a seeded stage vector k the library's stage residual F(k),
Newton operator J(k) x and finest-level Vanka correction (patches cut from J,
whose velocity blocks depend on the row stage and couple the components)
match the oracle's; the inexact Newton solve (Eisenstat-Walker tolerances,
multigrid-preconditioned FGMRES) reaches the oracle's Newton root."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

N0, NL, S, DT, NU = 2, 4, 2, 0.05, 0.01


def _setup(irkmg):
    from oracle import mesh as M, ns, tableau, vanka
    A, b, c = irkmg.irkmg_radau_iia(S)
    o = irkmg.irkmg_default_options()
    o.nlevels = NL
    o.maxit = 400
    ctx = irkmg.irkmg_setup(*synth.square_mesh(N0), A, b, c, DT, NU, o)
    mesh = M.hierarchy(*synth.square_mesh(N0), NL)[-1]
    st = ns.NSStages(mesh, tableau.radau_iia(S)[0], DT, NU)
    X = mesh.p2_coords
    lx, ly = synth.lid_velocity(X[:, 0], X[:, 1])
    un = np.stack([lx, ly], axis=1)                       # [np2, 2]
    return ctx, st, un, vanka


def _stage_velocities(st, un, k):
    U, _ = st.stage_fields(un, np.zeros(st.nv), k)        # [s, np2, 2]
    return np.ascontiguousarray(np.transpose(U, (0, 2, 1)))  # [s, 2, np2]


def test_ns_residual_operator_and_vanka_match_oracle():
    irkmg = need_gpu()
    ctx, st, un, vanka = _setup(irkmg)
    try:
        k = 0.3 * synth.random_vector(41, st.N)
        k = st.project_pressure(k)
        pn = np.zeros(st.nv)
        f = np.zeros((S, st.mesh.np2, 2))
        irkmg.irkmg_ns_set_state(ctx, _stage_velocities(st, un, k))
        F = dev(np.zeros(st.N))
        irkmg.irkmg_ns_residual(ctx, dev(un.T.ravel()), dev(pn), dev(np.zeros(S * 2 * st.mesh.np2)),
                                dev(k), F)
        F_ref = st.residual(k, un, pn, f)
        assert rel(host(F), F_ref) < 1e-12
        J = st.jacobian(k, un, pn)
        x = synth.random_vector(42, st.N)
        y = dev(np.zeros(st.N))
        irkmg.irkmg_apply(ctx, dev(x), y)
        assert rel(host(y), J @ x) < 1e-12
        dofs = vanka.all_patch_dofs(st.mesh, S)
        V = vanka.Vanka(J, dofs)
        r = synth.random_vector(43, st.N)
        cc = dev(np.zeros(st.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), cc)
        assert rel(host(cc), V.correction(r)) < 1e-11
    finally:
        ctx.close()


def test_ns_newton_reaches_the_oracle_root():
    irkmg = need_gpu()
    from oracle import ns
    ctx, st, un, _ = _setup(irkmg)
    try:
        pn = np.zeros(st.nv)
        f = np.zeros((S, st.mesh.np2, 2))
        k_ref, hist, _ = ns.newton(st, un, pn, f, np.zeros(st.N), ns.bordered_solve(st), atol=1e-11)
        k = dev(np.zeros(st.N))
        stats = irkmg.irkmg_ns_newton(ctx, dev(un.T.ravel()), dev(pn),
                                      dev(np.zeros(S * 2 * st.mesh.np2)), k, atol=1e-11, maxit=20)
        assert stats["status"] == 0 and stats["ffinal"] <= 1e-11
        assert stats["newton_iters"] <= len(hist) + 3
        kk = host(k)
        mask = st.pressure_mask()
        assert rel(kk[~mask], k_ref[~mask]) < 1e-8
        assert rel(st.project_pressure(kk)[mask], st.project_pressure(k_ref)[mask]) < 1e-8
        assert np.linalg.norm(st.residual(kk, un, pn, f)) <= 1e-10
    finally:
        ctx.close()

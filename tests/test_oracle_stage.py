"""Pins for the oracle's IRK stage system, right-hand side and update
(Section 3.1, Kronecker form; Section 2, RK update and stability function;
index-2 DAE order limits)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem, mesh as M, stage, tableau


@pytest.mark.parametrize("s", [1, 2, 3])
def test_dahlquist_reduction(s):
    """One velocity DoF, no pressure: the stage solve + update must give
    u^{n+1} = r(-lam dt) u^n for every component."""
    A, b, _ = tableau.radau_iia(s)
    lam, dt = 3.7, 0.25
    ops = {"M": sp.csr_matrix([[1.0]]), "K": sp.csr_matrix([[lam]]),
           "Mall": sp.csr_matrix([[1.0]]), "B": sp.csr_matrix((2, 0))}
    J = stage.stage_matrix(ops, A, dt)
    un, pn = np.array([1.3, -0.4]), np.zeros(0)
    F = stage.stage_rhs(ops, un, pn, np.zeros((s, 2, 1)))
    k = spla.spsolve(J.tocsc(), F)
    u1, _ = stage.advance(k, un, pn, b, dt)
    np.testing.assert_allclose(u1, tableau.stability_function(A, b, -lam * dt) * un, rtol=1e-13)


def test_stage_blocks_and_null_space():
    A, _, _ = tableau.radau_iia(3)
    m = M.Mesh(*synth.square_mesh(3))
    ops = fem.assemble(m)
    J = stage.stage_matrix(ops, A, 0.1)
    mm = 2 * m.nf + m.nv
    # constant pressure in one stage and nothing else lies in the kernel of J
    for t in range(3):
        x = np.zeros(3 * mm)
        x[t * mm + 2 * m.nf:(t + 1) * mm] = 1.0
        assert np.abs(J @ x).max() < 1e-14
    # the (i, j) stage block is delta_ij Mt + dt a_ij St
    Mt, St = stage.single_stage_blocks(ops)
    Jd = J.toarray()
    for i in range(3):
        for j in range(3):
            blk = Jd[i * mm:(i + 1) * mm, j * mm:(j + 1) * mm]
            ref = (i == j) * Mt.toarray() + 0.1 * A[i, j] * St.toarray()
            assert np.abs(blk - ref).max() < 1e-15


def _run(n, s, nsteps, T, kind="exp"):
    A, b, c = tableau.radau_iia(s)
    m = M.Mesh(*synth.square_mesh(n))
    ops = fem.assemble(m)
    dt = T / nsteps
    J = stage.stage_matrix(ops, A, dt)
    mm = 2 * m.nf + m.nv
    # border the per-stage pressure constants so the solve is nonsingular
    Nm = np.zeros((s * mm, s))
    for t in range(s):
        Nm[t * mm + 2 * m.nf:(t + 1) * mm, t] = 1.0
    Jb = sp.bmat([[J, sp.csr_matrix(Nm)], [sp.csr_matrix(Nm.T), None]], format="csc")
    lu = spla.splu(Jb)
    X, Y = m.p2_coords.T
    xf, yf = X[m.free_p2], Y[m.free_p2]
    un = np.concatenate(synth.mms_velocity(xf, yf, 0.0, kind))
    pn = synth.mms_pressure(m.coords[:, 0], m.coords[:, 1], 0.0, kind)
    for step in range(nsteps):
        t0 = step * dt
        f = np.stack([np.stack(synth.mms_forcing(X, Y, t0 + ci * dt, 1.0, kind)) for ci in c])
        F = stage.stage_rhs(ops, un, pn, f)
        k = lu.solve(np.concatenate([F, np.zeros(s)]))[: s * mm]
        un, pn = stage.advance(k, un, pn, b, dt)
    return un, pn - pn.mean()


@pytest.mark.parametrize("s", [2, 3])
def test_temporal_self_convergence(s):
    """Fixed mesh, g(t) = exp(-t), self-convergence in dt.  For index-2 DAEs the
    order is limited by the stage order (Section 2), so the pin asks for a
    velocity rate of at least s (observed: about 2.3-3.9 for s=2, 4.6-8.5 for s=3)."""
    T = 0.5
    ref_u, ref_p = _run(4, s, 64, T)
    errs = []
    for N in (2, 4, 8):
        u, p = _run(4, s, N, T)
        errs.append((np.abs(u - ref_u).max(), np.abs(p - ref_p).max()))
    ru = [np.log2(errs[i][0] / errs[i + 1][0]) for i in range(2)]
    assert min(ru) > s - 0.3, (errs, ru)

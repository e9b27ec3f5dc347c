"""Pins for the oracle's P2-P1 element matrices and assembly (Section 3.1).

The reference integrals are checked against an independent Duffy-collapsed
Gauss-Legendre quadrature with hand-differentiated Cartesian basis functions;
global identities follow from partition of unity and the divergence theorem;
the steady manufactured solution pins the discretisation orders."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem, mesh as M


def _ref_basis(x, y):
    l0 = 1 - x - y
    phi = np.array([l0 * (2 * l0 - 1), x * (2 * x - 1), y * (2 * y - 1),
                    4 * x * l0, 4 * x * y, 4 * y * l0])
    dphi = np.array([[-(4 * l0 - 1), -(4 * l0 - 1)], [4 * x - 1, 0 * x], [0 * x, 4 * y - 1],
                     [4 * (1 - 2 * x - y), -4 * x], [4 * y, 4 * x], [-4 * y, 4 * (1 - x - 2 * y)]])
    psi = np.array([l0, x, y])
    return phi, dphi, psi


def _quad(npts=8):
    g, w = np.polynomial.legendre.leggauss(npts)
    g, w = (g + 1) / 2, w / 2
    U, V = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w)
    x, y = U, V * (1 - U)
    return x.ravel(), y.ravel(), (W * (1 - U)).ravel()


TRI = np.array([[0.1, 0.2], [0.9, 0.35], [0.3, 1.1]])


def _physical(tri):
    x, y, w = _quad()
    Jm = np.stack([tri[1] - tri[0], tri[2] - tri[0]], axis=1)   # [2x2]
    detJ = abs(np.linalg.det(Jm))
    Jinv = np.linalg.inv(Jm)
    phi, dphi, psi = _ref_basis(x, y)
    grad = np.einsum("kd,adq->akq", Jinv.T, dphi)              # physical gradients
    return phi, grad, psi, w * detJ


def test_element_matrices_match_independent_quadrature():
    phi, grad, psi, w = _physical(TRI)
    Mq = np.einsum("aq,bq,q->ab", phi, phi, w)
    Kq = np.einsum("akq,bkq,q->ab", grad, grad, w)
    Bq = -np.einsum("qp,adp,p->daq", psi, grad, w)             # [d, a, q]
    Me, Ke, Be = fem.element_matrices(TRI, np.array([[0, 1, 2]]))
    np.testing.assert_allclose(Me[0], Mq, atol=1e-15)
    np.testing.assert_allclose(Ke[0], Kq, atol=2e-14)
    np.testing.assert_allclose(Be[0], Bq, atol=1e-15)


def test_convection_matches_independent_quadrature():
    rng = np.random.default_rng(3)
    wnod = rng.standard_normal((6, 2))
    phi, grad, psi, w = _physical(TRI)
    wq = np.einsum("cq,cd->dq", phi, wnod)
    Cq = np.einsum("dq,bdq,aq,q->ab", wq, grad, phi, w)
    Ce = fem.convection_matrices(TRI, np.array([[0, 1, 2]]), np.arange(6)[None], wnod)
    np.testing.assert_allclose(Ce[0], Cq, atol=1e-14)


@pytest.mark.parametrize("n", [2, 5])
def test_global_identities(n):
    m = M.Mesh(*synth.square_mesh(n))
    ops = fem.assemble(m)
    assert abs(ops["Mfull"].sum() - 1.0) < 1e-14                # partition of unity: area
    assert np.abs(ops["Kfull"] @ np.ones(m.np2)).max() < 1e-12   # K 1 = 0
    assert np.abs(ops["B"] @ np.ones(m.nv)).max() < 1e-14        # B 1_p = 0 on free rows
    # discrete divergence of a linear field is exact: -(a+e) int psi_q
    a, bb, c, d, e, f = 0.3, -1.2, 0.5, 0.7, 2.1, -0.4
    X, Y = m.p2_coords[:, 0], m.p2_coords[:, 1]
    ux, uy = a * X + bb * Y + c, d * X + e * Y + f
    div = ops["Bfull"][0].T @ ux + ops["Bfull"][1].T @ uy
    area = 0.5 / n ** 2
    star = np.bincount(m.cells.ravel(), minlength=m.nv) * area
    np.testing.assert_allclose(div, -(a + e) * star / 3.0, atol=1e-13)


def _steady_stokes_errors(n):
    m = M.Mesh(*synth.square_mesh(n))
    ops = fem.assemble(m)
    X, Y = m.p2_coords[:, 0], m.p2_coords[:, 1]
    fx, fy = synth.mms_forcing(X, Y)
    K2 = sp.block_diag([ops["K"], ops["K"]])
    B = ops["B"]
    one = np.ones((m.nv, 1))
    S = sp.bmat([[K2, B, None], [B.T, None, sp.csr_matrix(one)], [None, sp.csr_matrix(one.T), None]],
                format="csc")
    rhs = np.concatenate([ops["Mall"] @ fx, ops["Mall"] @ fy, np.zeros(m.nv + 1)])
    sol = spla.spsolve(S, rhs)
    uh, ph = sol[: 2 * m.nf], sol[2 * m.nf: 2 * m.nf + m.nv]
    xf, yf = m.p2_coords[m.free_p2, 0], m.p2_coords[m.free_p2, 1]
    ux, uy = synth.mms_velocity(xf, yf)
    eu = uh - np.concatenate([ux, uy])
    M2 = sp.block_diag([ops["M"], ops["M"]])
    pe = ph - synth.mms_pressure(m.coords[:, 0], m.coords[:, 1])
    pe -= pe.mean()
    return np.sqrt(eu @ (M2 @ eu)), np.sqrt(np.mean(pe ** 2))


def test_steady_mms_orders():
    e = [_steady_stokes_errors(n) for n in (4, 8, 16)]
    ru = np.log2(e[1][0] / e[2][0])
    rp = np.log2(e[1][1] / e[2][1])
    assert ru > 2.8, (e, ru)       # P2 velocity: O(h^3) in L2
    assert rp > 1.8, (e, rp)       # P1 pressure: O(h^2)

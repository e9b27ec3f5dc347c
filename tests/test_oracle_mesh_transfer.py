"""Pins for the oracle's mesh hierarchy, numbering and grid transfers
(Section 4.1: uniform refinement; canonical P2/P1 interpolation, I_s (x) P,
restriction = transpose; rediscretised coarse operators are Galerkin)."""
import numpy as np
import pytest

import synth
from oracle import fem, mesh as M, mg, stage, tableau, transfer


@pytest.mark.parametrize("n", [1, 2, 3, 8])
def test_counts(n):
    m = M.Mesh(*synth.square_mesh(n))
    assert m.nv == (n + 1) ** 2 and m.nc == 2 * n * n
    assert m.ne == 3 * n * n + 2 * n                      # Euler: V - E + F = 1
    assert m.nf == (2 * n - 1) ** 2                       # interior of the half-grid
    assert np.all(m.p2_dirichlet == ((m.p2_coords == 0) | (m.p2_coords == 1)).any(axis=1))


def test_refinement_is_the_structured_mesh_at_half_h():
    ms = M.hierarchy(*synth.square_mesh(2), 3)
    for l in range(2):
        # P2 nodes of level l are the vertices of level l+1, same ids and places
        np.testing.assert_array_equal(ms[l].p2_coords, ms[l + 1].coords)
        np.testing.assert_array_equal(ms[l].p2_dirichlet, ms[l + 1].bnd)
    ref = M.Mesh(*synth.square_mesh(8))
    f = ms[2]
    key = lambda m: set(map(tuple, np.round(np.sort(m.coords[m.cells], axis=1).reshape(m.nc, -1) * 64).astype(int)))
    assert key(f) == key(ref)
    assert f.nf == ref.nf and f.ne == ref.ne


def _quadratic(x, y):
    return 1.0 + 2 * x - 3 * y + 0.5 * x * x - 1.5 * x * y + 2.5 * y * y


def test_prolongation_reproduces_polynomials():
    ms = M.hierarchy(*synth.square_mesh(3), 2)
    P2, P1 = transfer.prolongation_full(ms[0], ms[1])
    qc = _quadratic(*ms[0].p2_coords.T)
    qf = _quadratic(*ms[1].p2_coords.T)
    np.testing.assert_allclose(P2 @ qc, qf, atol=1e-13)
    lc = 0.3 + 1.7 * ms[0].coords[:, 0] - 0.9 * ms[0].coords[:, 1]
    lf = 0.3 + 1.7 * ms[1].coords[:, 0] - 0.9 * ms[1].coords[:, 1]
    np.testing.assert_allclose(P1 @ lc, lf, atol=1e-14)
    assert np.allclose(P2.sum(axis=1), 1.0) and np.allclose(P1.sum(axis=1), 1.0)


@pytest.mark.parametrize("s,dt,nu", [(2, 1 / 8, 1.0), (3, 1 / 64, 0.37)])
def test_galerkin_identity(s, dt, nu):
    """Rediscretisation equals Galerkin coarsening for nested P2/P1 spaces with
    exact integration (Section 4.1): (I_s (x) P)^T J_f (I_s (x) P) = J_c."""
    A, _, _ = tableau.radau_iia(s)
    H = mg.Hierarchy(*synth.square_mesh(2), 3, A, dt, nu=nu, build_patches=False)
    for l in (1, 2):
        G = (H.levels[l].P.T @ H.levels[l].J @ H.levels[l].P).toarray()
        Jc = H.levels[l - 1].J.toarray()
        assert np.abs(G - Jc).max() <= 1e-14 * np.abs(Jc).max()


def test_galerkin_identity_oseen():
    """The same identity with the convection term, the wind injected (coarse P2
    nodes are fine P2 nodes with the same ids)."""
    A, _, _ = tableau.radau_iia(2)
    ms = M.hierarchy(*synth.square_mesh(2), 2)
    X, Y = ms[1].p2_coords.T
    # a globally quadratic wind is represented exactly on both levels
    wq = np.stack([_quadratic(X, Y), 0.5 - X * Y], axis=1)
    H = mg.Hierarchy(*synth.square_mesh(2), 2, A, 0.1, nu=0.01, wind_finest=wq, build_patches=False)
    G = (H.levels[1].P.T @ H.levels[1].J @ H.levels[1].P).toarray()
    Jc = H.levels[0].J.toarray()
    assert np.abs(G - Jc).max() <= 1e-13 * np.abs(Jc).max()

"""Pins for the oracle's vertex-star Vanka patches, colouring and relaxation
(Section 4.2, Fig. 1; Section 5.1 Chebyshev acceleration)."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import mesh as M, mg, tableau, vanka


def _in_closed_star(m, v, pts):
    """Geometric test: is each point inside one of the triangles around v?"""
    inside = np.zeros(len(pts), dtype=bool)
    for c in np.nonzero((m.cells == v).any(axis=1))[0]:
        x = m.coords[m.cells[c]]
        T = np.stack([x[1] - x[0], x[2] - x[0]], 1)
        lam = np.linalg.solve(T, (pts - x[0]).T).T
        inside |= (lam >= -1e-12).all(1) & (lam.sum(1) <= 1 + 1e-12)
    return inside


@pytest.mark.parametrize("n", [3, 4])
def test_patch_nodes_match_geometric_definition(n):
    m = M.Mesh(*synth.square_mesh(n))
    nodes = vanka.patch_nodes(m)
    free_pts = m.p2_coords[m.free_p2]
    for v in range(m.nv):
        geo = np.nonzero(_in_closed_star(m, v, free_pts))[0]
        np.testing.assert_array_equal(nodes[v], geo)


def test_patch_sizes_hand_counted():
    """Interior vertex of the 2-triangle-per-square mesh: 6 triangles, 7
    vertices and 12 edges in the closed star -> 19 P2 nodes, 38 velocity + 1
    pressure DoFs per stage (Fig. 1 left): 78 for s=2, 117 for s=3."""
    m = M.Mesh(*synth.square_mesh(6))
    v = 3 + 7 * 3
    nodes = vanka.patch_nodes(m)[v]
    assert nodes.size == 19
    assert vanka.patch_dofs(m, nodes, v, 2).size == 78
    assert vanka.patch_dofs(m, nodes, v, 3).size == 117
    assert max(len(x) for x in vanka.patch_nodes(m)) == 19


def test_colouring_valid_and_greedy():
    m = M.Mesh(*synth.square_mesh(7))
    col = vanka.distance2_colouring(m)
    dofs = vanka.all_patch_dofs(m, 1)
    owner = {}
    for v, d in enumerate(dofs):                         # same-colour patches share no DoF
        for i in d:
            owner.setdefault(i, []).append(v)
    for vs in owner.values():
        cs = col[vs]
        assert len(set(cs.tolist())) == len(cs)
    # greedy in id order: colour = smallest not used by lower-id vertices within distance 2
    nb = m.vertex_neighbours()
    for v in range(m.nv):
        near = set(nb[v].tolist())
        for w in nb[v]:
            near.update(nb[w].tolist())
        near.discard(v)
        lower = {col[w] for w in near if w < v}
        assert col[v] not in lower and all(c in lower for c in range(col[v]))
    assert col.max() + 1 >= 7                             # dist-2 clique of the lattice has 7


def test_additive_correction_equals_explicit_sum():
    A, _, _ = tableau.radau_iia(2)
    H = mg.Hierarchy(*synth.square_mesh(2), 2, A, 0.125, build_patches=True)
    L = H.finest
    Jd = L.J.toarray()
    Dinv = np.zeros_like(Jd)
    for idx in L.dofs:
        R = np.zeros((idx.size, L.N))
        R[np.arange(idx.size), idx] = 1.0
        Dinv += R.T @ np.linalg.inv(R @ Jd @ R.T) @ R
    r = synth.random_vector(5, L.N)
    np.testing.assert_allclose(L.vanka.correction(r), Dinv @ r, rtol=1e-10, atol=1e-10)


def test_chebyshev_is_the_scaled_chebyshev_polynomial():
    """With D^{-1} J = diag(lam) and F = 0, nu steps map x0 to
    T_nu((theta - lam)/delta) / T_nu(theta/delta) x0."""
    lam = np.linspace(0.1, 9.0, 40)

    class Diag(vanka.Vanka):
        def __init__(self):
            pass

        def correction(self, r):
            return r.copy()

    J = np.diag(lam) * 1.0
    x0 = np.ones_like(lam)
    lo, hi = 2.0, 8.0
    theta, delta = 5.0, 3.0
    for nu in (1, 2, 3, 4):
        x = Diag().chebyshev(J, np.zeros_like(lam), x0, nu, lo, hi)
        T = np.polynomial.chebyshev.Chebyshev.basis(nu)
        np.testing.assert_allclose(x, T((theta - lam) / delta) / T(theta / delta), atol=1e-13)


def test_smoother_spectrum_matches_paper_interval():
    """The largest real part of the spectrum of the Vanka-preconditioned stage
    operator sits near 8, the top of the paper's hand-tuned Chebyshev interval
    [2, 8] (Section 5.1)."""
    A, _, _ = tableau.radau_iia(2)
    H = mg.Hierarchy(*synth.square_mesh(2), 2, A, 0.125)
    L = H.finest
    Jd = L.J.toarray()
    DJ = np.stack([L.vanka.correction(Jd[:, j]) for j in range(L.N)], axis=1)
    ev = np.linalg.eigvals(DJ)
    assert 7.0 < ev.real.max() < 8.5


@pytest.mark.parametrize("fam,s,dt,wind", [("radau_iia", 3, 1 / 64, False), ("gauss", 2, 1 / 8, False),
                                           ("lobatto_iiic", 3, 1 / 16, True)])
def test_patch_system_decouples_by_eigenvectors_of_A(fam, s, dt, wind):
    """A patch cut from the assembled stage operator has the Kronecker form
    I_s ⊗ M̃ + dt A ⊗ K̃ (Section 3 and the patch definition of Section 4.2),
    so with A = V Λ V⁻¹ (LAPACK eig) its inverse is
    (V ⊗ I) diag((M̃ + dt λ_k K̃)⁻¹) (V⁻¹ ⊗ I).  Checked on every patch of an
    8x8 level, Stokes and (LobattoIIIC) Oseen with a seeded wind."""
    from oracle import stage
    A = getattr(tableau, fam)(s)[0]
    coords, cells, bnd = synth.square_mesh(2)
    w = None
    if wind:
        fine = M.hierarchy(coords, cells, bnd, 2)[-1]
        wx, wy = synth.wind_field(fine.p2_coords[:, 0], fine.p2_coords[:, 1],
                                  synth.wind_coefficients(7))
        w = np.stack([wx, wy], axis=1) / np.max(np.hypot(wx, wy))
    H = mg.Hierarchy(coords, cells, bnd, 2, A, dt, nu=1.0 / 300 if wind else 1.0, wind_finest=w)
    L = H.levels[-1]
    Mt, St = stage.single_stage_blocks(L.ops)
    lam, V = np.linalg.eig(A)
    Vi = np.linalg.inv(V)
    J = L.J.tocsr()
    worst = 0.0
    for idx in L.dofs:
        n = len(idx) // s
        one = idx[:n]
        Mv = Mt[one][:, one].toarray()
        Kv = St[one][:, one].toarray()
        Av = J[idx][:, idx].toarray()
        blocks = [np.linalg.inv(Mv + dt * l * Kv) for l in lam]
        Xd = np.kron(V, np.eye(n)) @ sla.block_diag(*blocks) @ np.kron(Vi, np.eye(n))
        X = np.linalg.inv(Av)
        assert np.abs(Xd.imag).max() < 1e-10 * np.abs(X).max()
        worst = max(worst, np.abs(Xd.real - X).max() / np.abs(X).max())
    assert worst < 1e-11


def test_ritz_estimate_finds_the_largest_eigenvalue_of_the_preconditioned_operator():
    """Section 5.1's estimate: 20 Arnoldi steps on D^{-1}J give the largest
    real part of its spectrum (dense eigenvalues of the explicit D^{-1}J) to
    1%, and [λ/4, λ] lands near the paper's hand-tuned [2, 8] for 2D Stokes."""
    A = tableau.radau_iia(2)[0]
    H = mg.Hierarchy(*synth.square_mesh(2), 2, A, 1 / 8)
    L = H.finest
    lam, ritz = H.ritz_estimate(1, 20)
    DJ = np.column_stack([L.vanka.correction(L.J[:, i].toarray().ravel()) for i in range(L.N)])
    ev = np.linalg.eigvals(DJ)
    assert abs(lam - ev.real.max()) <= 0.01 * ev.real.max()
    assert 6.5 < lam < 9.0
    assert len(ritz) == 20

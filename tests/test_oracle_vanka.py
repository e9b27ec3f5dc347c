"""Pins for the oracle's vertex-star Vanka patches, colouring and relaxation
(Section 4.2, Fig. 1; Section 5.1 Chebyshev acceleration)."""
import numpy as np
import pytest

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

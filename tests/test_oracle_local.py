"""Pins for oracle/local.py: the rows of J and the Vanka patch systems built
from the element matrices of the cells around the sampled nodes equal the
ones cut out of the globally assembled stage matrix (Section 3.1, 4.2), on
2D and 3D hierarchies and for s = 2, 3; the local Vanka entries equal
oracle.vanka's correction."""
import numpy as np
import pytest

import synth
from oracle import fem, local, mesh, stage, tableau, vanka


def _global(msh, A, dt):
    ops = fem.assemble(msh)
    return stage.stage_matrix(ops, A, dt).tocsr()


@pytest.mark.parametrize("dim,n0,nl,s,dt", [(2, 2, 3, 3, 1 / 64), (2, 2, 2, 2, 1 / 8),
                                            (3, 2, 1, 2, 1 / 16)])
def test_local_rows_and_patches_equal_the_assembled_matrix(dim, n0, nl, s, dt):
    make = synth.square_mesh if dim == 2 else synth.cube_mesh
    msh = mesh.hierarchy(*make(n0), nl)[-1]
    A, _, _ = tableau.radau_iia(s)
    J = _global(msh, A, dt)
    L = local.LocalStage(msh, A, dt)
    assert L.N == J.shape[0]
    rng = np.random.default_rng(7)
    rows = rng.choice(L.N, size=min(60, L.N), replace=False)
    for i in rows:
        ref = J.getrow(i)
        got = L.row(i)
        dense_ref = dict(zip(ref.indices.tolist(), ref.data.tolist()))
        keys = set(got) | {j for j, a in dense_ref.items() if a != 0.0}
        for j in keys:
            a, b = got.get(j, 0.0), dense_ref.get(j, 0.0)
            assert abs(a - b) <= 1e-14 * max(1.0, abs(b)) + 1e-15 * abs(J[i].toarray()).max(), (i, j, a, b)
    x = rng.standard_normal(L.N)
    y, _ = L.apply_rows(rows, x)
    np.testing.assert_allclose(y, (J @ x)[rows], rtol=1e-12, atol=1e-13 * np.abs(J @ x).max())
    # Stokes: [[M, 0], [0, 0]] and [[K, B], [B^T, 0]] are symmetric, so the rows
    # of J^T are those of the same system with A^T
    LT = local.LocalStage(msh, A.T, dt)
    yt, _ = LT.apply_rows(rows, x)
    np.testing.assert_allclose(yt, (J.T @ x)[rows], rtol=1e-12, atol=1e-13 * np.abs(J.T @ x).max())
    nodes = vanka.patch_nodes(msh)
    for v in rng.choice(msh.nv, size=min(8, msh.nv), replace=False):
        Av, idx = L.patch_matrix(int(v))
        np.testing.assert_array_equal(idx, vanka.patch_dofs(msh, nodes[v], v, s))
        ref = J[idx][:, idx].toarray()
        assert np.abs(Av - ref).max() <= 1e-14 * np.abs(ref).max()


def test_local_vanka_entries_equal_the_oracle_correction():
    msh = mesh.hierarchy(*synth.square_mesh(2), 3)[-1]
    A, _, _ = tableau.radau_iia(3)
    dt = 1 / 64
    J = _global(msh, A, dt)
    V = vanka.Vanka(J, vanka.all_patch_dofs(msh, 3))
    L = local.LocalStage(msh, A, dt)
    r = synth.random_vector(31, L.N)
    full = V.correction(r)
    rows = np.random.default_rng(3).choice(L.N, size=40, replace=False)
    got = L.vanka_entries(rows, r)
    np.testing.assert_allclose(got, full[rows], rtol=1e-11, atol=1e-12 * np.abs(full).max())
    # a DoF is in the patches of the vertices of the cells around its node
    for i in rows:
        pv = {v for v, idx in enumerate(V.dofs) if i in set(idx.tolist())}
        assert pv == set(L.patches_containing(i).tolist())

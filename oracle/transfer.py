"""Grid transfers (Section 4.1): prolongation is canonical finite-element
interpolation, P = diag(P_u, P_p) with P_u the P2 interpolation (for each
velocity component) and P_p the P1 interpolation; for s stages it is
I_s (x) P, and restriction is its transpose.

P_u[f, c] is the value of coarse P2 basis function c at fine node f, found by
locating each fine node in its parent cell (child cell 4c+k, or 8c+k in 3D,
has parent c) and evaluating the parent's P2 basis functions at the node's
barycentric coordinates.  Only free (non-Dirichlet) nodes are kept: coarse
Dirichlet basis functions carry zero coefficients.
"""
import numpy as np
import scipy.sparse as sp


def _barycentric(coords_parent, pts):
    """Barycentric coordinates of pts in the parent simplices (by solving
    [x_1 - x_0 ... x_d - x_0] l = p - x_0)."""
    d = pts.shape[1]
    Jm = np.stack([coords_parent[:, i + 1] - coords_parent[:, 0] for i in range(d)], axis=2)
    lam = np.linalg.solve(Jm, (pts - coords_parent[:, 0])[..., None])[..., 0]
    return np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)


def _p2_values(lam):
    from .mesh import LOCAL_EDGES
    d = lam.shape[1] - 1
    V = [lam[:, i] * (2 * lam[:, i] - 1) for i in range(d + 1)]
    E = [4 * lam[:, a] * lam[:, b] for a, b in LOCAL_EDGES[d]]
    return np.stack(V + E, axis=1)


def _unique_entries(rows, cols, vals, shape):
    key = rows * shape[1] + cols
    _, first = np.unique(key, return_index=True)
    rows, cols, vals = rows[first], cols[first], vals[first]
    keep = np.abs(vals) > 1e-12
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=shape)


def prolongation(coarse, fine):
    """Return (Pu, Pp): Pu is nf_fine x nf_coarse (scalar P2, free nodes only),
    Pp is nv_fine x nv_coarse (P1)."""
    P2, Pp = prolongation_full(coarse, fine)
    return P2[fine.free_p2][:, coarse.free_p2].tocsr(), Pp


def prolongation_full(coarse, fine):
    """Interpolation between all P2 nodes (np2_fine x np2_coarse) and all
    vertices (P1)."""
    kids = 2 ** fine.dim
    parent = np.arange(fine.nc) // kids
    pc = coarse.coords[coarse.cells[parent]]            # [ncf, d+1, d]
    nn = fine.cell_p2.shape[1]
    rows, cols, vals = [], [], []
    for a in range(nn):
        fnode = fine.cell_p2[:, a]
        lam = _barycentric(pc, fine.p2_coords[fnode])
        phi = _p2_values(lam)
        for b in range(nn):
            rows.append(fnode)
            cols.append(coarse.cell_p2[parent, b])
            vals.append(phi[:, b])
    P2 = _unique_entries(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                         (fine.np2, coarse.np2))
    rows, cols, vals = [], [], []
    for a in range(fine.dim + 1):
        fv = fine.cells[:, a]
        lam = _barycentric(pc, fine.coords[fv])
        for b in range(fine.dim + 1):
            rows.append(fv)
            cols.append(coarse.cells[parent, b])
            vals.append(lam[:, b])
    Pp = _unique_entries(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                         (fine.nv, coarse.nv))
    return P2, Pp


def stage_prolongation(Pu, Pp, s, dim=2):
    """I_s (x) diag(Pu, ..., Pu, Pp) (dim copies of Pu)."""
    one = sp.block_diag([Pu] * dim + [Pp], format="csr")
    return sp.kron(sp.identity(s), one, format="csr")

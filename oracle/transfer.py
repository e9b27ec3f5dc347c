"""Grid transfers (Section 4.1): prolongation is canonical finite-element
interpolation, P = diag(P_u, P_p) with P_u the P2 interpolation (for each
velocity component) and P_p the P1 interpolation; for s stages it is
I_s (x) P, and restriction is its transpose.

P_u[f, c] is the value of coarse P2 basis function c at fine node f, found by
locating each fine node in its parent cell (child cell 4c+k has parent c) and
evaluating the parent's six basis functions at the node's barycentric
coordinates.  Only free (non-Dirichlet) nodes are kept: coarse Dirichlet basis
functions carry zero coefficients.
"""
import numpy as np
import scipy.sparse as sp


def _barycentric(coords_parent, pts):
    x0, x1, x2 = coords_parent[:, 0], coords_parent[:, 1], coords_parent[:, 2]
    d1, d2, r = x1 - x0, x2 - x0, pts - x0
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    l1 = (r[:, 0] * d2[:, 1] - r[:, 1] * d2[:, 0]) / det
    l2 = (d1[:, 0] * r[:, 1] - d1[:, 1] * r[:, 0]) / det
    return np.stack([1.0 - l1 - l2, l1, l2], axis=1)


def _p2_values(lam):
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    return np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                     4 * l0 * l1, 4 * l1 * l2, 4 * l0 * l2], axis=1)


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
    parent = np.arange(fine.nc) // 4
    pc = coarse.coords[coarse.cells[parent]]            # [ncf, 3, 2]
    rows, cols, vals = [], [], []
    for a in range(6):
        fnode = fine.cell_p2[:, a]
        lam = _barycentric(pc, fine.p2_coords[fnode])
        phi = _p2_values(lam)
        for b in range(6):
            rows.append(fnode)
            cols.append(coarse.cell_p2[parent, b])
            vals.append(phi[:, b])
    P2 = _unique_entries(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                         (fine.np2, coarse.np2))
    rows, cols, vals = [], [], []
    for a in range(3):
        fv = fine.cells[:, a]
        lam = _barycentric(pc, fine.coords[fv])
        for b in range(3):
            rows.append(fv)
            cols.append(coarse.cells[parent, b])
            vals.append(lam[:, b])
    Pp = _unique_entries(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                         (fine.nv, coarse.nv))
    return P2, Pp


def stage_prolongation(Pu, Pp, s):
    """I_s (x) diag(Pu, Pu, Pp)."""
    one = sp.block_diag([Pu, Pu, Pp], format="csr")
    return sp.kron(sp.identity(s), one, format="csr")

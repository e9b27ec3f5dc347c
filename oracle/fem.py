"""Taylor-Hood P2-P1 element matrices and global assembly (Section 3.1: the
semi-discrete system [M u_t; 0] + [[K, B], [B^T, 0]] [u; p] = [M f; 0], with M
and K the (P2)^d mass and stiffness matrices and B the weak gradient coming from
-<p, div v>; Section 3.2: the Navier-Stokes convection term, here linearised
about a frozen wind w (Oseen), <(w . grad) u, v>).

All integrals are exact: every integrand is a polynomial in the barycentric
coordinates lambda of an affine triangle T, and
    int_T lambda_0^a lambda_1^b lambda_2^c dx = 2 |T| a! b! c! / (a+b+c+2)!.
"""
from math import factorial
import numpy as np
import scipy.sparse as sp

# A polynomial in (l0, l1, l2) is a dict {(a, b, c): coefficient}.


def _mul(p, q):
    r = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            r[e] = r.get(e, 0.0) + ca * cb
    return r


def _add(p, q, s=1.0):
    r = dict(p)
    for e, c in q.items():
        r[e] = r.get(e, 0.0) + s * c
    return r


def _diff(p, i):
    r = {}
    for e, c in p.items():
        if e[i] > 0:
            f = list(e)
            f[i] -= 1
            r[tuple(f)] = r.get(tuple(f), 0.0) + c * e[i]
    return r


def _integral_over_area(p):
    """int_T p / |T|."""
    tot = 0.0
    for (a, b, c), coef in p.items():
        tot += coef * 2.0 * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)
    return tot


def _lam(i):
    e = [0, 0, 0]
    e[i] = 1
    return {tuple(e): 1.0}


ONE = {(0, 0, 0): 1.0}
# P2 basis, local order: vertices 0,1,2, then edges (0,1), (1,2), (0,2)
P2 = [_mul(_lam(i), _add(_mul({(0, 0, 0): 2.0}, _lam(i)), ONE, -1.0)) for i in range(3)]
P2 += [_mul({(0, 0, 0): 4.0}, _mul(_lam(a), _lam(b))) for a, b in [(0, 1), (1, 2), (0, 2)]]
P1 = [_lam(i) for i in range(3)]

# Reference tensors (divided by |T|); geometry enters via grad(lambda).
MREF = np.array([[_integral_over_area(_mul(P2[a], P2[b])) for b in range(6)] for a in range(6)])
# KREF[i, j, a, b] = int d_i phi_a d_j phi_b / |T|   (d_i = d/d lambda_i)
KREF = np.array([[[[_integral_over_area(_mul(_diff(P2[a], i), _diff(P2[b], j)))
                    for b in range(6)] for a in range(6)] for j in range(3)] for i in range(3)])
# BREF[i, a, q] = int psi_q d_i phi_a / |T|
BREF = np.array([[[_integral_over_area(_mul(P1[q], _diff(P2[a], i))) for q in range(3)]
                  for a in range(6)] for i in range(3)])
# CREF[c, i, b, a] = int phi_c d_i phi_b phi_a / |T|   (wind node c)
CREF = np.array([[[[_integral_over_area(_mul(_mul(P2[c], _diff(P2[b], i)), P2[a]))
                    for a in range(6)] for b in range(6)] for i in range(3)] for c in range(6)])


def geometry(coords, cells):
    """Areas and barycentric gradients: G[e, i, :] = grad lambda_i on cell e."""
    x = coords[cells]                                  # [nc, 3, 2]
    d1 = x[:, 1] - x[:, 0]
    d2 = x[:, 2] - x[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    area = 0.5 * np.abs(det)
    # lambda_1 = ((x-x0) x d2)/det ... solve the 2x2 system per cell
    g1 = np.stack([d2[:, 1], -d2[:, 0]], 1) / det[:, None]
    g2 = np.stack([-d1[:, 1], d1[:, 0]], 1) / det[:, None]
    g0 = -g1 - g2
    return area, np.stack([g0, g1, g2], axis=1)


def element_matrices(coords, cells):
    """Per-cell scalar P2 mass Me [nc,6,6], stiffness Ke [nc,6,6] and weak-gradient
    blocks Be [nc,2,6,3]: Be[e,d,a,q] = -int psi_q d(phi_a)/dx_d."""
    area, G = geometry(coords, cells)
    Me = area[:, None, None] * MREF[None]
    GG = np.einsum("eid,ejd->eij", G, G)
    Ke = area[:, None, None] * np.einsum("eij,ijab->eab", GG, KREF)
    Be = -area[:, None, None, None] * np.einsum("eid,iaq->edaq", G, BREF)
    return Me, Ke, Be


def convection_matrices(coords, cells, cell_p2, wind):
    """Oseen term per cell: Ce[e, a, b] = int (w . grad phi_b) phi_a, with w the
    P2 interpolant of the nodal wind [np2, 2]."""
    area, G = geometry(coords, cells)
    wl = wind[cell_p2]                                 # [nc, 6, 2]
    # (w . grad) phi_b = sum_c sum_d w_c^d phi_c sum_i G_id d_i phi_b
    WG = np.einsum("ecd,eid->eci", wl, G)
    Ce = area[:, None, None] * np.einsum("eci,ciba->eab", WG, CREF)
    return Ce


def assemble(mesh, nu=1.0, wind=None):
    """Global free-DoF matrices of one level.

    Returns dict with scalar P2 blocks on free nodes: M, K (nu * stiffness
    [+ convection]); the all-column mass Mall (free rows x all P2 nodes, used for
    M f with f the interpolant at every node); Kall (free rows x all P2 nodes);
    and B as a (2 nf) x nv matrix (rows: u_x free nodes then u_y free nodes).
    """
    Me, Ke, Be = element_matrices(mesh.coords, mesh.cells)
    Ve = nu * Ke
    if wind is not None:
        Ve = Ve + convection_matrices(mesh.coords, mesh.cells, mesh.cell_p2, wind)
    nodes = mesh.cell_p2
    r = np.repeat(nodes, 6, axis=1).ravel()
    c = np.tile(nodes, (1, 6)).ravel()
    shape = (mesh.np2, mesh.np2)
    Mfull = sp.coo_matrix((Me.ravel(), (r, c)), shape=shape).tocsr()
    Vfull = sp.coo_matrix((Ve.ravel(), (r, c)), shape=shape).tocsr()
    fr = mesh.free_p2
    out = {
        "M": Mfull[fr][:, fr].tocsr(),
        "K": Vfull[fr][:, fr].tocsr(),
        "Mall": Mfull[fr].tocsr(),
        "Kall": Vfull[fr].tocsr(),
    }
    rb = np.repeat(nodes, 3, axis=1).ravel()
    cb = np.tile(mesh.cells, (1, 6)).ravel()
    Bd = []
    for d in range(2):
        Bfull = sp.coo_matrix((Be[:, d].ravel(), (rb, cb)), shape=(mesh.np2, mesh.nv)).tocsr()
        Bd.append(Bfull[fr])
    out["B"] = sp.vstack(Bd).tocsr()
    out["Bfull"] = [sp.coo_matrix((Be[:, d].ravel(), (rb, cb)), shape=(mesh.np2, mesh.nv)).tocsr()
                    for d in range(2)]            # every P2 row, per component
    out["Mfull"] = Mfull
    out["Kfull"] = Vfull
    return out

"""Taylor-Hood P2-P1 element matrices and global assembly (Section 3.1: the
semi-discrete system [M u_t; 0] + [[K, B], [B^T, 0]] [u; p] = [M f; 0], with M
and K the (P2)^d mass and stiffness matrices and B the weak gradient coming from
-<p, div v>; Section 3.2: the Navier-Stokes convection term, here linearised
about a frozen wind w (Oseen), <(w . grad) u, v>).

All integrals are exact: every integrand is a polynomial in the barycentric
coordinates lambda of an affine d-simplex T, and
    int_T prod_i lambda_i^a_i dx = d! |T| prod_i a_i! / (sum_i a_i + d)!.
The module-level tensors MREF, KREF, BREF, CREF are those of the triangle;
reference_tensors(d) gives them for any d.
"""
from math import factorial
import numpy as np
import scipy.sparse as sp

# A polynomial in (l0, l1, l2) is a dict {(a, b, c): coefficient}.


def _mul(p, q):
    r = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
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
    """int_T p / |T| over a simplex of dimension len(exponents) - 1."""
    tot = 0.0
    for e, coef in p.items():
        d = len(e) - 1
        num = factorial(d)
        for a in e:
            num *= factorial(a)
        tot += coef * num / factorial(sum(e) + d)
    return tot


def _lam(i, d=2):
    e = [0] * (d + 1)
    e[i] = 1
    return {tuple(e): 1.0}


def _const(v, d=2):
    return {tuple([0] * (d + 1)): v}


def p2_basis(d):
    """P2 basis on the d-simplex: vertices lambda_i (2 lambda_i - 1), then edge
    functions 4 lambda_a lambda_b in the local edge order of the mesh module."""
    from .mesh import LOCAL_EDGES
    V = [_mul(_lam(i, d), _add(_mul(_const(2.0, d), _lam(i, d)), _const(1.0, d), -1.0))
         for i in range(d + 1)]
    E = [_mul(_const(4.0, d), _mul(_lam(a, d), _lam(b, d))) for a, b in LOCAL_EDGES[d]]
    return V + E


_REF = {}


def reference_tensors(d):
    """(MREF, KREF, BREF, CREF) of the d-simplex, each divided by |T|."""
    if d in _REF:
        return _REF[d]
    P2_ = p2_basis(d)
    P1_ = [_lam(i, d) for i in range(d + 1)]
    n, k = len(P2_), d + 1
    I = _integral_over_area
    M = np.array([[I(_mul(P2_[a], P2_[b])) for b in range(n)] for a in range(n)])
    K = np.array([[[[I(_mul(_diff(P2_[a], i), _diff(P2_[b], j))) for b in range(n)]
                    for a in range(n)] for j in range(k)] for i in range(k)])
    B = np.array([[[I(_mul(P1_[q], _diff(P2_[a], i))) for q in range(k)] for a in range(n)]
                  for i in range(k)])
    C = None
    if d == 2:
        C = np.array([[[[I(_mul(_mul(P2_[c], _diff(P2_[b], i)), P2_[a])) for a in range(n)]
                        for b in range(n)] for i in range(k)] for c in range(n)])
    _REF[d] = (M, K, B, C)
    return _REF[d]


ONE = _const(1.0, 2)
# P2 basis of the triangle, local order: vertices 0,1,2, then edges (0,1), (1,2), (0,2)
P2 = p2_basis(2)
P1 = [_lam(i) for i in range(3)]
# Reference tensors of the triangle (divided by |T|): MREF[a, b] = int phi_a phi_b,
# KREF[i, j, a, b] = int d_i phi_a d_j phi_b (d_i = d/d lambda_i),
# BREF[i, a, q] = int psi_q d_i phi_a, CREF[c, i, b, a] = int phi_c d_i phi_b phi_a.
MREF, KREF, BREF, CREF = reference_tensors(2)


def geometry(coords, cells):
    """Volumes and barycentric gradients: G[e, i, :] = grad lambda_i on cell e.
    With J = [x_1 - x_0, ..., x_d - x_0], lambda_{1..d} = J^{-1}(x - x_0)."""
    x = coords[cells]                                  # [nc, d+1, d]
    d = x.shape[2]
    Jm = np.stack([x[:, i + 1] - x[:, 0] for i in range(d)], axis=2)   # columns
    det = np.linalg.det(Jm)
    vol = np.abs(det) / factorial(d)
    Ginv = np.linalg.inv(Jm)                           # rows: grad lambda_1..d
    g0 = -Ginv.sum(axis=1)
    return vol, np.concatenate([g0[:, None, :], Ginv], axis=1)


def element_matrices(coords, cells):
    """Per-cell scalar P2 mass Me [nc,n,n], stiffness Ke [nc,n,n] and weak-gradient
    blocks Be [nc,d,n,d+1]: Be[e,c,a,q] = -int psi_q d(phi_a)/dx_c."""
    vol, G = geometry(coords, cells)
    M, K, B, _ = reference_tensors(np.asarray(coords).shape[1])
    Me = vol[:, None, None] * M[None]
    GG = np.einsum("eid,ejd->eij", G, G)
    Ke = vol[:, None, None] * np.einsum("eij,ijab->eab", GG, K)
    Be = -vol[:, None, None, None] * np.einsum("eid,iaq->edaq", G, B)
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
    and B as a (d nf) x nv matrix (rows: u_x free nodes, then u_y, [then u_z]).
    """
    Me, Ke, Be = element_matrices(mesh.coords, mesh.cells)
    Ve = nu * Ke
    if wind is not None:
        Ve = Ve + convection_matrices(mesh.coords, mesh.cells, mesh.cell_p2, wind)
    nodes = mesh.cell_p2
    n = nodes.shape[1]
    dim = mesh.dim
    r = np.repeat(nodes, n, axis=1).ravel()
    c = np.tile(nodes, (1, n)).ravel()
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
    rb = np.repeat(nodes, dim + 1, axis=1).ravel()
    cb = np.tile(mesh.cells, (1, n)).ravel()
    Bd = []
    for d in range(dim):
        Bfull = sp.coo_matrix((Be[:, d].ravel(), (rb, cb)), shape=(mesh.np2, mesh.nv)).tocsr()
        Bd.append(Bfull[fr])
    out["B"] = sp.vstack(Bd).tocsr()
    out["Bfull"] = [sp.coo_matrix((Be[:, d].ravel(), (rb, cb)), shape=(mesh.np2, mesh.nv)).tocsr()
                    for d in range(dim)]          # every P2 row, per component
    out["dim"] = dim
    out["Mfull"] = Mfull
    out["Kfull"] = Vfull
    return out

"""Additive vertex-star Vanka relaxation extended to all IRK stages (Section 4.2).

Patch S_v (one per mesh vertex v): every velocity degree of freedom in the
closure of the cells touching v, plus the single pressure DoF at v, for every
stage.  Order inside S_v: stage by stage; inside a stage the free velocity DoFs
in ascending global index (all u_x, then all u_y [, then all u_z]), then p_v.

One relaxation step (the additive update of Section 4.2):
    k <- k + omega * sum_v R_v^T (R_v J R_v^T)^{-1} R_v (F - J k),
with R_v J R_v^T cut out of the assembled J.  Corrections are added in
ascending v.  The patch solve is a partial-pivoting LU (LAPACK getrf/getrs).

Chebyshev acceleration (Section 5.1: Chebyshev polynomials of the first kind on
a hand-tuned interval [lo, hi], e.g. [2, 8], ahead of the Vanka-preconditioned
operator D^{-1} J with D^{-1} = sum_v R_v^T A_v^{-1} R_v): the classical
three-term Chebyshev iteration (Saad, Iterative Methods, Alg. 12.1) with
theta = (hi+lo)/2, delta = (hi-lo)/2, sigma = theta/delta:
    d_0 = D^{-1}(F - J x_0) / theta,                    rho_0 = 1/sigma
    x_{k+1} = x_k + d_k
    rho_{k+1} = 1/(2 sigma - rho_k)
    d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) D^{-1}(F - J x_{k+1})
nu steps cost nu residuals and nu patch applications, like nu damped steps.

The colouring used to scatter without write conflicts is the greedy
distance-2 colouring in vertex-id order (smallest colour not taken by any
already-coloured vertex at graph distance 1 or 2).
"""
import numpy as np
import scipy.linalg as sla


def patch_nodes(mesh):
    """Free P2 node indices (free numbering) in the closure of star(v), ascending."""
    stars = mesh.vertex_stars()
    out = []
    for v in range(mesh.nv):
        nodes = np.unique(mesh.cell_p2[stars[v]].ravel())
        f = mesh.p2_to_free[nodes]
        out.append(np.sort(f[f >= 0]))
    return out


def patch_dofs(mesh, nodes_v, v, s):
    """Global stage-vector indices of S_v (see module docstring)."""
    nf, nv, d = mesh.nf, mesh.nv, mesh.dim
    m = d * nf + nv
    one = np.concatenate([c * nf + nodes_v for c in range(d)] + [[d * nf + v]])
    return np.concatenate([t * m + one for t in range(s)]).astype(np.int64)


def all_patch_dofs(mesh, s):
    nodes = patch_nodes(mesh)
    return [patch_dofs(mesh, nodes[v], v, s) for v in range(mesh.nv)]


def distance2_colouring(mesh):
    nb = mesh.vertex_neighbours()
    colour = -np.ones(mesh.nv, dtype=np.int64)
    for v in range(mesh.nv):
        near = set(nb[v].tolist())
        for w in nb[v]:
            near.update(nb[w].tolist())
        near.discard(v)
        taken = {colour[w] for w in near if colour[w] >= 0}
        c = 0
        while c in taken:
            c += 1
        colour[v] = c
    return colour


class Vanka:
    """Patch factors of one level and the additive relaxation step."""

    def __init__(self, J, dofs):
        self.dofs = dofs
        Jc = J.tocsr()
        self.lu = []
        self.min_pivot_ratio = np.inf
        for idx in dofs:
            Av = Jc[idx][:, idx].toarray()
            lu, piv = sla.lu_factor(Av, check_finite=True)
            d = np.abs(np.diag(lu))
            ratio = d.min() / np.abs(Av).max()
            self.min_pivot_ratio = min(self.min_pivot_ratio, ratio)
            if ratio <= 1e3 * np.finfo(float).eps:
                raise np.linalg.LinAlgError("singular patch")
            self.lu.append((lu, piv))

    def correction(self, r):
        """sum_v R_v^T A_v^{-1} R_v r, summed in ascending v."""
        c = np.zeros_like(r)
        for idx, f in zip(self.dofs, self.lu):
            c[idx] += sla.lu_solve(f, r[idx])
        return c

    def sweep(self, J, F, k, omega):
        """One additive Vanka step: k + omega * correction(F - J k)."""
        return k + omega * self.correction(F - J @ k)

    def chebyshev(self, J, F, x, nsteps, lo, hi):
        """nsteps Chebyshev-accelerated Vanka steps on [lo, hi] from x."""
        theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = self.correction(F - J @ x) / theta
        for k in range(nsteps):
            x = x + d
            if k + 1 == nsteps:
                break
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * self.correction(F - J @ x)
            rho = rho_new
        return x

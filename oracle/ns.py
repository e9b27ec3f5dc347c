"""Navier-Stokes stage equations and Newton's method (Section 3.2; test
infrastructure only, like the rest of the oracle).

With U_i = u^n + dt sum_j a_ij k_j^u and P_i = p^n + dt sum_j a_ij k_j^p, the
stage residual of stage i is

    F_i^u = M k_i^u + N(U_i) + K U_i + B P_i - M f_i,      F_i^p = B^T U_i,

which is the linear stage system of the Stokes case plus N(U) = C(U) U, the
discrete <u . grad u, v> (C(w) the convection matrix of the wind w).  Newton's
method solves F = 0 with the Jacobian

    J_ij = delta_ij [[M, 0], [0, 0]] + dt a_ij [[K + C(U_i) + R(U_i), B], [B^T, 0]],
    R(w)_dc[a, b] = int phi_a phi_b d w_d / d x_c,

whose velocity blocks depend on the row stage i and couple the velocity
components (R), so it is not of Kronecker form.  Velocities here are P2 nodal
values at every node (Dirichlet data included: the lid of the cavity); the
stage unknowns live on free nodes.  The linear solves use Eisenstat and
Walker's choice 2 forcing terms, eta_l = gamma (|F_l| / |F_{l-1}|)^alpha with
gamma = 0.9, alpha = 2, the safeguard max(eta_l, gamma eta_{l-1}^alpha) when
that exceeds 0.1, and eta_l <= eta_max = 0.9 (eta_0 = 0.5).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def reaction_matrices(coords, cells, cell_p2, wind):
    """Re[e, d, c, a, b] = int_e phi_a phi_b d w_d / d x_c for the P2
    interpolant w of the nodal wind [np2, 2] (2D)."""
    area, G = fem.geometry(coords, cells)
    wl = wind[cell_p2]                                    # [nc, 6, 2]
    # d w_d / d x_c = sum_e w_e^d sum_i (d phi_e / d lambda_i) G[i, c];
    # CREF[a, i, e, b] = int phi_a d_i phi_e phi_b
    return area[:, None, None, None, None] * np.einsum("eqd,eic,aiqb->edcab", wl, G, fem.CREF)


class NSStages:
    """Stage residual and Jacobian of one IRK step of 2D Navier-Stokes on a
    level mesh (free-node numbering as the library: per stage u_x, u_y on free
    nodes, then p on every vertex)."""

    def __init__(self, mesh, A, dt, nu):
        self.mesh, self.A, self.dt, self.nu = mesh, np.asarray(A, float), dt, nu
        self.s = self.A.shape[0]
        self.ops = fem.assemble(mesh, nu=nu)
        nodes = mesh.cell_p2
        n = nodes.shape[1]
        self._r = np.repeat(nodes, n, axis=1).ravel()
        self._c = np.tile(nodes, (1, n)).ravel()
        self.fr = mesh.free_p2
        self.nf, self.nv = mesh.nf, mesh.nv
        self.m = 2 * self.nf + self.nv
        self.N = self.s * self.m
        self.Kfull = self.ops["Kall"]                     # free rows x all nodes (nu K)

    def _full(self, Ee):
        return sp.coo_matrix((Ee.ravel(), (self._r, self._c)),
                             shape=(self.mesh.np2, self.mesh.np2)).tocsr()

    def stage_fields(self, un_all, pn, k):
        """U_i at every P2 node [s, np2, 2] and P_i [s, nv]."""
        s, nf, m, dt = self.s, self.nf, self.m, self.dt
        U = np.repeat(un_all[None], s, axis=0).copy()
        P = np.repeat(pn[None], s, axis=0).copy()
        for i in range(s):
            for j in range(s):
                kj = k[j * m:(j + 1) * m]
                U[i, self.fr, 0] += dt * self.A[i, j] * kj[:nf]
                U[i, self.fr, 1] += dt * self.A[i, j] * kj[nf:2 * nf]
                P[i] += dt * self.A[i, j] * kj[2 * nf:]
        return U, P

    def residual(self, k, un_all, pn, f_all):
        """F(k); f_all [s, np2, 2] nodal forcing at the stage times."""
        s, nf, m = self.s, self.nf, self.m
        U, P = self.stage_fields(un_all, pn, k)
        M, Mall, B = self.ops["M"], self.ops["Mall"], self.ops["B"]
        F = np.zeros(self.N)
        for i in range(s):
            ki = k[i * m:(i + 1) * m]
            Cf = self._full(fem.convection_matrices(self.mesh.coords, self.mesh.cells,
                                                     self.mesh.cell_p2, U[i]))[self.fr]
            BP = B @ P[i]
            for d in range(2):
                sl = slice(i * m + d * nf, i * m + (d + 1) * nf)
                F[sl] = (M @ ki[d * nf:(d + 1) * nf] + Cf @ U[i, :, d] + self.Kfull @ U[i, :, d]
                         + BP[d * nf:(d + 1) * nf] - Mall @ f_all[i, :, d])
            # divergence of U_i with its Dirichlet values (B^T with every velocity column)
            F[i * m + 2 * nf:(i + 1) * m] = sum(self.ops["Bfull"][d].T @ U[i, :, d] for d in range(2))
        return F

    def jacobian(self, k, un_all, pn):
        s, nf, m, dt = self.s, self.nf, self.m, self.dt
        U, _ = self.stage_fields(un_all, pn, k)
        M, K, B = self.ops["M"], self.ops["K"], self.ops["B"]
        fr = self.fr
        rows = []
        for i in range(s):
            mesh = self.mesh
            C = self._full(fem.convection_matrices(mesh.coords, mesh.cells, mesh.cell_p2,
                                                   U[i]))[fr][:, fr]
            Re = reaction_matrices(mesh.coords, mesh.cells, mesh.cell_p2, U[i])
            R = [[self._full(Re[:, d, c])[fr][:, fr] for c in range(2)] for d in range(2)]
            V = sp.bmat([[K + C + R[0][0], R[0][1]], [R[1][0], K + C + R[1][1]]])
            Z = sp.csr_matrix((self.nv, self.nv))
            row = []
            for j in range(s):
                a = dt * self.A[i, j]
                Mij = sp.block_diag([M, M]) if i == j else sp.csr_matrix((2 * nf, 2 * nf))
                row.append(sp.bmat([[Mij + a * V, a * B], [a * B.T, Z]]))
            rows.append(row)
        return sp.bmat(rows).tocsr()

    def pressure_mask(self):
        mask = np.zeros(self.N, bool)
        for t in range(self.s):
            mask[t * self.m + 2 * self.nf:(t + 1) * self.m] = True
        return mask

    def project_pressure(self, x):
        y = x.copy()
        for t in range(self.s):
            sl = slice(t * self.m + 2 * self.nf, (t + 1) * self.m)
            y[sl] -= y[sl].mean()
        return y


def eisenstat_walker(eta_prev, fnorm, fnorm_prev, gamma=0.9, alpha=2.0, eta_max=0.9):
    """Choice 2 forcing term with its safeguard."""
    eta = gamma * (fnorm / fnorm_prev) ** alpha
    safe = gamma * eta_prev ** alpha
    if safe > 0.1:
        eta = max(eta, safe)
    return min(eta, eta_max)


def newton(ns, un_all, pn, f_all, k0, linear_solve, atol=1e-10, maxit=30, eta0=0.5):
    """Inexact Newton: linear_solve(J, rhs, eta) returns d with
    |rhs - J d| <= eta |rhs|.  Returns (k, history of |F|, etas)."""
    k = k0.copy()
    F = ns.residual(k, un_all, pn, f_all)
    hist, etas = [np.linalg.norm(F)], []
    eta = eta0
    for it in range(maxit):
        if hist[-1] <= atol:
            break
        if it > 0:
            eta = eisenstat_walker(eta, hist[-1], hist[-2])
        J = ns.jacobian(k, un_all, pn)
        d = linear_solve(J, -F, eta)
        k = k + d
        F = ns.residual(k, un_all, pn, f_all)
        hist.append(np.linalg.norm(F))
        etas.append(eta)
    return k, hist, etas


def bordered_solve(ns):
    """Exact linear solve with the per-stage pressure constants fixed by
    zero-mean borders (used where eta is irrelevant)."""
    def solve(J, rhs, eta):
        N, s, m, nf = ns.N, ns.s, ns.m, ns.nf
        Nb = np.zeros((N, s))
        for t in range(s):
            Nb[t * m + 2 * nf:(t + 1) * m, t] = 1.0
        Jb = sp.bmat([[J, sp.csr_matrix(Nb)], [sp.csr_matrix(Nb.T), None]]).tocsc()
        x = spla.spsolve(Jb, np.concatenate([rhs, np.zeros(s)]))
        return x[:N]
    return solve

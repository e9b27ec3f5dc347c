"""Discrete adjoint of the IRK time stepping (the paper's forward model,
Section 3.1, differentiated step by step; the differentiation itself is not
in the paper).

Forward step n (Section 3.1):
    F^n_i = [ M f_i + C th - K u^n - B p^n ; -B^T u^n ]   (every stage i)
    J k^n = F^n,   u^{n+1} = u^n + dt sum_j b_j k^n_j,u,   p^{n+1} likewise,
with th a per-cell P0 forcing (2 values per cell: x then y blocks) entering as
int th . v, C[a, c] = int_c phi_a.  Objective after N steps:
    Jobj = 1/2 (u^N - u_T)^T M2 (u^N - u_T),  M2 = diag(M, M).
Adjoint step (from (ub, pb) at n+1 to n):
    kb_j = dt b_j [ub; pb],   J^T lam = kb,
    ub <- ub - sum_i (K^T lam_i,u + B lam_i,p),  pb <- pb - sum_i B^T lam_i,u,
    thb += C^T sum_i lam_i,u,
    d/dnu += -(1/nu) sum_i lam_i,u . K (u^n + dt sum_j a_ij k_j,u)
(K = nu K_1 carries nu, so dK/dnu = K/nu; J depends on nu through dt A (x) K
and F through -K u^n).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, stage


def cell_load_matrix(mesh):
    """C[a, c] = int_c phi_a for free P2 nodes a (scalar; applied per component)."""
    area, _ = fem.geometry(mesh.coords, mesh.cells)
    ref = np.array([fem._integral_over_area(fem.P2[a]) for a in range(6)])
    rows = mesh.p2_to_free[mesh.cell_p2].ravel()
    cols = np.repeat(np.arange(mesh.nc), 6)
    vals = (area[:, None] * ref[None, :]).ravel()
    keep = (rows >= 0) & (vals != 0.0)
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(mesh.nf, mesh.nc))


class Problem:
    """Forward model and its adjoint on one level, solved with a direct sparse
    LU of the bordered stage system (exact to rounding)."""

    def __init__(self, mesh, A, b, dt, nu):
        self.mesh, self.A, self.b, self.dt, self.nu = mesh, np.asarray(A), np.asarray(b), dt, nu
        self.s = len(b)
        self.set_nu(nu)
        self.C = cell_load_matrix(mesh)
        self.C2 = sp.block_diag([self.C, self.C], format="csr")

    def set_nu(self, nu):
        self.nu = nu
        self.ops = fem.assemble(self.mesh, nu=nu)
        self.J = stage.stage_matrix(self.ops, self.A, self.dt)
        m = self.mesh
        self.m = 2 * m.nf + m.nv
        Nm = np.zeros((self.s * self.m, self.s))
        for t in range(self.s):
            Nm[t * self.m + 2 * m.nf:(t + 1) * self.m, t] = 1.0
        Nm = sp.csr_matrix(Nm)
        self.lu = spla.splu(sp.bmat([[self.J, Nm], [Nm.T, None]], format="csc"))
        self.luT = spla.splu(sp.bmat([[self.J.T, Nm], [Nm.T, None]], format="csc"))
        self.K2 = sp.block_diag([self.ops["K"], self.ops["K"]], format="csr")
        self.M2 = sp.block_diag([self.ops["M"], self.ops["M"]], format="csr")

    def solve(self, F):
        return self.lu.solve(np.concatenate([F, np.zeros(self.s)]))[: self.s * self.m]

    def solveT(self, G):
        return self.luT.solve(np.concatenate([G, np.zeros(self.s)]))[: self.s * self.m]

    def step(self, un, pn, f_all, theta):
        F = stage.stage_rhs(self.ops, un, pn, f_all)
        g = self.C2 @ theta
        nu_ = 2 * self.mesh.nf
        for i in range(self.s):
            F[i * self.m: i * self.m + nu_] += g
        k = self.solve(F)
        u1, p1 = stage.advance(k, un, pn, self.b, self.dt)
        return u1, p1, k

    def objective(self, u, u_target):
        e = u - u_target
        return 0.5 * e @ (self.M2 @ e), self.M2 @ e

    def adjoint_step(self, ub, pb, k, un):
        s, m, nu_ = self.s, self.m, 2 * self.mesh.nf
        kb = np.concatenate([self.dt * self.b[j] * np.concatenate([ub, pb]) for j in range(s)])
        lam = self.solveT(kb).reshape(s, m)
        ks = k.reshape(s, m)
        B = self.ops["B"]
        ub_new, pb_new = ub.copy(), pb.copy()
        thb = np.zeros(self.C2.shape[1])
        dnu = 0.0
        for i in range(s):
            lu_, lp_ = lam[i, :nu_], lam[i, nu_:]
            ub_new -= self.K2.T @ lu_ + B @ lp_
            pb_new -= B.T @ lu_
            thb += self.C2.T @ lu_
            z = un + self.dt * (self.A[i] @ ks[:, :nu_])
            dnu -= lu_ @ (self.K2 @ z) / self.nu
        return ub_new, pb_new, thb, dnu


def run(prob, u0, p0, forcing, theta, nsteps, u_target, checkpoint_every=2):
    """Objective and gradients (d/dtheta, d/dnu) by the adjoint, with the
    forward states stored only every `checkpoint_every` steps and recomputed
    segment by segment in the reverse sweep.  forcing(n) -> f_all of step n."""
    ckpt = {0: (u0.copy(), p0.copy())}
    u, p = u0, p0
    for n in range(nsteps):
        u, p, _ = prob.step(u, p, forcing(n), theta)
        if (n + 1) % checkpoint_every == 0 and n + 1 < nsteps:
            ckpt[n + 1] = (u.copy(), p.copy())
    Jobj, ub = prob.objective(u, u_target)
    pb = np.zeros_like(p)
    thb = np.zeros_like(theta)
    dnu = 0.0
    starts = sorted(ckpt)
    for seg in reversed(range(len(starts))):
        n0 = starts[seg]
        n1 = starts[seg + 1] if seg + 1 < len(starts) else nsteps
        states, ks = [], []
        u, p = ckpt[n0]
        for n in range(n0, n1):
            states.append(u)
            u, p, k = prob.step(u, p, forcing(n), theta)
            ks.append(k)
        for n in reversed(range(n0, n1)):
            ub, pb, tb, dn = prob.adjoint_step(ub, pb, ks[n - n0], states[n - n0])
            thb += tb
            dnu += dn
    return Jobj, thb, dnu


def objective_only(prob, u0, p0, forcing, theta, nsteps, u_target):
    u, p = u0, p0
    for n in range(nsteps):
        u, p, _ = prob.step(u, p, forcing(n), theta)
    return prob.objective(u, u_target)[0]

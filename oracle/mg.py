"""Monolithic multigrid V-cycle for the IRK stage system (Section 4).

Levels come from uniform refinement of the coarsest mesh (Section 4.1); each
level's operator is rediscretised (assembled on that level); prolongation is
I_s (x) P and restriction its transpose; the coarsest system is solved
directly (Section 4.1).  Relaxation is the additive Vanka step (Section 4.2)
applied nu_pre times before and nu_post times after the coarse correction,
either accelerated by Chebyshev polynomials on [lo, hi] (Section 5.1, the
paper's choice, [2, 8] for 2D Stokes) or as plain damped steps with weight
omega.

The coarsest solve handles the pressure null space (one constant per stage)
by bordering: [[J, N], [N^T, 0]] [x; l] = [r; 0], N the per-stage constant
pressure indicators, solved with a dense LU (LAPACK gesv).  The solution has
zero pressure sum in every stage.
"""
import numpy as np
import scipy.sparse as sp

from . import mesh as mesh_mod
from . import fem, stage, transfer, vanka


class Level:
    pass


class Hierarchy:
    def __init__(self, coords, cells, bnd, nlevels, A, dt, nu=1.0, wind_finest=None,
                 nu_pre=2, nu_post=2, smoother="chebyshev", omega=0.5, cheb=(2.0, 8.0),
                 build_patches=True):
        self.A = np.asarray(A, dtype=np.float64)
        self.s = self.A.shape[0]
        self.dt = dt
        self.nu = nu
        self.nu_pre, self.nu_post, self.omega = nu_pre, nu_post, omega
        if smoother not in ("chebyshev", "richardson"):
            raise ValueError(smoother)
        self.smoother, self.cheb = smoother, cheb
        meshes = mesh_mod.hierarchy(coords, cells, bnd, nlevels)
        winds = [None] * nlevels
        if wind_finest is not None:
            # coarse P2 nodes are a subset of the fine ones with the same ids
            # (P2 nodes of level l == vertices of level l+1): inject
            winds[-1] = np.asarray(wind_finest)
            for l in range(nlevels - 2, -1, -1):
                winds[l] = winds[l + 1][: meshes[l].np2]
        self.levels = []
        for l, m in enumerate(meshes):
            L = Level()
            L.mesh = m
            L.ops = fem.assemble(m, nu=nu, wind=winds[l])
            L.J = stage.stage_matrix(L.ops, self.A, dt)
            L.m = m.dim * m.nf + m.nv
            L.N = self.s * L.m
            if l > 0:
                Pu, Pp = transfer.prolongation(meshes[l - 1], m)
                L.P = transfer.stage_prolongation(Pu, Pp, self.s, m.dim)
                if build_patches:
                    L.dofs = vanka.all_patch_dofs(m, self.s)
                    L.vanka = vanka.Vanka(L.J, L.dofs)
            self.levels.append(L)
        self._build_coarse()

    def _build_coarse(self):
        L = self.levels[0]
        Nmat = np.zeros((L.N, self.s))
        for t in range(self.s):
            Nmat[t * L.m + L.mesh.dim * L.mesh.nf: (t + 1) * L.m, t] = 1.0
        Jd = L.J.toarray()
        self.coarse_bordered = np.block([[Jd, Nmat], [Nmat.T, np.zeros((self.s, self.s))]])

    def coarse_solve(self, r):
        L = self.levels[0]
        rhs = np.concatenate([r, np.zeros(self.s)])
        return np.linalg.solve(self.coarse_bordered, rhs)[: L.N]

    def vcycle(self, r, level=None):
        """z = MG(r): one V(nu_pre, nu_post) cycle with zero initial guess."""
        if level is None:
            level = len(self.levels) - 1
        if level == 0:
            return self.coarse_solve(r)
        L = self.levels[level]
        z = self.smooth(L, r, np.zeros_like(r), self.nu_pre)
        rc = L.P.T @ (r - L.J @ z)
        z = z + L.P @ self.vcycle(rc, level - 1)
        return self.smooth(L, r, z, self.nu_post)

    def smooth(self, L, r, z, nsteps):
        if nsteps == 0:
            return z
        if self.smoother == "chebyshev":
            return L.vanka.chebyshev(L.J, r, z, nsteps, *self.cheb)
        for _ in range(nsteps):
            z = L.vanka.sweep(L.J, r, z, self.omega)
        return z

    @property
    def finest(self):
        return self.levels[-1]

    def pressure_mask(self, level=None):
        L = self.levels[-1 if level is None else level]
        mask = np.zeros(L.N, dtype=bool)
        for t in range(self.s):
            mask[t * L.m + L.mesh.dim * L.mesh.nf: (t + 1) * L.m] = True
        return mask

    def project_pressure(self, x, level=None):
        """Remove the per-stage mean of the pressure entries (l2 projection onto
        the complement of the null space of J)."""
        L = self.levels[-1 if level is None else level]
        y = x.copy()
        for t in range(self.s):
            sl = slice(t * L.m + L.mesh.dim * L.mesh.nf, (t + 1) * L.m)
            y[sl] -= y[sl].mean()
        return y

    def ritz_estimate(self, level, k, x0=None):
        """Section 5.1's eigenvalue estimate for the Chebyshev interval: k
        Arnoldi steps on the Vanka-preconditioned operator D^{-1} J of a level
        (D^{-1} the additive patch correction), modified Gram-Schmidt applied
        twice, from x0 (default x0_i = sin(i + 1)).  Returns (lambda, Ritz
        values), lambda = the largest real part of the Ritz values (the
        eigenvalues of the k x k Hessenberg matrix, by LAPACK)."""
        L = self.levels[level]
        x = np.sin(np.arange(1, L.N + 1, dtype=np.float64)) if x0 is None else np.array(x0, float)
        V = np.zeros((k + 1, L.N))
        H = np.zeros((k + 1, k))
        V[0] = x / np.linalg.norm(x)
        kk = k
        for j in range(k):
            w = L.vanka.correction(L.J @ V[j])
            for _ in range(2):
                for i in range(j + 1):
                    h = V[i] @ w
                    H[i, j] += h
                    w = w - h * V[i]
            hn = np.linalg.norm(w)
            if j + 1 == k:
                break
            if hn <= 1e-14 * abs(H[j, j]):
                kk = j + 1
                break
            H[j + 1, j] = hn
            V[j + 1] = w / hn
        ritz = np.linalg.eigvals(H[:kk, :kk])
        return float(ritz.real.max()), ritz

"""Flexible GMRES (Saad 1993), the outer Krylov method of Section 4:
right-preconditioned, the preconditioned vectors z_j = M_j(v_j) are stored
alongside the Arnoldi basis, modified Gram-Schmidt, Givens rotations, restart
after m steps.  Convergence: ||F - J k||_2 <= max(rtol ||F||_2, atol), judged on
the Arnoldi residual estimate and confirmed on the true residual at the end of
every cycle.
"""
import numpy as np


def fgmres(J, F, precond, x0=None, rtol=1e-10, atol=1e-30, restart=30, maxit=500,
           project=None):
    """Solve J x = F.  Returns (x, iterations, residual history)."""
    n = F.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(F)
    target = max(rtol * bnorm, atol)
    hist = []
    its = 0
    r = F - J @ x
    beta = np.linalg.norm(r)
    hist.append(beta)
    while beta > target and its < maxit:
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            z = precond(V[j])
            if project is not None:
                z = project(z)
            Z[j] = z
            w = J @ z
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                   # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= target or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + y @ Z[:j_done]
        r = F - J @ x
        beta = np.linalg.norm(r)
        hist[-1] = beta
    return x, its, hist

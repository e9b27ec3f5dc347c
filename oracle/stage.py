"""The stage-coupled IRK system (Section 3.1, the Kronecker form of the DAE
Runge-Kutta stage equations):

    ( I_s (x) [[M, 0], [0, 0]] + dt A (x) [[K, B], [B^T, 0]] ) k = F,
    F_i = [ M f_i - K u^n - B p^n ;  -B^T u^n ],

with k ordered stage by stage and, inside a stage, [k_u; k_p] (u_x block, then
u_y block, then the pressure block).  After the solve,
    u^{n+1} = u^n + dt sum_j b_j k_j^u,   p^{n+1} = p^n + dt sum_j b_j k_j^p.
"""
import numpy as np
import scipy.sparse as sp


def velocity_block(S, dim=2):
    """Scalar P2 block S applied to every velocity component."""
    return sp.block_diag([S] * dim, format="csr")


def single_stage_blocks(ops):
    """Return (Mt, St): Mt = [[Md, 0], [0, 0]], St = [[Kd, B], [B^T, 0]]
    with Md = diag(M, ..., M), Kd = diag(K, ..., K) (d copies), size m x m."""
    dim = ops.get("dim", 2)
    M2 = velocity_block(ops["M"], dim)
    K2 = velocity_block(ops["K"], dim)
    B = ops["B"]
    nv = B.shape[1]
    Z = sp.csr_matrix((nv, nv))
    Mt = sp.bmat([[M2, None], [None, Z]], format="csr")
    St = sp.bmat([[K2, B], [B.T, Z]], format="csr")
    return Mt, St


def stage_matrix(ops, A, dt):
    """J = I_s (x) Mt + dt A (x) St (Section 3.1)."""
    Mt, St = single_stage_blocks(ops)
    s = A.shape[0]
    return (sp.kron(sp.identity(s), Mt) + dt * sp.kron(sp.csr_matrix(A), St)).tocsr()


def stage_rhs(ops, un, pn, f_all):
    """F_i = [M f_i - K u^n - B p^n; -B^T u^n].

    un: free velocity [d nf]; pn: [nv]; f_all: [s, d, np2] forcing interpolant
    at every P2 node (M f uses boundary columns too, since f need not vanish
    there).
    """
    dim = ops.get("dim", 2)
    s = f_all.shape[0]
    K2 = velocity_block(ops["K"], dim)
    B = ops["B"]
    base_u = -(K2 @ un) - B @ pn
    base_p = -(B.T @ un)
    out = []
    for i in range(s):
        mf = np.concatenate([ops["Mall"] @ f_all[i, c] for c in range(dim)])
        out.append(np.concatenate([mf + base_u, base_p]))
    return np.concatenate(out)


def advance(k, un, pn, b, dt):
    """u^{n+1} = u^n + dt sum_j b_j k_j^u (and the same for p)."""
    nu_ = un.size
    m = nu_ + pn.size
    s = b.size
    ks = k.reshape(s, m)
    return un + dt * (b @ ks[:, :nu_]), pn + dt * (b @ ks[:, nu_:])

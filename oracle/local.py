"""Sampled entries of the stage system at any mesh size (test infrastructure,
like the rest of oracle/; nothing else imports it).

The assembled stage matrix of Section 3.1,
    J = I_s (x) [[M, 0], [0, 0]] + dt A (x) [[K, B], [B^T, 0]],
is too large to form in Python at the 512 x 512 size (about 3e8 nonzeros for
s = 3).  Its entries are sums over cells of element integrals, so a row of J,
or the patch system A_v = R_v J R_v^T of one Vanka patch (Section 4.2), needs
only the element matrices of the cells around the nodes involved.  This module
computes exactly those from oracle.fem.element_matrices, in the DoF layout of
oracle.stage (stage by stage; inside a stage every u_x, every u_y [, every
u_z] on free P2 nodes, then the pressure at every vertex) and the patch layout
of oracle.vanka.  At small sizes every row and patch equals the one cut out of
oracle.stage.stage_matrix (tests/test_oracle_local.py).
"""
import numpy as np

from oracle import fem


class LocalStage:
    """Rows of J and patch systems of one level, from local element matrices.

    mesh: oracle.mesh.Mesh of the level; A: s x s Butcher matrix; dt; nu
    scales the stiffness (Stokes, no wind).
    """

    def __init__(self, mesh, A, dt, nu=1.0):
        self.mesh = mesh
        self.A = np.asarray(A, dtype=np.float64)
        self.s = self.A.shape[0]
        self.dt = float(dt)
        self.nu = float(nu)
        self.d = mesh.dim
        self.nf, self.nv = mesh.nf, mesh.nv
        self.m = self.d * self.nf + self.nv
        self.N = self.s * self.m
        k = mesh.cell_p2.shape[1]
        flat = mesh.cell_p2.ravel()
        order = np.argsort(flat, kind="stable")
        self._cell = order // k                       # cells by P2 node, ascending
        self._ptr = np.searchsorted(flat[order], np.arange(mesh.np2 + 1))

    def cells_of(self, node):
        """Cells containing P2 node `node` (a vertex id is also a P2 node id)."""
        return self._cell[self._ptr[node]:self._ptr[node + 1]]

    def _split(self, i):
        """(stage t, component c or -1 for pressure, P2 node or vertex)."""
        t, off = divmod(int(i), self.m)
        if off < self.d * self.nf:
            c, f = divmod(off, self.nf)
            return t, c, int(self.mesh.free_p2[f])
        return t, -1, off - self.d * self.nf

    def _vel(self, u, c, node):
        f = self.mesh.p2_to_free[node]
        return None if f < 0 else u * self.m + c * self.nf + int(f)

    def _pres(self, u, v):
        return u * self.m + self.d * self.nf + int(v)

    def row(self, i):
        """Row i of J as {column: value} (every structural entry)."""
        t, c, node = self._split(i)
        mesh, s, d = self.mesh, self.s, self.d
        cells = self.cells_of(node)
        Me, Ke, Be = fem.element_matrices(mesh.coords, mesh.cells[cells])
        out = {}

        def add(col, val):
            if col is not None:
                out[col] = out.get(col, 0.0) + val

        for e, cell in enumerate(cells):
            p2 = mesh.cell_p2[cell]
            if c >= 0:                                    # velocity row (c, node)
                la = int(np.nonzero(p2 == node)[0][0])
                for u in range(s):
                    dtA = self.dt * self.A[t, u]
                    for lb, b in enumerate(p2):           # M and K: same component
                        val = dtA * self.nu * Ke[e, la, lb] + (Me[e, la, lb] if u == t else 0.0)
                        add(self._vel(u, c, b), val)
                    for lq, q in enumerate(mesh.cells[cell]):   # B: pressure columns
                        add(self._pres(u, q), dtA * Be[e, c, la, lq])
            else:                                         # pressure row at vertex node
                lq = int(np.nonzero(mesh.cells[cell] == node)[0][0])
                for u in range(s):
                    dtA = self.dt * self.A[t, u]
                    for cc in range(d):                   # B^T: velocity columns
                        for lb, b in enumerate(p2):
                            add(self._vel(u, cc, b), dtA * Be[e, cc, lb, lq])
        return out

    def apply_rows(self, rows, x):
        """(J x)_i for the sampled rows i, and sum_j |J_ij x_j| (for a rounding bound)."""
        y = np.zeros(len(rows))
        mag = np.zeros(len(rows))
        for k, i in enumerate(rows):
            for j, a in self.row(i).items():
                y[k] += a * x[j]
                mag[k] += abs(a * x[j])
        return y, mag

    def patch_nodes(self, v):
        """Free P2 nodes (free numbering) in the closure of star(v), ascending
        (oracle.vanka.patch_nodes for one vertex)."""
        nodes = np.unique(self.mesh.cell_p2[self.cells_of(v)].ravel())
        f = self.mesh.p2_to_free[nodes]
        return np.sort(f[f >= 0])

    def patch_dofs(self, v):
        """Global indices of S_v in the order of oracle.vanka.patch_dofs."""
        nodes = self.patch_nodes(v)
        one = np.concatenate([c * self.nf + nodes for c in range(self.d)] +
                             [[self.d * self.nf + v]])
        return np.concatenate([t * self.m + one for t in range(self.s)]).astype(np.int64)

    def patch_matrix(self, v):
        """A_v = R_v J R_v^T (dense) and the DoFs of S_v."""
        idx = self.patch_dofs(v)
        pos = {int(j): k for k, j in enumerate(idx)}
        Av = np.zeros((idx.size, idx.size))
        for k, i in enumerate(idx):
            for j, a in self.row(i).items():
                if j in pos:
                    Av[k, pos[j]] = a
        return Av, idx

    def patches_containing(self, i):
        """Vertices v whose patch S_v holds DoF i, ascending."""
        _, c, node = self._split(i)
        if c < 0:
            return np.array([node])
        return np.unique(self.mesh.cells[self.cells_of(node)].ravel())

    def vanka_entries(self, rows, r, transpose=False):
        """(sum_v R_v^T A_v^{-1} R_v r)_i for the sampled DoFs i (with
        transpose: A_v^{-T}), each patch solved by LAPACK (numpy.linalg)."""
        out = np.zeros(len(rows))
        cache = {}
        for k, i in enumerate(rows):
            for v in self.patches_containing(i):
                v = int(v)
                if v not in cache:
                    Av, idx = self.patch_matrix(v)
                    rhs = r[idx]
                    sol = np.linalg.solve(Av.T if transpose else Av, rhs)
                    cache[v] = ({int(j): p for p, j in enumerate(idx)}, sol)
                pos, sol = cache[v]
                out[k] += sol[pos[int(i)]]
        return out

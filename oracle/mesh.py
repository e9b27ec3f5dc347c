"""Mesh hierarchy and degree-of-freedom numbering (Section 4.1: hierarchies are
uniform refinements of a coarsest grid; Section 3.1: Taylor-Hood P2-P1 on
simplices, triangles in 2D and tetrahedra in 3D).

Conventions (fixed for this project, stated once here):
  * local edges of a cell: (0,1), (1,2), (0,2) for triangles and
    (0,1), (1,2), (0,2), (0,3), (1,3), (2,3) for tetrahedra;
  * edges of a mesh are the sorted vertex pairs (min, max), numbered in
    lexicographic order;
  * P2 nodes are all vertices (ids 0..nv-1) followed by all edge midpoints
    (id nv + edge id);
  * uniform refinement keeps the coarse vertex ids and appends one vertex per
    coarse edge (id nv_c + edge id).  Child k of cell c gets id 4c + k (2D red
    refinement) or 8c + k (3D Bey refinement);
  * an edge is Dirichlet iff it lies on the boundary (on a boundary facet, a
    facet belonging to one cell) and both its end vertices are flagged; a new
    vertex inherits that flag;
  * free P2 nodes are the non-Dirichlet ones, renumbered in P2-node order.
"""
import itertools

import numpy as np

LOCAL_EDGES = {2: [(0, 1), (1, 2), (0, 2)],
               3: [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]}


class Mesh:
    def __init__(self, coords, cells, bnd):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.bnd = np.asarray(bnd, dtype=bool)
        self.dim = self.coords.shape[1]
        self.nv = self.coords.shape[0]
        self.nc = self.cells.shape[0]
        loc = LOCAL_EDGES[self.dim]
        pairs = np.concatenate([np.sort(self.cells[:, [a, b]], axis=1) for a, b in loc])
        edges, inv = np.unique(pairs, axis=0, return_inverse=True)
        self.edges = edges                               # [ne, 2] lexicographic
        self.ne = edges.shape[0]
        self.cell_edges = inv.reshape(len(loc), self.nc).T
        # boundary facets (faces in 3D, edges in 2D) belong to exactly one cell
        fsub = list(itertools.combinations(range(self.dim + 1), self.dim))
        facets = np.concatenate([np.sort(self.cells[:, list(f)], axis=1) for f in fsub])
        uf, cnt = np.unique(facets, axis=0, return_counts=True)
        bf = uf[cnt == 1]
        on_bnd = np.zeros(self.ne, dtype=bool)
        ekey = {tuple(e): i for i, e in enumerate(edges)}
        for f in bf:
            for a, b in itertools.combinations(sorted(f), 2):
                on_bnd[ekey[(a, b)]] = True
        self.edge_bnd = on_bnd & self.bnd[edges[:, 0]] & self.bnd[edges[:, 1]]
        self.cell_p2 = np.concatenate([self.cells, self.nv + self.cell_edges], axis=1)
        self.np2 = self.nv + self.ne
        self.p2_dirichlet = np.concatenate([self.bnd, self.edge_bnd])
        free = ~self.p2_dirichlet
        self.free_p2 = np.nonzero(free)[0]               # free index -> P2 node
        self.p2_to_free = -np.ones(self.np2, dtype=np.int64)
        self.p2_to_free[self.free_p2] = np.arange(self.free_p2.size)
        self.nf = self.free_p2.size
        mid = 0.5 * (self.coords[edges[:, 0]] + self.coords[edges[:, 1]])
        self.p2_coords = np.concatenate([self.coords, mid])

    def refine(self):
        """2D red refinement: the 4 children of (a,b,c) are (a,m_ab,m_ca),
        (m_ab,b,m_bc), (m_ca,m_bc,c), (m_ab,m_bc,m_ca).  3D Bey refinement of
        (x0,x1,x2,x3) with midpoints xij: (x0,x01,x02,x03), (x01,x1,x12,x13),
        (x02,x12,x2,x23), (x03,x13,x23,x3), and the octahedron cut along
        x02-x13: (x01,x02,x03,x13), (x01,x02,x12,x13), (x02,x03,x13,x23),
        (x02,x12,x13,x23)."""
        e = self.nv + self.cell_edges
        if self.dim == 2:
            a, b, c = self.cells[:, 0], self.cells[:, 1], self.cells[:, 2]
            mab, mbc, mca = e[:, 0], e[:, 1], e[:, 2]
            kids = np.stack([
                np.stack([a, mab, mca], 1), np.stack([mab, b, mbc], 1),
                np.stack([mca, mbc, c], 1), np.stack([mab, mbc, mca], 1)], axis=1)
            cells = kids.reshape(-1, 3)
        else:
            x0, x1, x2, x3 = (self.cells[:, i] for i in range(4))
            m01, m12, m02, m03, m13, m23 = (e[:, i] for i in range(6))
            kids = np.stack([
                np.stack([x0, m01, m02, m03], 1), np.stack([m01, x1, m12, m13], 1),
                np.stack([m02, m12, x2, m23], 1), np.stack([m03, m13, m23, x3], 1),
                np.stack([m01, m02, m03, m13], 1), np.stack([m01, m02, m12, m13], 1),
                np.stack([m02, m03, m13, m23], 1), np.stack([m02, m12, m13, m23], 1)], axis=1)
            cells = kids.reshape(-1, 4)
        return Mesh(self.p2_coords.copy(), cells, self.p2_dirichlet.copy())

    def vertex_stars(self):
        """List of arrays: cells containing each vertex."""
        k = self.dim + 1
        order = np.argsort(self.cells.ravel(), kind="stable")
        vert = self.cells.ravel()[order]
        cell = order // k
        ptr = np.searchsorted(vert, np.arange(self.nv + 1))
        return [cell[ptr[v]:ptr[v + 1]] for v in range(self.nv)]

    def vertex_neighbours(self):
        """Vertex adjacency through mesh edges, as a list of sorted arrays."""
        nb = [[] for _ in range(self.nv)]
        for a, b in self.edges:
            nb[a].append(b)
            nb[b].append(a)
        return [np.array(sorted(x), dtype=np.int64) for x in nb]


def hierarchy(coords, cells, bnd, nlevels):
    """Coarsest mesh followed by nlevels-1 uniform refinements (coarse first)."""
    meshes = [Mesh(coords, cells, bnd)]
    for _ in range(nlevels - 1):
        meshes.append(meshes[-1].refine())
    return meshes

"""Mesh hierarchy and degree-of-freedom numbering (Section 4.1: hierarchies are
uniform refinements of a coarsest grid; Section 3.1: Taylor-Hood P2-P1 on
triangles).

Conventions (fixed for this project, stated once here):
  * edges of a mesh are the sorted vertex pairs (min, max), numbered in
    lexicographic order;
  * P2 nodes are all vertices (ids 0..nv-1) followed by all edge midpoints
    (id nv + edge id);
  * red refinement keeps the coarse vertex ids and appends one vertex per
    coarse edge (id nv_c + edge id); child k of coarse cell c gets id 4c + k;
  * an edge is Dirichlet iff it lies on the boundary (one adjacent cell) and
    both its end vertices are flagged; a new vertex inherits that flag;
  * free P2 nodes are the non-Dirichlet ones, renumbered in P2-node order.
"""
import numpy as np


class Mesh:
    def __init__(self, coords, cells, bnd):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.bnd = np.asarray(bnd, dtype=bool)
        self.nv = self.coords.shape[0]
        self.nc = self.cells.shape[0]
        # all cell edges, each as a sorted pair; local edges (0,1), (1,2), (0,2)
        loc = [(0, 1), (1, 2), (0, 2)]
        pairs = np.concatenate([np.sort(self.cells[:, [a, b]], axis=1) for a, b in loc])
        edges, inv, counts = np.unique(pairs, axis=0, return_inverse=True, return_counts=True)
        self.edges = edges                               # [ne, 2] lexicographic
        self.ne = edges.shape[0]
        inv = inv.reshape(len(loc), self.nc).T           # [nc, 3] edge id per local edge
        self.cell_edges = inv
        edge_cells = counts  # number of cells sharing each edge
        self.edge_bnd = (edge_cells == 1) & self.bnd[edges[:, 0]] & self.bnd[edges[:, 1]]
        # P2 nodes of each cell: 3 vertices then edges (0,1), (1,2), (0,2)
        self.cell_p2 = np.concatenate([self.cells, self.nv + inv], axis=1)
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
        """Red refinement: the 4 children of (a,b,c) are (a,m_ab,m_ca),
        (m_ab,b,m_bc), (m_ca,m_bc,c), (m_ab,m_bc,m_ca)."""
        e = self.cell_edges
        a, b, c = self.cells[:, 0], self.cells[:, 1], self.cells[:, 2]
        mab, mbc, mca = self.nv + e[:, 0], self.nv + e[:, 1], self.nv + e[:, 2]
        kids = np.stack([
            np.stack([a, mab, mca], 1), np.stack([mab, b, mbc], 1),
            np.stack([mca, mbc, c], 1), np.stack([mab, mbc, mca], 1)], axis=1)
        cells = kids.reshape(-1, 3)
        return Mesh(self.p2_coords.copy(), cells, self.p2_dirichlet.copy())

    def vertex_stars(self):
        """List of arrays: cells containing each vertex."""
        order = np.argsort(self.cells.ravel(), kind="stable")
        vert = self.cells.ravel()[order]
        cell = order // 3
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

// Host-side assembly of the Taylor–Hood P2–P1 operators of one level
// (Section 3.1: M, K, B with B the weak gradient from -<p, div v>;
// Section 3.2: Oseen convection <(w . grad) u, v> for a frozen wind w).
//
// Element integrals use the 7-point degree-5 rule of Radon (Stroud T2:5-1),
// which integrates every integrand here exactly on affine triangles: the mass
// matrix is degree 4, the stiffness degree 2, the gradient block degree 2 and
// the convection block (P2 wind x grad P2 x P2) degree 5.
#include <algorithm>
#include <cmath>

#include "irkmg_internal.h"

namespace irkmg {

namespace {

struct QuadRule {
  double lam[7][3];
  double w[7];  // weights sum to 1 (multiply by the area)
};

QuadRule radon7() {
  QuadRule q;
  const double r15 = std::sqrt(15.0);
  const double a1 = (6.0 - r15) / 21.0, a2 = (6.0 + r15) / 21.0;
  const double w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
  q.lam[0][0] = q.lam[0][1] = q.lam[0][2] = 1.0 / 3.0;
  q.w[0] = 9.0 / 40.0;
  const double as[2] = {a1, a2}, ws[2] = {w1, w2};
  int k = 1;
  for (int g = 0; g < 2; ++g)
    for (int r = 0; r < 3; ++r) {
      for (int j = 0; j < 3; ++j) q.lam[k][j] = (j == r) ? 1.0 - 2.0 * as[g] : as[g];
      q.w[k] = ws[g];
      ++k;
    }
  return q;
}

// P2 basis on barycentrics: vertex i -> l_i (2 l_i - 1); edge (i, j) -> 4 l_i l_j,
// local edges (0,1), (1,2), (0,2).  Gradients by the chain rule from grad l.
const int kEdge[3][2] = {{0, 1}, {1, 2}, {0, 2}};

inline void p2_eval(const double l[3], const double gl[3][2], double phi[6], double gphi[6][2]) {
  for (int i = 0; i < 3; ++i) {
    phi[i] = l[i] * (2.0 * l[i] - 1.0);
    for (int d = 0; d < 2; ++d) gphi[i][d] = (4.0 * l[i] - 1.0) * gl[i][d];
  }
  for (int e = 0; e < 3; ++e) {
    int i = kEdge[e][0], j = kEdge[e][1];
    phi[3 + e] = 4.0 * l[i] * l[j];
    for (int d = 0; d < 2; ++d) gphi[3 + e][d] = 4.0 * (l[j] * gl[i][d] + l[i] * gl[j][d]);
  }
}

// Find the slot of column `col` in row `row` of a CSR with sorted columns.
inline int64_t slot(const HostCSR& A, int64_t row, int32_t col) {
  auto b = A.col.begin() + A.ptr[row], e = A.col.begin() + A.ptr[row + 1];
  auto it = std::lower_bound(b, e, col);
  return (it != e && *it == col) ? (it - A.col.begin()) : -1;
}

}  // namespace

void assemble_level(const HostMesh& m, double nu, const double* wind, HostOps& ops) {
  const QuadRule q = radon7();
  // node -> cells, then sparsity patterns by union over cells
  std::vector<int32_t> nc_ptr(m.np2 + 1, 0), nc_idx(6 * m.nc);
  auto cell_node = [&](int64_t c, int a) -> int32_t {
    return a < 3 ? m.cells[3 * c + a] : (int32_t)(m.nv + m.cell_edges[3 * c + a - 3]);
  };
  for (int64_t c = 0; c < m.nc; ++c)
    for (int a = 0; a < 6; ++a) nc_ptr[cell_node(c, a) + 1]++;
  for (int64_t n = 0; n < m.np2; ++n) nc_ptr[n + 1] += nc_ptr[n];
  {
    std::vector<int32_t> fill(nc_ptr.begin(), nc_ptr.end() - 1);
    for (int64_t c = 0; c < m.nc; ++c)
      for (int a = 0; a < 6; ++a) nc_idx[fill[cell_node(c, a)]++] = (int32_t)c;
  }
  HostCSR& V = ops.vel;
  HostCSR& MA = ops.mall;
  HostCSR& B = ops.b;
  V = HostCSR();
  MA = HostCSR();
  B = HostCSR();
  V.nrows = MA.nrows = B.nrows = m.nf;
  V.ncols = m.nf;
  MA.ncols = m.np2;
  B.ncols = m.nv;
  V.ptr.assign(1, 0);
  MA.ptr.assign(1, 0);
  B.ptr.assign(1, 0);
  std::vector<int32_t> nodes, verts;
  for (int64_t i = 0; i < m.nf; ++i) {
    int32_t n = m.free_to_p2[i];
    nodes.clear();
    verts.clear();
    for (int32_t p = nc_ptr[n]; p < nc_ptr[n + 1]; ++p) {
      int64_t c = nc_idx[p];
      for (int a = 0; a < 6; ++a) nodes.push_back(cell_node(c, a));
      for (int a = 0; a < 3; ++a) verts.push_back(m.cells[3 * c + a]);
    }
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    std::sort(verts.begin(), verts.end());
    verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
    for (int32_t x : nodes) {
      MA.col.push_back(x);
      if (m.p2_to_free[x] >= 0) V.col.push_back(m.p2_to_free[x]);
    }
    for (int32_t x : verts) B.col.push_back(x);
    V.ptr.push_back((int32_t)V.col.size());
    MA.ptr.push_back((int32_t)MA.col.size());
    B.ptr.push_back((int32_t)B.col.size());
  }
  V.v[0].assign(V.col.size(), 0.0);
  V.v[1].assign(V.col.size(), 0.0);
  MA.v[0].assign(MA.col.size(), 0.0);
  MA.v[1].assign(MA.col.size(), 0.0);
  // B with every P2 row (Dirichlet rows too), for the lifted right-hand side
  std::vector<std::vector<std::pair<int32_t, double>>> bfull_x(m.np2), bfull_y(m.np2);
  B.v[0].assign(B.col.size(), 0.0);
  B.v[1].assign(B.col.size(), 0.0);

  double Me[6][6], Ke[6][6], Be[2][6][3];
  for (int64_t c = 0; c < m.nc; ++c) {
    const int32_t* t = &m.cells[3 * c];
    const double x0 = m.xy[2 * t[0]], y0 = m.xy[2 * t[0] + 1];
    const double d1x = m.xy[2 * t[1]] - x0, d1y = m.xy[2 * t[1] + 1] - y0;
    const double d2x = m.xy[2 * t[2]] - x0, d2y = m.xy[2 * t[2] + 1] - y0;
    const double det = d1x * d2y - d1y * d2x;
    const double area = 0.5 * std::fabs(det);
    double gl[3][2];
    gl[1][0] = d2y / det;
    gl[1][1] = -d2x / det;
    gl[2][0] = -d1y / det;
    gl[2][1] = d1x / det;
    gl[0][0] = -gl[1][0] - gl[2][0];
    gl[0][1] = -gl[1][1] - gl[2][1];
    int32_t node[6];
    for (int a = 0; a < 6; ++a) node[a] = cell_node(c, a);
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) Me[a][b] = Ke[a][b] = 0.0;
    for (int d = 0; d < 2; ++d)
      for (int a = 0; a < 6; ++a)
        for (int p = 0; p < 3; ++p) Be[d][a][p] = 0.0;
    for (int k = 0; k < 7; ++k) {
      double phi[6], g[6][2];
      p2_eval(q.lam[k], gl, phi, g);
      const double wk = q.w[k] * area;
      double wx = 0.0, wy = 0.0;
      if (wind) {
        for (int a = 0; a < 6; ++a) {
          wx += wind[2 * node[a]] * phi[a];
          wy += wind[2 * node[a] + 1] * phi[a];
        }
      }
      for (int a = 0; a < 6; ++a) {
        for (int b = 0; b < 6; ++b) {
          Me[a][b] += wk * phi[a] * phi[b];
          double kab = nu * (g[a][0] * g[b][0] + g[a][1] * g[b][1]);
          if (wind) kab += (wx * g[b][0] + wy * g[b][1]) * phi[a];
          Ke[a][b] += wk * kab;
        }
        for (int p = 0; p < 3; ++p) {
          Be[0][a][p] -= wk * q.lam[k][p] * g[a][0];
          Be[1][a][p] -= wk * q.lam[k][p] * g[a][1];
        }
      }
    }
    for (int a = 0; a < 6; ++a)
      for (int p = 0; p < 3; ++p) {
        bfull_x[node[a]].push_back({t[p], Be[0][a][p]});
        bfull_y[node[a]].push_back({t[p], Be[1][a][p]});
      }
    for (int a = 0; a < 6; ++a) {
      const int32_t row = m.p2_to_free[node[a]];
      if (row < 0) continue;
      for (int b = 0; b < 6; ++b) {
        int64_t sa = slot(MA, row, node[b]);
        MA.v[0][sa] += Me[a][b];
        MA.v[1][sa] += Ke[a][b];
        const int32_t cf = m.p2_to_free[node[b]];
        if (cf >= 0) {
          int64_t sv = slot(V, row, cf);
          V.v[0][sv] += Me[a][b];
          V.v[1][sv] += Ke[a][b];
        }
      }
      for (int p = 0; p < 3; ++p) {
        int64_t sb = slot(B, row, t[p]);
        B.v[0][sb] += Be[0][a][p];
        B.v[1][sb] += Be[1][a][p];
      }
    }
  }
  // transpose of the velocity operator (same pattern, which is symmetric)
  V.v[2].resize(V.col.size());
  for (int64_t i = 0; i < m.nf; ++i)
    for (int32_t p = V.ptr[i]; p < V.ptr[i + 1]; ++p) {
      int64_t st = slot(V, V.col[p], (int32_t)i);
      V.v[2][p] = V.v[1][st];
    }
  ops.bt = transpose_csr(B, 2);
  // Bᵀ over every velocity column: vertex rows, P2-node columns, summed per pair
  HostCSR Bf;
  Bf.nrows = m.np2;
  Bf.ncols = m.nv;
  Bf.ptr.assign(1, 0);
  for (int64_t n = 0; n < m.np2; ++n) {
    std::vector<std::pair<int32_t, std::pair<double, double>>> e;
    for (size_t k = 0; k < bfull_x[n].size(); ++k)
      e.push_back({bfull_x[n][k].first, {bfull_x[n][k].second, bfull_y[n][k].second}});
    std::stable_sort(e.begin(), e.end(),
                     [](const auto& a, const auto& b) { return a.first < b.first; });
    for (size_t k = 0; k < e.size();) {
      size_t j = k;
      double sx = 0.0, sy = 0.0;
      for (; j < e.size() && e[j].first == e[k].first; ++j) {
        sx += e[j].second.first;
        sy += e[j].second.second;
      }
      Bf.col.push_back(e[k].first);
      Bf.v[0].push_back(sx);
      Bf.v[1].push_back(sy);
      k = j;
    }
    Bf.ptr.push_back((int32_t)Bf.col.size());
  }
  ops.btall = transpose_csr(Bf, 2);
}

// Load of a per-cell constant (P0) forcing: C[a, c] = int_c phi_a for the free
// P2 nodes a of cell c (the same for both velocity components).  P2 vertex
// functions integrate to zero on a triangle, edge functions to |c|/3; the
// degree-5 rule is exact for these quadratics.
void assemble_cell_load(const HostMesh& m, HostCSR& C) {
  const QuadRule q = radon7();
  C = HostCSR();
  C.nrows = m.nf;
  C.ncols = m.nc;
  std::vector<std::vector<std::pair<int32_t, double>>> rows(m.nf);
  for (int64_t c = 0; c < m.nc; ++c) {
    const int32_t* t = &m.cells[3 * c];
    const double x0 = m.xy[2 * t[0]], y0 = m.xy[2 * t[0] + 1];
    const double d1x = m.xy[2 * t[1]] - x0, d1y = m.xy[2 * t[1] + 1] - y0;
    const double d2x = m.xy[2 * t[2]] - x0, d2y = m.xy[2 * t[2] + 1] - y0;
    const double area = 0.5 * std::fabs(d1x * d2y - d1y * d2x);
    double gl[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    double w[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 7; ++k) {
      double phi[6], g[6][2];
      p2_eval(q.lam[k], gl, phi, g);
      for (int a = 0; a < 6; ++a) w[a] += q.w[k] * area * phi[a];
    }
    for (int a = 0; a < 6; ++a) {
      const int32_t node = a < 3 ? t[a] : (int32_t)(m.nv + m.cell_edges[3 * c + a - 3]);
      const int32_t f = m.p2_to_free[node];
      if (f < 0 || std::fabs(w[a]) <= 1e-12 * area) continue;  // vertex functions: zero
      rows[f].push_back({(int32_t)c, w[a]});
    }
  }
  C.ptr.assign(1, 0);
  for (int64_t i = 0; i < m.nf; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    for (auto& pr : rows[i]) {
      C.col.push_back(pr.first);
      C.v[0].push_back(pr.second);
    }
    C.ptr.push_back((int32_t)C.col.size());
  }
}

}  // namespace irkmg

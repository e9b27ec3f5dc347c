// Host-side mesh hierarchy, numbering, transfer weights and Butcher tableau.
//
// Section 4.1: levels are uniform (red) refinements of a coarsest triangle
// mesh, and prolongation is canonical P2 (velocity) / P1 (pressure)
// interpolation; restriction is its transpose.  Section 5: RadauIIA(s).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "irkmg_internal.h"

namespace irkmg {

static inline uint64_t key2(int32_t a, int32_t b) {
  return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
}

int64_t find_edge(const HostMesh& m, int32_t a, int32_t b) {
  if (a > b) std::swap(a, b);
  // edges are sorted lexicographically: binary search on the (a, b) key
  int64_t lo = 0, hi = m.ne;
  const uint64_t k = key2(a, b);
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    uint64_t km = key2(m.edges[2 * mid], m.edges[2 * mid + 1]);
    if (km < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < m.ne && key2(m.edges[2 * lo], m.edges[2 * lo + 1]) == k) return lo;
  return -1;
}

static void finish_mesh(HostMesh& m) {
  const int64_t nc = m.nc, nv = m.nv;
  // edges: sorted vertex pairs, unique, lexicographic
  std::vector<uint64_t> keys(3 * nc);
  static const int le[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) {
      int32_t a = m.cells[3 * c + le[k][0]], b = m.cells[3 * c + le[k][1]];
      if (a > b) std::swap(a, b);
      keys[3 * c + k] = key2(a, b);
    }
  std::vector<uint64_t> sorted = keys;
  std::sort(sorted.begin(), sorted.end());
  std::vector<int32_t> mult;
  std::vector<uint64_t> uniq;
  uniq.reserve(sorted.size());
  for (size_t i = 0; i < sorted.size(); ++i) {
    if (uniq.empty() || uniq.back() != sorted[i]) {
      uniq.push_back(sorted[i]);
      mult.push_back(1);
    } else {
      mult.back()++;
    }
  }
  m.ne = (int64_t)uniq.size();
  m.edges.resize(2 * m.ne);
  m.edge_dir.assign(m.ne, 0);
  for (int64_t e = 0; e < m.ne; ++e) {
    m.edges[2 * e] = (int32_t)(uniq[e] >> 32);
    m.edges[2 * e + 1] = (int32_t)(uniq[e] & 0xffffffffu);
    m.edge_dir[e] = (mult[e] == 1 && m.bnd[m.edges[2 * e]] && m.bnd[m.edges[2 * e + 1]]) ? 1 : 0;
  }
  m.cell_edges.resize(3 * nc);
  for (int64_t i = 0; i < 3 * nc; ++i)
    m.cell_edges[i] =
        (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), keys[i]) - uniq.begin());
  // P2 nodes: vertices, then edges; free numbering in that order
  m.np2 = nv + m.ne;
  m.p2_to_free.assign(m.np2, -1);
  m.free_to_p2.clear();
  for (int64_t n = 0; n < m.np2; ++n) {
    bool dir = n < nv ? m.bnd[n] != 0 : m.edge_dir[n - nv] != 0;
    if (!dir) {
      m.p2_to_free[n] = (int32_t)m.free_to_p2.size();
      m.free_to_p2.push_back((int32_t)n);
    }
  }
  m.nf = (int64_t)m.free_to_p2.size();
  // vertex -> cells
  m.vc_ptr.assign(nv + 1, 0);
  for (int64_t i = 0; i < 3 * nc; ++i) m.vc_ptr[m.cells[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) m.vc_ptr[v + 1] += m.vc_ptr[v];
  m.vc_idx.resize(3 * nc);
  std::vector<int32_t> fill(m.vc_ptr.begin(), m.vc_ptr.end() - 1);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) m.vc_idx[fill[m.cells[3 * c + k]]++] = (int32_t)c;
  // vertex -> vertices (edge graph); edges are lexicographic so rows come out sorted
  m.vv_ptr.assign(nv + 1, 0);
  for (int64_t e = 0; e < m.ne; ++e) {
    m.vv_ptr[m.edges[2 * e] + 1]++;
    m.vv_ptr[m.edges[2 * e + 1] + 1]++;
  }
  for (int64_t v = 0; v < nv; ++v) m.vv_ptr[v + 1] += m.vv_ptr[v];
  m.vv_idx.resize(2 * m.ne);
  fill.assign(m.vv_ptr.begin(), m.vv_ptr.end() - 1);
  for (int64_t e = 0; e < m.ne; ++e) {
    int32_t a = m.edges[2 * e], b = m.edges[2 * e + 1];
    m.vv_idx[fill[a]++] = b;
    m.vv_idx[fill[b]++] = a;
  }
  for (int64_t v = 0; v < nv; ++v)
    std::sort(m.vv_idx.begin() + m.vv_ptr[v], m.vv_idx.begin() + m.vv_ptr[v + 1]);
}

std::string build_mesh(const double* xy, const int64_t* cells, const uint8_t* bnd, int64_t nv,
                       int64_t nc, HostMesh& m) {
  if (nv < 3 || nc < 1) return "mesh needs at least one triangle";
  if (nv > (1LL << 30) || nc > (1LL << 29)) return "mesh too large for 32-bit indices";
  m.nv = nv;
  m.nc = nc;
  m.xy.assign(xy, xy + 2 * nv);
  m.bnd.assign(bnd, bnd + nv);
  m.cells.resize(3 * nc);
  for (int64_t i = 0; i < 3 * nc; ++i) {
    if (cells[i] < 0 || cells[i] >= nv) return "cell vertex id out of range";
    m.cells[i] = (int32_t)cells[i];
  }
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* t = &m.cells[3 * c];
    if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) return "degenerate cell";
    double d1x = xy[2 * t[1]] - xy[2 * t[0]], d1y = xy[2 * t[1] + 1] - xy[2 * t[0] + 1];
    double d2x = xy[2 * t[2]] - xy[2 * t[0]], d2y = xy[2 * t[2] + 1] - xy[2 * t[0] + 1];
    if (std::fabs(d1x * d2y - d1y * d2x) <= 0.0) return "zero-area cell";
  }
  finish_mesh(m);
  return "";
}

// Red refinement: coarse vertices keep their ids, edge e gets vertex nv + e;
// the children of (a, b, c) are (a, m01, m02), (m01, b, m12), (m02, m12, c),
// (m01, m12, m02) with ids 4c + k.
void refine_mesh(const HostMesh& c, HostMesh& f) {
  f = HostMesh();
  f.nv = c.np2;
  f.nc = 4 * c.nc;
  f.xy.resize(2 * f.nv);
  std::copy(c.xy.begin(), c.xy.end(), f.xy.begin());
  f.bnd.resize(f.nv);
  std::copy(c.bnd.begin(), c.bnd.end(), f.bnd.begin());
  for (int64_t e = 0; e < c.ne; ++e) {
    int32_t a = c.edges[2 * e], b = c.edges[2 * e + 1];
    f.xy[2 * (c.nv + e)] = 0.5 * (c.xy[2 * a] + c.xy[2 * b]);
    f.xy[2 * (c.nv + e) + 1] = 0.5 * (c.xy[2 * a + 1] + c.xy[2 * b + 1]);
    f.bnd[c.nv + e] = c.edge_dir[e];
  }
  f.cells.resize(3 * f.nc);
  for (int64_t k = 0; k < c.nc; ++k) {
    int32_t a = c.cells[3 * k], b = c.cells[3 * k + 1], cc = c.cells[3 * k + 2];
    int32_t m01 = (int32_t)(c.nv + c.cell_edges[3 * k]);
    int32_t m12 = (int32_t)(c.nv + c.cell_edges[3 * k + 1]);
    int32_t m02 = (int32_t)(c.nv + c.cell_edges[3 * k + 2]);
    int32_t kids[4][3] = {{a, m01, m02}, {m01, b, m12}, {m02, m12, cc}, {m01, m12, m02}};
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < 3; ++j) f.cells[3 * (4 * k + q) + j] = kids[q][j];
  }
  finish_mesh(f);
}

// Canonical interpolation weights of a red refinement, in closed form:
//  * a fine vertex is a coarse P2 node (same id): weight 1;
//  * the midpoint of a fine edge (u, m) with u a coarse vertex and m the
//    midpoint of coarse edge (u, w) sits at barycentrics (3/4, 1/4) on that
//    edge: weights 3/8 (u), -1/8 (w), 3/4 (edge node m);
//  * the midpoint of a fine edge (m1, m2) joining the midpoints of coarse
//    edges (a, b) and (b, c) sits at (1/4, 1/2, 1/4) in (a, b, c): weights
//    -1/8 (a), 0 (b), -1/8 (c), 1/2 (m1), 1/2 (m2), 1/4 (edge node of (a, c)).
//  P1: a fine vertex at a coarse vertex takes it with weight 1, a midpoint
//  takes 1/2 from each end.
void build_prolongation(const HostMesh& c, const HostMesh& f, HostCSR& Pu, HostCSR& Pp) {
  const int64_t nvc = c.nv;
  // P2, all nodes, then restrict to free rows / cols
  std::vector<std::vector<std::pair<int32_t, double>>> rows(f.np2);
  for (int64_t v = 0; v < f.nv; ++v) rows[v].push_back({(int32_t)v, 1.0});
  for (int64_t e = 0; e < f.ne; ++e) {
    int32_t u = f.edges[2 * e], w = f.edges[2 * e + 1];  // u < w
    auto& row = rows[f.nv + e];
    if (u < nvc) {
      // w is the midpoint of coarse edge (u, other)
      int64_t ce = w - nvc;
      int32_t a = c.edges[2 * ce], b = c.edges[2 * ce + 1];
      int32_t other = (a == u) ? b : a;
      row.push_back({u, 3.0 / 8.0});
      row.push_back({other, -1.0 / 8.0});
      row.push_back({w, 3.0 / 4.0});
    } else {
      int64_t e1 = u - nvc, e2 = w - nvc;
      int32_t a1 = c.edges[2 * e1], b1 = c.edges[2 * e1 + 1];
      int32_t a2 = c.edges[2 * e2], b2 = c.edges[2 * e2 + 1];
      int32_t shared = (a1 == a2 || a1 == b2) ? a1 : b1;
      int32_t p = (a1 == shared) ? b1 : a1;
      int32_t q = (a2 == shared) ? b2 : a2;
      int64_t e3 = find_edge(c, p, q);
      row.push_back({p, -1.0 / 8.0});
      row.push_back({q, -1.0 / 8.0});
      row.push_back({u, 0.5});
      row.push_back({w, 0.5});
      row.push_back({(int32_t)(nvc + e3), 0.25});
    }
  }
  Pu = HostCSR();
  Pu.nrows = f.nf;
  Pu.ncols = c.nf;
  Pu.ptr.assign(1, 0);
  for (int64_t i = 0; i < f.nf; ++i) {
    auto row = rows[f.free_to_p2[i]];
    std::sort(row.begin(), row.end());
    for (auto& pr : row) {
      int32_t cf = c.p2_to_free[pr.first];
      if (cf < 0 || pr.second == 0.0) continue;
      Pu.col.push_back(cf);
      Pu.v[0].push_back(pr.second);
    }
    Pu.ptr.push_back((int32_t)Pu.col.size());
  }
  Pp = HostCSR();
  Pp.nrows = f.nv;
  Pp.ncols = c.nv;
  Pp.ptr.assign(1, 0);
  for (int64_t v = 0; v < f.nv; ++v) {
    if (v < nvc) {
      Pp.col.push_back((int32_t)v);
      Pp.v[0].push_back(1.0);
    } else {
      int64_t ce = v - nvc;
      Pp.col.push_back(c.edges[2 * ce]);
      Pp.v[0].push_back(0.5);
      Pp.col.push_back(c.edges[2 * ce + 1]);
      Pp.v[0].push_back(0.5);
    }
    Pp.ptr.push_back((int32_t)Pp.col.size());
  }
}

HostCSR transpose_csr(const HostCSR& A, int nvals) {
  HostCSR T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.ptr.assign(T.nrows + 1, 0);
  for (int32_t j : A.col) T.ptr[j + 1]++;
  for (int64_t i = 0; i < T.nrows; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  for (int k = 0; k < nvals; ++k) T.v[k].resize(A.col.size());
  std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int64_t i = 0; i < A.nrows; ++i)  // ascending rows -> sorted columns of T
    for (int32_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
      int32_t j = A.col[p];
      int32_t q = fill[j]++;
      T.col[q] = (int32_t)i;
      for (int k = 0; k < nvals; ++k) T.v[k][q] = A.v[k][p];
    }
  return T;
}

// Radau IIA(s), s = 1..3, in closed form (Hairer & Wanner, Solving ODEs II,
// Section IV.5); the paper uses RadauIIA(2) and RadauIIA(3) (Section 5).
int radau_iia(int s, double* A, double* b, double* c) {
  if (s == 1) {
    A[0] = 1.0;
    b[0] = 1.0;
    c[0] = 1.0;
    return IRKMG_OK;
  }
  if (s == 2) {
    const double a[4] = {5.0 / 12.0, -1.0 / 12.0, 3.0 / 4.0, 1.0 / 4.0};
    std::copy(a, a + 4, A);
    b[0] = 3.0 / 4.0;
    b[1] = 1.0 / 4.0;
    c[0] = 1.0 / 3.0;
    c[1] = 1.0;
    return IRKMG_OK;
  }
  if (s == 3) {
    const double r6 = std::sqrt(6.0);
    const double a[9] = {(88.0 - 7.0 * r6) / 360.0,   (296.0 - 169.0 * r6) / 1800.0,
                         (-2.0 + 3.0 * r6) / 225.0,   (296.0 + 169.0 * r6) / 1800.0,
                         (88.0 + 7.0 * r6) / 360.0,   (-2.0 - 3.0 * r6) / 225.0,
                         (16.0 - r6) / 36.0,          (16.0 + r6) / 36.0,
                         1.0 / 9.0};
    std::copy(a, a + 9, A);
    for (int j = 0; j < 3; ++j) b[j] = a[6 + j];
    c[0] = (4.0 - r6) / 10.0;
    c[1] = (4.0 + r6) / 10.0;
    c[2] = 1.0;
    return IRKMG_OK;
  }
  return IRKMG_EINVAL;
}

}  // namespace irkmg

// Host-side mesh hierarchy, numbering, transfer weights and Butcher tableau.
//
// Section 4.1: levels are uniform refinements of a coarsest simplicial mesh
// (red refinement of triangles, Bey's refinement of tetrahedra), and
// prolongation is canonical P2 (velocity) / P1 (pressure) interpolation;
// restriction is its transpose.  Section 5: RadauIIA(s).
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include <cstdlib>
#include <thread>

#include "irkmg_internal.h"

namespace irkmg {

// local edges of a cell; triangles use the first three
const int kLocalEdges[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};

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
  const int kv = m.nvc(), ke = m.nle();
  // edges: sorted vertex pairs, unique, lexicographic
  std::vector<uint64_t> keys(ke * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < ke; ++k) {
      int32_t a = m.cells[kv * c + kLocalEdges[k][0]], b = m.cells[kv * c + kLocalEdges[k][1]];
      if (a > b) std::swap(a, b);
      keys[ke * c + k] = key2(a, b);
    }
  std::vector<uint64_t> uniq = keys;
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  m.ne = (int64_t)uniq.size();
  m.edges.resize(2 * m.ne);
  for (int64_t e = 0; e < m.ne; ++e) {
    m.edges[2 * e] = (int32_t)(uniq[e] >> 32);
    m.edges[2 * e + 1] = (int32_t)(uniq[e] & 0xffffffffu);
  }
  m.cell_edges.resize(ke * nc);
  for (int64_t i = 0; i < ke * nc; ++i)
    m.cell_edges[i] =
        (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), keys[i]) - uniq.begin());
  // boundary facets (edges in 2D, faces in 3D) belong to exactly one cell;
  // an edge is on the boundary iff it lies in a boundary facet
  std::vector<uint8_t> on_bnd(m.ne, 0);
  if (m.dim == 2) {
    std::vector<int32_t> cnt(m.ne, 0);
    for (int32_t e : m.cell_edges) cnt[e]++;
    for (int64_t e = 0; e < m.ne; ++e) on_bnd[e] = cnt[e] == 1;
  } else {
    std::vector<std::array<int32_t, 3>> faces;
    faces.reserve(4 * nc);
    static const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    for (int64_t c = 0; c < nc; ++c)
      for (int f = 0; f < 4; ++f) {
        std::array<int32_t, 3> t = {m.cells[4 * c + fv[f][0]], m.cells[4 * c + fv[f][1]],
                                    m.cells[4 * c + fv[f][2]]};
        std::sort(t.begin(), t.end());
        faces.push_back(t);
      }
    std::sort(faces.begin(), faces.end());
    for (size_t i = 0; i < faces.size();) {
      size_t j = i;
      while (j < faces.size() && faces[j] == faces[i]) ++j;
      if (j - i == 1) {
        const auto& t = faces[i];
        for (int a = 0; a < 3; ++a)
          for (int b = a + 1; b < 3; ++b) on_bnd[find_edge(m, t[a], t[b])] = 1;
      }
      i = j;
    }
  }
  m.edge_dir.assign(m.ne, 0);
  for (int64_t e = 0; e < m.ne; ++e)
    m.edge_dir[e] = (on_bnd[e] && m.bnd[m.edges[2 * e]] && m.bnd[m.edges[2 * e + 1]]) ? 1 : 0;
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
  for (int64_t i = 0; i < kv * nc; ++i) m.vc_ptr[m.cells[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) m.vc_ptr[v + 1] += m.vc_ptr[v];
  m.vc_idx.resize(kv * nc);
  std::vector<int32_t> fill(m.vc_ptr.begin(), m.vc_ptr.end() - 1);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < kv; ++k) m.vc_idx[fill[m.cells[kv * c + k]]++] = (int32_t)c;
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
                       int64_t nc, int dim, HostMesh& m) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  const int kv = dim + 1;
  if (nv < kv || nc < 1) return "mesh needs at least one cell";
  if (nv > (1LL << 30) || nc > (1LL << 28)) return "mesh too large for 32-bit indices";
  m.dim = dim;
  m.nv = nv;
  m.nc = nc;
  m.xy.assign(xy, xy + dim * nv);
  m.bnd.assign(bnd, bnd + nv);
  m.cells.resize(kv * nc);
  for (int64_t i = 0; i < kv * nc; ++i) {
    if (cells[i] < 0 || cells[i] >= nv) return "cell vertex id out of range";
    m.cells[i] = (int32_t)cells[i];
  }
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* t = &m.cells[kv * c];
    for (int a = 0; a < kv; ++a)
      for (int b = a + 1; b < kv; ++b)
        if (t[a] == t[b]) return "degenerate cell";
    double J[3][3] = {{0}};
    for (int i = 0; i < dim; ++i)
      for (int k = 0; k < dim; ++k) J[k][i] = xy[dim * t[i + 1] + k] - xy[dim * t[0] + k];
    const double det = dim == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                                : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                      J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                      J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (std::fabs(det) <= 0.0) return "zero-volume cell";
  }
  finish_mesh(m);
  return "";
}

// Uniform refinement.  Coarse vertices keep their ids and edge e gets vertex
// nv + e.  Triangles (red): the children of (a, b, c) are (a, m01, m02),
// (m01, b, m12), (m02, m12, c), (m01, m12, m02) with ids 4c + k.
// Tetrahedra (Bey): the children of (x0, x1, x2, x3) are (x0, x01, x02, x03),
// (x01, x1, x12, x13), (x02, x12, x2, x23), (x03, x13, x23, x3) and the inner
// octahedron cut along x02-x13: (x01, x02, x03, x13), (x01, x02, x12, x13),
// (x02, x03, x13, x23), (x02, x12, x13, x23), with ids 8c + k.
void refine_mesh(const HostMesh& c, HostMesh& f) {
  const int d = c.dim;
  f = HostMesh();
  f.dim = d;
  f.nv = c.np2;
  f.nc = (d == 2 ? 4 : 8) * c.nc;
  f.xy.resize(d * f.nv);
  std::copy(c.xy.begin(), c.xy.end(), f.xy.begin());
  f.bnd.resize(f.nv);
  std::copy(c.bnd.begin(), c.bnd.end(), f.bnd.begin());
  for (int64_t e = 0; e < c.ne; ++e) {
    int32_t a = c.edges[2 * e], b = c.edges[2 * e + 1];
    for (int k = 0; k < d; ++k) f.xy[d * (c.nv + e) + k] = 0.5 * (c.xy[d * a + k] + c.xy[d * b + k]);
    f.bnd[c.nv + e] = c.edge_dir[e];
  }
  const int kv = d + 1, ke = c.nle();
  f.cells.resize(kv * f.nc);
  for (int64_t k = 0; k < c.nc; ++k) {
    const int32_t* x = &c.cells[kv * k];
    int32_t m[6];
    for (int e = 0; e < ke; ++e) m[e] = (int32_t)(c.nv + c.cell_edges[ke * k + e]);
    if (d == 2) {
      // m[0] = m01, m[1] = m12, m[2] = m02
      const int32_t kids[4][3] = {{x[0], m[0], m[2]}, {m[0], x[1], m[1]}, {m[2], m[1], x[2]},
                                  {m[0], m[1], m[2]}};
      for (int q = 0; q < 4; ++q)
        for (int j = 0; j < 3; ++j) f.cells[3 * (4 * k + q) + j] = kids[q][j];
    } else {
      // m01 = m[0], m12 = m[1], m02 = m[2], m03 = m[3], m13 = m[4], m23 = m[5]
      const int32_t m01 = m[0], m12 = m[1], m02 = m[2], m03 = m[3], m13 = m[4], m23 = m[5];
      const int32_t kids[8][4] = {{x[0], m01, m02, m03}, {m01, x[1], m12, m13},
                                  {m02, m12, x[2], m23}, {m03, m13, m23, x[3]},
                                  {m01, m02, m03, m13},  {m01, m02, m12, m13},
                                  {m02, m03, m13, m23},  {m02, m12, m13, m23}};
      for (int q = 0; q < 8; ++q)
        for (int j = 0; j < 4; ++j) f.cells[4 * (8 * k + q) + j] = kids[q][j];
    }
  }
  finish_mesh(f);
}

// Canonical interpolation weights of a uniform refinement, in closed form:
//  * a fine vertex is a coarse P2 node (same id): weight 1;
//  * the midpoint of a fine edge (u, m) with u a coarse vertex and m the
//    midpoint of coarse edge (u, w) sits at barycentrics (3/4, 1/4) on that
//    edge: weights 3/8 (u), -1/8 (w), 3/4 (edge node m);
//  * the midpoint of a fine edge (m1, m2) joining the midpoints of two coarse
//    edges (p, b) and (b, q) that share the vertex b sits at (1/4, 1/2, 1/4) in
//    the face (p, b, q): weights -1/8 (p), 0 (b), -1/8 (q), 1/2 (m1), 1/2 (m2),
//    1/4 (edge node of (p, q));
//  * (tetrahedra) the midpoint of the fine edge joining the midpoints of two
//    opposite coarse edges is the centroid, barycentrics 1/4 each: weight
//    -1/8 at the four vertices and 1/4 at the six edge nodes.
//  P1: a fine vertex at a coarse vertex takes it with weight 1, a midpoint
//  takes 1/2 from each end.
void build_prolongation(const HostMesh& c, const HostMesh& f, HostCSR& Pu, HostCSR& Pp) {
  const int64_t nvc = c.nv;
  std::vector<std::vector<std::pair<int32_t, double>>> rows(f.np2);
  for (int64_t v = 0; v < f.nv; ++v) rows[v].push_back({(int32_t)v, 1.0});
  auto enode = [&](int32_t a, int32_t b) { return (int32_t)(nvc + find_edge(c, a, b)); };
  for (int64_t e = 0; e < f.ne; ++e) {
    int32_t u = f.edges[2 * e], w = f.edges[2 * e + 1];  // u < w
    auto& row = rows[f.nv + e];
    if (u < nvc) {
      const int64_t ce = w - nvc;
      const int32_t a = c.edges[2 * ce], b = c.edges[2 * ce + 1];
      const int32_t other = (a == u) ? b : a;
      row.push_back({u, 3.0 / 8.0});
      row.push_back({other, -1.0 / 8.0});
      row.push_back({w, 3.0 / 4.0});
      continue;
    }
    const int64_t e1 = u - nvc, e2 = w - nvc;
    const int32_t a1 = c.edges[2 * e1], b1 = c.edges[2 * e1 + 1];
    const int32_t a2 = c.edges[2 * e2], b2 = c.edges[2 * e2 + 1];
    int32_t shared = -1;
    if (a1 == a2 || a1 == b2) shared = a1;
    if (b1 == a2 || b1 == b2) shared = b1;
    if (shared >= 0) {
      const int32_t p = (a1 == shared) ? b1 : a1;
      const int32_t q = (a2 == shared) ? b2 : a2;
      row.push_back({p, -1.0 / 8.0});
      row.push_back({q, -1.0 / 8.0});
      row.push_back({u, 0.5});
      row.push_back({w, 0.5});
      row.push_back({enode(p, q), 0.25});
    } else {
      const int32_t vt[4] = {a1, b1, a2, b2};
      for (int i = 0; i < 4; ++i) row.push_back({vt[i], -1.0 / 8.0});
      for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) row.push_back({enode(vt[i], vt[j]), 0.25});
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
      const int64_t ce = v - nvc;
      Pp.col.push_back(c.edges[2 * ce]);
      Pp.v[0].push_back(0.5);
      Pp.col.push_back(c.edges[2 * ce + 1]);
      Pp.v[0].push_back(0.5);
    }
    Pp.ptr.push_back((int32_t)Pp.col.size());
  }
}

unsigned host_threads() {
  if (const char* e = std::getenv("IRKMG_HOST_THREADS")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 1) return (unsigned)std::min(v, 64L);
  }
  const unsigned T = std::thread::hardware_concurrency();
  return std::max(1u, std::min(T, 64u));
}

// Counting-sort transpose; with many rows, T threads take contiguous row
// ranges, count their columns, and write their entries at offsets that
// follow the ranges in order, so every column of the result lists its rows
// in ascending order whatever T is.
HostCSR transpose_csr(const HostCSR& A, int nvals) {
  HostCSR T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.col.resize(A.col.size());
  for (int k = 0; k < nvals; ++k) T.v[k].resize(A.col.size());
  const unsigned nt = A.nrows >= 65536 ? host_threads() : 1u;
  const int64_t chunk = (A.nrows + nt - 1) / nt;
  std::vector<std::vector<int32_t>> cnt(nt);
  auto run = [&](auto&& f) {
    std::vector<std::thread> th;
    for (unsigned k = 1; k < nt; ++k) th.emplace_back(f, k);
    f(0u);
    for (auto& t : th) t.join();
  };
  run([&](unsigned k) {
    std::vector<int32_t>& c = cnt[k];
    c.assign(T.nrows, 0);
    for (int64_t i = k * chunk; i < std::min<int64_t>(A.nrows, (k + 1) * chunk); ++i)
      for (int32_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) c[A.col[p]]++;
  });
  T.ptr.assign(T.nrows + 1, 0);
  for (int64_t j = 0; j < T.nrows; ++j) {  // column j: range k's rows start after range k-1's
    int32_t o = T.ptr[j];
    for (unsigned k = 0; k < nt; ++k) {
      const int32_t c = cnt[k][j];
      cnt[k][j] = o;
      o += c;
    }
    T.ptr[j + 1] = o;
  }
  run([&](unsigned k) {
    std::vector<int32_t>& fill = cnt[k];
    for (int64_t i = k * chunk; i < std::min<int64_t>(A.nrows, (k + 1) * chunk); ++i)
      for (int32_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        const int32_t q = fill[A.col[p]]++;
        T.col[q] = (int32_t)i;
        for (int v = 0; v < nvals; ++v) T.v[v][q] = A.v[v][p];
      }
  });
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

// Gauss(s) (collocation at the Gauss points, order 2s) and LobattoIIIC(s)
// (Lobatto points, order 2s - 2, L-stable), s = 2, 3, in closed form (Hairer &
// Wanner, Section IV.5); the paper runs both beside RadauIIA (Section 5).
int gauss_tableau(int s, double* A, double* b, double* c) {
  if (s == 2) {
    const double r3 = std::sqrt(3.0);
    const double a[4] = {0.25, 0.25 - r3 / 6.0, 0.25 + r3 / 6.0, 0.25};
    std::copy(a, a + 4, A);
    b[0] = b[1] = 0.5;
    c[0] = 0.5 - r3 / 6.0;
    c[1] = 0.5 + r3 / 6.0;
    return IRKMG_OK;
  }
  if (s == 3) {
    const double r = std::sqrt(15.0);
    const double a[9] = {5.0 / 36.0,          2.0 / 9.0 - r / 15.0, 5.0 / 36.0 - r / 30.0,
                         5.0 / 36.0 + r / 24.0, 2.0 / 9.0,            5.0 / 36.0 - r / 24.0,
                         5.0 / 36.0 + r / 30.0, 2.0 / 9.0 + r / 15.0, 5.0 / 36.0};
    std::copy(a, a + 9, A);
    b[0] = 5.0 / 18.0;
    b[1] = 4.0 / 9.0;
    b[2] = 5.0 / 18.0;
    c[0] = 0.5 - r / 10.0;
    c[1] = 0.5;
    c[2] = 0.5 + r / 10.0;
    return IRKMG_OK;
  }
  return IRKMG_EINVAL;
}

int lobatto_iiic_tableau(int s, double* A, double* b, double* c) {
  if (s == 2) {
    const double a[4] = {0.5, -0.5, 0.5, 0.5};
    std::copy(a, a + 4, A);
    b[0] = b[1] = 0.5;
    c[0] = 0.0;
    c[1] = 1.0;
    return IRKMG_OK;
  }
  if (s == 3) {
    const double a[9] = {1.0 / 6.0, -1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 5.0 / 12.0,
                         -1.0 / 12.0, 1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    std::copy(a, a + 9, A);
    b[0] = 1.0 / 6.0;
    b[1] = 2.0 / 3.0;
    b[2] = 1.0 / 6.0;
    c[0] = 0.0;
    c[1] = 0.5;
    c[2] = 1.0;
    return IRKMG_OK;
  }
  return IRKMG_EINVAL;
}

}  // namespace irkmg

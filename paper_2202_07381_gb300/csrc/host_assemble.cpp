// Host-side assembly of the Taylor–Hood P2–P1 operators of one level
// (Section 3.1: M, K, B with B the weak gradient from -<p, div v>;
// Section 3.2: Oseen convection <(w . grad) u, v> for a frozen wind w, 2D).
//
// Element integrals are exact quadratures on affine simplices: the 7-point
// degree-5 rule of Radon (Stroud T2:5-1) on triangles, and on tetrahedra the
// collapsed (Duffy) product of 4-point Gauss–Legendre rules, exact for
// degree 7 in each collapsed direction, hence for every integrand of degree
// <= 5 here (mass degree 4, stiffness and gradient degree 2).
#include <algorithm>
#include <array>
#include <cmath>
#include <memory>
#include <thread>

#include "irkmg_internal.h"

namespace irkmg {

namespace {

struct QuadRule {
  std::vector<std::array<double, 4>> lam;  // barycentric coordinates
  std::vector<double> w;                   // weights sum to 1 (multiply by the volume)
};

QuadRule radon7() {
  QuadRule q;
  const double r15 = std::sqrt(15.0);
  const double a1 = (6.0 - r15) / 21.0, a2 = (6.0 + r15) / 21.0;
  const double w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
  q.lam.push_back({1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 0.0});
  q.w.push_back(9.0 / 40.0);
  const double as[2] = {a1, a2}, ws[2] = {w1, w2};
  for (int g = 0; g < 2; ++g)
    for (int r = 0; r < 3; ++r) {
      std::array<double, 4> l = {as[g], as[g], as[g], 0.0};
      l[r] = 1.0 - 2.0 * as[g];
      q.lam.push_back(l);
      q.w.push_back(ws[g]);
    }
  return q;
}

QuadRule duffy_tet() {
  // 4-point Gauss–Legendre on [-1, 1]: nodes +-sqrt((3 -+ 2 sqrt(6/5)) / 7),
  // weights (18 +- sqrt(30)) / 36, mapped to [0, 1]
  const double s65 = std::sqrt(6.0 / 5.0), s30 = std::sqrt(30.0);
  const double x1 = std::sqrt((3.0 - 2.0 * s65) / 7.0), x2 = std::sqrt((3.0 + 2.0 * s65) / 7.0);
  const double w1 = (18.0 + s30) / 36.0, w2 = (18.0 - s30) / 36.0;
  const double xs[4] = {-x2, -x1, x1, x2}, wsg[4] = {w2, w1, w1, w2};
  QuadRule q;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) {
        const double u = 0.5 * (xs[i] + 1), v = 0.5 * (xs[j] + 1), t = 0.5 * (xs[k] + 1);
        const double x = u, y = v * (1 - u), z = t * (1 - u) * (1 - v);
        // reference volume 1/6: weights scaled by 6 to sum to one
        const double wt = 6.0 * 0.125 * wsg[i] * wsg[j] * wsg[k] * (1 - u) * (1 - u) * (1 - v);
        q.lam.push_back({1.0 - x - y - z, x, y, z});
        q.w.push_back(wt);
      }
  return q;
}

// P2 basis on barycentrics: vertex i -> l_i (2 l_i - 1); edge (i, j) -> 4 l_i l_j
// in the local edge order; gradients by the chain rule from grad l.
inline void p2_eval(int d, const double* l, const double gl[4][3], double* phi,
                    double gphi[10][3]) {
  const int kv = d + 1, ke = d == 2 ? 3 : 6;
  for (int i = 0; i < kv; ++i) {
    phi[i] = l[i] * (2.0 * l[i] - 1.0);
    for (int c = 0; c < d; ++c) gphi[i][c] = (4.0 * l[i] - 1.0) * gl[i][c];
  }
  for (int e = 0; e < ke; ++e) {
    const int i = kLocalEdges[e][0], j = kLocalEdges[e][1];
    phi[kv + e] = 4.0 * l[i] * l[j];
    for (int c = 0; c < d; ++c) gphi[kv + e][c] = 4.0 * (l[j] * gl[i][c] + l[i] * gl[j][c]);
  }
}

// Volume and barycentric gradients of cell c.
double cell_geometry(const HostMesh& m, int64_t c, double gl[4][3]) {
  const int d = m.dim;
  const int32_t* t = &m.cells[(d + 1) * c];
  double J[3][3] = {{0}};
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) J[k][i] = m.xy[d * t[i + 1] + k] - m.xy[d * t[0] + k];
  if (d == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    // rows of J^{-1} are grad l_1, grad l_2
    gl[1][0] = J[1][1] / det;
    gl[1][1] = -J[0][1] / det;
    gl[2][0] = -J[1][0] / det;
    gl[2][1] = J[0][0] / det;
    gl[0][0] = -gl[1][0] - gl[2][0];
    gl[0][1] = -gl[1][1] - gl[2][1];
    return 0.5 * std::fabs(det);
  }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) gl[i + 1][k] = inv[i][k];
  for (int k = 0; k < 3; ++k) gl[0][k] = -gl[1][k] - gl[2][k] - gl[3][k];
  return std::fabs(det) / 6.0;
}

// Find the slot of column `col` in row `row` of a CSR with sorted columns.
inline int64_t slot(const HostCSR& A, int64_t row, int32_t col) {
  auto b = A.col.begin() + A.ptr[row], e = A.col.begin() + A.ptr[row + 1];
  auto it = std::lower_bound(b, e, col);
  return (it != e && *it == col) ? (it - A.col.begin()) : -1;
}

// f(lo, hi) over contiguous ranges of [0, n), one per host thread (serially
// below min_n); every index is handled by exactly one call, so no result
// depends on the thread count.
template <typename F>
void parallel_ranges(int64_t n, F f, int64_t min_n = 2048) {
  const unsigned T = host_threads();
  if (T == 1 || n < min_n) {
    f((int64_t)0, n);
    return;
  }
  const int64_t chunk = (n + T - 1) / T;
  std::vector<std::thread> th;
  for (unsigned k = 1; k < T; ++k) {
    const int64_t lo = k * chunk, hi = std::min(n, lo + chunk);
    if (lo < hi) th.emplace_back(f, lo, hi);
  }
  f((int64_t)0, std::min(n, chunk));
  for (auto& t : th) t.join();
}

// Element matrices of cell c: Me, Ke (nn x nn, row-major) and Be (d x nn x kv).
void cell_matrices(const HostMesh& m, const QuadRule& q, double nu, const double* wind, int64_t c,
                   double* Me, double* Ke, double* Be) {
  const int d = m.dim, kv = m.nvc(), nn = m.nn(), nq = (int)q.w.size();
  double gl[4][3];
  const double vol = cell_geometry(m, c, gl);
  int32_t node[10];
  for (int a = 0; a < nn; ++a)
    node[a] = a < kv ? m.cells[kv * c + a] : (int32_t)(m.nv + m.cell_edges[m.nle() * c + a - kv]);
  for (int a = 0; a < nn * nn; ++a) Me[a] = Ke[a] = 0.0;
  for (int a = 0; a < d * nn * kv; ++a) Be[a] = 0.0;
  for (int iq = 0; iq < nq; ++iq) {
    double phi[10], g[10][3];
    p2_eval(d, q.lam[iq].data(), gl, phi, g);
    const double wk = q.w[iq] * vol;
    double wv[3] = {0.0, 0.0, 0.0};
    if (wind && d == 2)
      for (int a = 0; a < nn; ++a)
        for (int k = 0; k < d; ++k) wv[k] += wind[d * node[a] + k] * phi[a];
    for (int a = 0; a < nn; ++a) {
      for (int b = 0; b < nn; ++b) {
        Me[a * nn + b] += wk * phi[a] * phi[b];
        double gg = 0.0, conv = 0.0;
        for (int k = 0; k < d; ++k) {
          gg += g[a][k] * g[b][k];
          conv += wv[k] * g[b][k];
        }
        Ke[a * nn + b] += wk * (nu * gg + (wind && d == 2 ? conv * phi[a] : 0.0));
      }
      for (int p = 0; p < kv; ++p)
        for (int k = 0; k < d; ++k) Be[(k * nn + a) * kv + p] -= wk * q.lam[iq][p] * g[a][k];
    }
  }
}

}  // namespace

// Every part is computed per row (or per cell) in parallel host threads.  A
// stored entry is the sum of its cells' element entries taken in ascending
// cell order, so the operators do not depend on the thread count.
void assemble_level(const HostMesh& m, double nu, const double* wind, HostOps& ops) {
  const int d = m.dim, kv = m.nvc(), nn = m.nn();
  const QuadRule q = d == 2 ? radon7() : duffy_tet();
  auto cell_node = [&](int64_t c, int a) -> int32_t {
    return a < kv ? m.cells[kv * c + a] : (int32_t)(m.nv + m.cell_edges[m.nle() * c + a - kv]);
  };
  // node -> cells in ascending order
  std::vector<int32_t> nc_ptr(m.np2 + 1, 0), nc_idx(nn * m.nc);
  for (int64_t c = 0; c < m.nc; ++c)
    for (int a = 0; a < nn; ++a) nc_ptr[cell_node(c, a) + 1]++;
  for (int64_t n = 0; n < m.np2; ++n) nc_ptr[n + 1] += nc_ptr[n];
  {
    std::vector<int32_t> fill(nc_ptr.begin(), nc_ptr.end() - 1);
    for (int64_t c = 0; c < m.nc; ++c)
      for (int a = 0; a < nn; ++a) nc_idx[fill[cell_node(c, a)]++] = (int32_t)c;
  }
  // element matrices of every cell
  // (uninitialised: cell_matrices writes every entry, first touch in parallel)
  const int64_t sM = (int64_t)nn * nn, sB = (int64_t)d * nn * kv;
  std::unique_ptr<double[]> Mall(new double[sM * m.nc]), Kall(new double[sM * m.nc]),
      Ball(new double[sB * m.nc]);
  parallel_ranges(m.nc, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; ++c)
      cell_matrices(m, q, nu, wind, c, &Mall[sM * c], &Kall[sM * c], &Ball[sB * c]);
  });
  // sparsity patterns by union over each row's cells, per thread range, then joined
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
  {
    struct Part {
      std::vector<int32_t> vc, mc, bc, vn, mn, bn;  // columns, then per-row counts
    };
    const unsigned T = host_threads();
    const int64_t chunk = (m.nf + T - 1) / T;
    std::vector<Part> part(T);
    parallel_ranges((int64_t)T, [&](int64_t k0, int64_t k1) {
      std::vector<int32_t> nodes, verts;
      for (int64_t k = k0; k < k1; ++k) {
        Part& P = part[k];
        for (int64_t i = k * chunk; i < std::min<int64_t>(m.nf, (k + 1) * chunk); ++i) {
          const int32_t n = m.free_to_p2[i];
          nodes.clear();
          verts.clear();
          for (int32_t p = nc_ptr[n]; p < nc_ptr[n + 1]; ++p) {
            const int64_t c = nc_idx[p];
            for (int a = 0; a < nn; ++a) nodes.push_back(cell_node(c, a));
            for (int a = 0; a < kv; ++a) verts.push_back(m.cells[kv * c + a]);
          }
          std::sort(nodes.begin(), nodes.end());
          nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
          std::sort(verts.begin(), verts.end());
          verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
          int32_t nvc = 0;
          for (int32_t x : nodes) {
            P.mc.push_back(x);
            if (m.p2_to_free[x] >= 0) {
              P.vc.push_back(m.p2_to_free[x]);
              ++nvc;
            }
          }
          for (int32_t x : verts) P.bc.push_back(x);
          P.vn.push_back(nvc);
          P.mn.push_back((int32_t)nodes.size());
          P.bn.push_back((int32_t)verts.size());
        }
      }
    }, 1);
    auto join = [&](HostCSR& A, std::vector<int32_t> Part::*cols, std::vector<int32_t> Part::*cnt) {
      A.ptr.assign(1, 0);
      for (const Part& P : part) {
        for (int32_t k : P.*cnt) A.ptr.push_back(A.ptr.back() + k);
        A.col.insert(A.col.end(), (P.*cols).begin(), (P.*cols).end());
      }
    };
    join(V, &Part::vc, &Part::vn);
    join(MA, &Part::mc, &Part::mn);
    join(B, &Part::bc, &Part::bn);
  }
  V.v[0].assign(V.col.size(), 0.0);
  V.v[1].assign(V.col.size(), 0.0);
  MA.v[0].assign(MA.col.size(), 0.0);
  MA.v[1].assign(MA.col.size(), 0.0);
  for (int c = 0; c < d; ++c) B.v[c].assign(B.col.size(), 0.0);
  // values: each free row takes row a of its cells' element matrices
  parallel_ranges(m.nf, [&](int64_t lo, int64_t hi) {
    for (int64_t row = lo; row < hi; ++row) {
      const int32_t n = m.free_to_p2[row];
      for (int32_t p = nc_ptr[n]; p < nc_ptr[n + 1]; ++p) {
        const int64_t c = nc_idx[p];
        int32_t node[10];
        int a = 0;
        for (int k = 0; k < nn; ++k) {
          node[k] = cell_node(c, k);
          if (node[k] == n) a = k;
        }
        const double* Me = &Mall[sM * c + a * nn];
        const double* Ke = &Kall[sM * c + a * nn];
        const double* Be = &Ball[sB * c];
        for (int b = 0; b < nn; ++b) {
          const int64_t sa = slot(MA, row, node[b]);
          MA.v[0][sa] += Me[b];
          MA.v[1][sa] += Ke[b];
          const int32_t cf = m.p2_to_free[node[b]];
          if (cf >= 0) {
            const int64_t sv = slot(V, row, cf);
            V.v[0][sv] += Me[b];
            V.v[1][sv] += Ke[b];
          }
        }
        const int32_t* t = &m.cells[kv * c];
        for (int pp = 0; pp < kv; ++pp) {
          const int64_t sb = slot(B, row, t[pp]);
          for (int k = 0; k < d; ++k) B.v[k][sb] += Be[(k * nn + a) * kv + pp];
        }
      }
    }
  });
  // transpose of the velocity operator (same pattern, which is symmetric)
  V.v[2].resize(V.col.size());
  parallel_ranges(m.nf, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      for (int32_t p = V.ptr[i]; p < V.ptr[i + 1]; ++p) {
        const int64_t st = slot(V, V.col[p], (int32_t)i);
        V.v[2][p] = V.v[1][st];
      }
  });
  ops.bt = transpose_csr(B, d);
  // Bᵀ over every velocity column: vertex rows, P2-node columns.  Per P2
  // node, its cells' entries in cell order, summed per vertex in that order.
  HostCSR Bf;
  Bf.nrows = m.np2;
  Bf.ncols = m.nv;
  {
    struct Part {
      std::vector<int32_t> cnt, col;
      std::vector<double> v[3];
    };
    const unsigned T = host_threads();
    const int64_t chunk = (m.np2 + T - 1) / T;
    std::vector<Part> part(T);
    parallel_ranges((int64_t)T, [&](int64_t k0, int64_t k1) {
      std::vector<std::pair<int32_t, std::array<double, 3>>> e;
      for (int64_t k = k0; k < k1; ++k) {
        Part& P = part[k];
        for (int64_t n = k * chunk; n < std::min<int64_t>(m.np2, (k + 1) * chunk); ++n) {
          e.clear();
          for (int32_t p = nc_ptr[n]; p < nc_ptr[n + 1]; ++p) {
            const int64_t c = nc_idx[p];
            int a = 0;
            for (int kk = 0; kk < nn; ++kk)
              if (cell_node(c, kk) == n) a = kk;
            const double* Be = &Ball[sB * c];
            const int32_t* t = &m.cells[kv * c];
            for (int pp = 0; pp < kv; ++pp)
              e.push_back({t[pp], {Be[(0 * nn + a) * kv + pp], Be[(1 * nn + a) * kv + pp],
                                   d == 3 ? Be[(2 * nn + a) * kv + pp] : 0.0}});
          }
          std::stable_sort(e.begin(), e.end(),
                           [](const auto& x, const auto& y) { return x.first < y.first; });
          int32_t cnt = 0;
          for (size_t i = 0; i < e.size();) {
            size_t j = i;
            double sum[3] = {0.0, 0.0, 0.0};
            for (; j < e.size() && e[j].first == e[i].first; ++j)
              for (int c = 0; c < 3; ++c) sum[c] += e[j].second[c];
            P.col.push_back(e[i].first);
            for (int c = 0; c < d; ++c) P.v[c].push_back(sum[c]);
            ++cnt;
            i = j;
          }
          P.cnt.push_back(cnt);
        }
      }
    }, 1);
    Bf.ptr.assign(1, 0);
    for (const Part& P : part) {
      for (int32_t k : P.cnt) Bf.ptr.push_back(Bf.ptr.back() + k);
      Bf.col.insert(Bf.col.end(), P.col.begin(), P.col.end());
      for (int c = 0; c < d; ++c) Bf.v[c].insert(Bf.v[c].end(), P.v[c].begin(), P.v[c].end());
    }
  }
  ops.btall = transpose_csr(Bf, d);
}

// Load of a per-cell constant (P0) forcing: C[a, c] = int_c phi_a for the free
// P2 nodes a of cell c (the same for every velocity component).  P2 vertex
// functions integrate to zero on a triangle, edge functions to |c|/3.
void assemble_cell_load(const HostMesh& m, HostCSR& C) {
  C = HostCSR();
  C.nrows = m.nf;
  C.ncols = m.nc;
  C.ptr.assign(m.nf + 1, 0);
  if (m.dim != 2) return;
  const QuadRule q = radon7();
  std::vector<std::vector<std::pair<int32_t, double>>> rows(m.nf);
  for (int64_t c = 0; c < m.nc; ++c) {
    double gl[4][3];
    const double area = cell_geometry(m, c, gl);
    double w[6] = {0, 0, 0, 0, 0, 0};
    for (size_t k = 0; k < q.w.size(); ++k) {
      double phi[10], g[10][3];
      p2_eval(2, q.lam[k].data(), gl, phi, g);
      for (int a = 0; a < 6; ++a) w[a] += q.w[k] * area * phi[a];
    }
    const int32_t* t = &m.cells[3 * c];
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

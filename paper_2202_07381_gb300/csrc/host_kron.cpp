// Kronecker decoupling of the IRK patch systems.
//
// The stage operator is J = I_s ⊗ M̂ + Δt A ⊗ K̂ (Section 3, the Kronecker
// form of the fully implicit stage system), and a vertex-star patch takes the
// same spatial DoFs in every stage, so its matrix is A_v = I_s ⊗ M̃ + Δt A ⊗ K̃
// (Section 4.2).  With a real block diagonalisation A = T D T⁻¹, D holding
// the real eigenvalues λ as 1×1 blocks and each complex pair α ± iβ (β > 0) as
// the 2×2 block [[α, β], [−β, α]],
//     A_v⁻¹ = (T ⊗ I) (I ⊗ M̃ + Δt D ⊗ K̃)⁻¹ (T⁻¹ ⊗ I),
// and the middle factor splits into one n×n system per real eigenvalue and
// one 2n×2n system per complex pair.  The 2n×2n block [[P, −Q], [Q, P]] with
// P = M̃ + Δt α K̃, Q = −Δt β K̃ is the real form of the complex matrix P + iQ,
// so its inverse is [[X, −Y], [Y, X]] with X + iY = (P + iQ)⁻¹ and only the
// n×n matrices X and Y are kept.
#include <cmath>
#include <complex>

#include "irkmg_internal.h"

namespace irkmg {

namespace {

using cplx = std::complex<double>;

// Characteristic polynomial λ^s + c[s-1] λ^{s-1} + ... + c[0] of A (s ≤ 3).
void charpoly(int s, const double* A, double* c) {
  if (s == 1) {
    c[0] = -A[0];
  } else if (s == 2) {
    c[1] = -(A[0] + A[3]);
    c[0] = A[0] * A[3] - A[1] * A[2];
  } else {
    const double tr = A[0] + A[4] + A[8];
    const double m2 = (A[0] * A[4] - A[1] * A[3]) + (A[0] * A[8] - A[2] * A[6]) +
                      (A[4] * A[8] - A[5] * A[7]);
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    c[2] = -tr;
    c[1] = m2;
    c[0] = -det;
  }
}

cplx peval(int s, const double* c, cplx z) {
  cplx p = 1.0;
  for (int k = s - 1; k >= 0; --k) p = p * z + c[k];
  return p;
}

cplx dpeval(int s, const double* c, cplx z) {
  cplx p = (double)s;
  for (int k = s - 1; k >= 1; --k) p = p * z + (double)k * c[k];
  return p;
}

// Roots of z² + b z + c.
void quadratic(double b, double c, cplx* r) {
  const double disc = 0.25 * b * b - c;
  if (disc >= 0.0) {
    const double q = -0.5 * b + (b <= 0.0 ? 1.0 : -1.0) * std::sqrt(disc);
    const double r1 = q, r2 = q != 0.0 ? c / q : 0.0;
    r[0] = r1;
    r[1] = r2;
  } else {
    r[0] = cplx(-0.5 * b, std::sqrt(-disc));
    r[1] = std::conj(r[0]);
  }
}

// Null vector of (A − λ I) for a simple eigenvalue λ (s ≤ 3).
void eigvec(int s, const double* A, cplx lam, cplx* v) {
  if (s == 1) {
    v[0] = 1.0;
    return;
  }
  cplx B[9];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) B[i * s + j] = A[i * s + j] - (i == j ? lam : cplx(0.0));
  if (s == 2) {
    // v ⟂ the larger row (in the bilinear sense: row · v = 0)
    const double n0 = std::abs(B[0]) + std::abs(B[1]), n1 = std::abs(B[2]) + std::abs(B[3]);
    const cplx* r = n0 >= n1 ? B : B + 2;
    v[0] = r[1];
    v[1] = -r[0];
    return;
  }
  // s = 3: cross product of the pair of rows with the largest result
  double best = -1.0;
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      const cplx* x = B + 3 * a;
      const cplx* y = B + 3 * b;
      const cplx w[3] = {x[1] * y[2] - x[2] * y[1], x[2] * y[0] - x[0] * y[2],
                         x[0] * y[1] - x[1] * y[0]};
      const double nw = std::abs(w[0]) + std::abs(w[1]) + std::abs(w[2]);
      if (nw > best) {
        best = nw;
        for (int k = 0; k < 3; ++k) v[k] = w[k];
      }
    }
}

bool invert_small(int s, const double* A, double* X) {
  double M[3][6];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < 2 * s; ++j) M[i][j] = j < s ? A[i * s + j] : (j - s == i ? 1.0 : 0.0);
  for (int k = 0; k < s; ++k) {
    int p = k;
    for (int i = k + 1; i < s; ++i)
      if (std::fabs(M[i][k]) > std::fabs(M[p][k])) p = i;
    if (M[p][k] == 0.0) return false;
    for (int j = 0; j < 2 * s; ++j) std::swap(M[k][j], M[p][j]);
    const double inv = 1.0 / M[k][k];
    for (int j = 0; j < 2 * s; ++j) M[k][j] *= inv;
    for (int i = 0; i < s; ++i)
      if (i != k) {
        const double f = M[i][k];
        for (int j = 0; j < 2 * s; ++j) M[i][j] -= f * M[k][j];
      }
  }
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) X[i * s + j] = M[i][s + j];
  return true;
}

}  // namespace

int kron_split(int s, const double* A, KronSplit* out) {
  if (s < 1 || s > 3) return IRKMG_EINVAL;
  double c[3];
  charpoly(s, A, c);
  cplx lam[3];
  if (s == 1) {
    lam[0] = A[0];
  } else if (s == 2) {
    quadratic(c[1], c[0], lam);
  } else {
    // one real root by bisection on a Cauchy bound bracket, then deflation
    double R = 1.0;
    for (int k = 0; k < 3; ++k) R = std::max(R, 1.0 + std::fabs(c[k]));
    double lo = -R, hi = R;
    auto p = [&](double x) { return ((x + c[2]) * x + c[1]) * x + c[0]; };
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      if ((p(mid) > 0.0) == (p(hi) > 0.0))
        hi = mid;
      else
        lo = mid;
    }
    const double r = 0.5 * (lo + hi);
    lam[0] = r;
    quadratic(c[2] + r, c[1] + r * (c[2] + r), lam + 1);
  }
  // polish every root by Newton on the full polynomial
  for (int k = 0; k < s; ++k)
    for (int it = 0; it < 3; ++it) {
      const cplx d = dpeval(s, c, lam[k]);
      if (std::abs(d) == 0.0) break;
      lam[k] -= peval(s, c, lam[k]) / d;
    }
  // distinct eigenvalues only (every RadauIIA, Gauss and LobattoIIIC tableau)
  double scale = 0.0;
  for (int k = 0; k < s * s; ++k) scale = std::max(scale, std::fabs(A[k]));
  for (int a = 0; a < s; ++a)
    for (int b = a + 1; b < s; ++b)
      if (std::abs(lam[a] - lam[b]) <= 1e-6 * std::max(scale, 1e-300)) return IRKMG_ENOTIMPL;
  // blocks: real eigenvalues first, then the pair (imaginary part > 0 kept)
  KronSplit K{};
  int col = 0;
  const double tiny = 1e-12 * std::max(scale, 1e-300);
  for (int k = 0; k < s; ++k) {
    if (std::fabs(lam[k].imag()) > tiny) continue;
    cplx v[3];
    eigvec(s, A, cplx(lam[k].real(), 0.0), v);
    double nrm = 0.0;
    for (int i = 0; i < s; ++i) nrm += v[i].real() * v[i].real();
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return IRKMG_ENOTIMPL;
    for (int i = 0; i < s; ++i) K.T[i * s + col] = v[i].real() / nrm;
    K.blk_size[K.nblk] = 1;
    K.blk[K.nblk][0] = lam[k].real();
    K.col0[K.nblk] = col;
    K.nblk++;
    col++;
  }
  for (int k = 0; k < s; ++k) {
    if (!(lam[k].imag() > tiny)) continue;
    cplx v[3];
    eigvec(s, A, lam[k], v);
    // rotate the phase so that Re v ⟂ Im v, then normalise
    double aa = 0.0, bb = 0.0, ab = 0.0;
    for (int i = 0; i < s; ++i) {
      aa += v[i].real() * v[i].real();
      bb += v[i].imag() * v[i].imag();
      ab += v[i].real() * v[i].imag();
    }
    const double phi = 0.5 * std::atan2(-2.0 * ab, aa - bb);
    const cplx rot = std::polar(1.0, phi);
    double nrm = 0.0;
    for (int i = 0; i < s; ++i) {
      v[i] *= rot;
      nrm += std::norm(v[i]);
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return IRKMG_ENOTIMPL;
    for (int i = 0; i < s; ++i) {
      K.T[i * s + col] = v[i].real() / nrm;
      K.T[i * s + col + 1] = v[i].imag() / nrm;
    }
    // A a = α a − β b, A b = β a + α b for v = a + ib, λ = α + iβ
    const double al = lam[k].real(), be = lam[k].imag();
    K.blk_size[K.nblk] = 2;
    K.blk[K.nblk][0] = al;
    K.blk[K.nblk][1] = be;
    K.blk[K.nblk][2] = -be;
    K.blk[K.nblk][3] = al;
    K.col0[K.nblk] = col;
    K.nblk++;
    col += 2;
  }
  if (col != s) return IRKMG_ENOTIMPL;
  if (!invert_small(s, K.T, K.Tinv)) return IRKMG_ENOTIMPL;
  // T D T⁻¹ must give back A
  double D[9] = {0};
  for (int b = 0; b < K.nblk; ++b) {
    const int c0 = K.col0[b], q = K.blk_size[b];
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) D[(c0 + i) * s + c0 + j] = K.blk[b][i * q + j];
  }
  double err = 0.0;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      double x = 0.0;
      for (int k = 0; k < s; ++k)
        for (int l = 0; l < s; ++l) x += K.T[i * s + k] * D[k * s + l] * K.Tinv[l * s + j];
      err = std::max(err, std::fabs(x - A[i * s + j]));
    }
  if (err > 1e-13 * std::max(scale, 1.0)) return IRKMG_ENOTIMPL;
  K.s = s;
  *out = K;
  return IRKMG_OK;
}

// The apply plan: stored n×n matrices, the source vectors (combinations of
// the rows of T⁻¹ applied to the gathered stage residuals), the mat-vec tasks
// (matrix, source) and the map from task results back to the stages.
//   layout 1 ("complex"): per pair X and Y; tasks X·w1, X·w2, Y·w1, Y·w2 and
//     y1 = X w1 − Y w2, y2 = Y w1 + X w2.  s·n² values, (s + 2·pairs)·n² FMAs.
//   layout 2 ("three-product"): per pair S = X + Y, X and Y; tasks S·w1,
//     X·(w2 − w1), Y·(w1 + w2) with k1, k2, k3 and y1 = k1 − k3, y2 = k1 + k2
//     (Gauss's three-multiplication complex product).  (s + pairs)·n² values
//     and FMAs.
int kron_plan(const KronSplit& K, int layout, KronPlan* out) {
  if (layout != 1 && layout != 2) return IRKMG_EINVAL;
  KronPlan P{};
  P.s = K.s;
  P.layout = layout;
  const int s = K.s;
  double C[3][kKronMaxTasks] = {};  // y_k = Σ_τ C[k][τ] acc_τ
  // layout 1 takes the complex pair first (matrices X, Y = 0, 1, sources
  // w1, w2 = 0, 1, tasks 0..3), then a real block (matrix, source 2, task 4):
  // the order the paired fixed-point apply is written for
  int border[3], nb = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int b = 0; b < K.nblk; ++b)
      if (layout == 2 ? pass == 0 : (pass == 0) == (K.blk_size[b] == 2)) border[nb++] = b;
  for (int bi = 0; bi < K.nblk; ++bi) {
    const int b = border[bi];
    const int c0 = K.col0[b];
    auto add_src = [&](double f0, int k0, double f1, int k1) {
      for (int t = 0; t < s; ++t)
        P.G[P.ns * 3 + t] = f0 * K.Tinv[k0 * s + t] + (k1 >= 0 ? f1 * K.Tinv[k1 * s + t] : 0.0);
      return P.ns++;
    };
    auto add_task = [&](int mat, int src) {
      P.task_mat[P.nt] = mat;
      P.task_src[P.nt] = src;
      return P.nt++;
    };
    if (K.blk_size[b] == 1) {
      P.blk_kind[P.nblk] = 0;
      P.blk_mat[P.nblk] = P.nm;
      const int m = P.nm++;
      const int w = add_src(1.0, c0, 0.0, -1);
      C[c0][add_task(m, w)] = 1.0;
    } else if (layout == 1) {
      P.blk_kind[P.nblk] = 1;
      P.blk_mat[P.nblk] = P.nm;
      const int mx = P.nm++, my = P.nm++;
      const int w1 = add_src(1.0, c0, 0.0, -1), w2 = add_src(1.0, c0 + 1, 0.0, -1);
      C[c0][add_task(mx, w1)] = 1.0;       // X w1
      C[c0 + 1][add_task(mx, w2)] = 1.0;   // X w2
      C[c0 + 1][add_task(my, w1)] = 1.0;   // Y w1
      C[c0][add_task(my, w2)] = -1.0;      // Y w2
    } else {
      P.blk_kind[P.nblk] = 2;
      P.blk_mat[P.nblk] = P.nm;
      const int ms = P.nm++, mx = P.nm++, my = P.nm++;
      const int w1 = add_src(1.0, c0, 0.0, -1);
      const int wd = add_src(1.0, c0 + 1, -1.0, c0);  // w2 − w1
      const int wsum = add_src(1.0, c0, 1.0, c0 + 1); // w1 + w2
      const int k1 = add_task(ms, w1), k2 = add_task(mx, wd), k3 = add_task(my, wsum);
      C[c0][k1] = 1.0;
      C[c0][k3] = -1.0;
      C[c0 + 1][k1] = 1.0;
      C[c0 + 1][k2] = 1.0;
    }
    P.blk_size[P.nblk] = K.blk_size[b];
    for (int k = 0; k < 4; ++k) P.blk[P.nblk][k] = K.blk[b][k];
    P.nblk++;
  }
  for (int t = 0; t < s; ++t)
    for (int tau = 0; tau < P.nt; ++tau) {
      double h = 0.0;
      for (int k = 0; k < s; ++k) h += K.T[t * s + k] * C[k][tau];
      P.H[t * kKronMaxTasks + tau] = h;
    }
  *out = P;
  return IRKMG_OK;
}

}  // namespace irkmg

// Eigenvalues of a small upper Hessenberg matrix: the Ritz values of an
// Arnoldi process on the Vanka-preconditioned stage operator, from which the
// Chebyshev interval [λ/4, λ] is chosen (Section 5.1: estimate the largest
// eigenvalue of the relaxation-preconditioned matrix from Ritz values).
//
// Method: the shifted QR algorithm in complex arithmetic (so complex pairs
// need no special case).  The active window [lo, hi] shrinks as subdiagonal
// entries become negligible; each step factors H − μI = QR with hi − lo
// Givens rotations and forms RQ + μI, with μ the eigenvalue of the trailing
// 2×2 block nearer to its last diagonal entry (Wilkinson's shift); every 10th
// step without deflation uses an exceptional shift to break cycles.
#include <cmath>
#include <complex>
#include <vector>

#include "irkmg_internal.h"

namespace irkmg {

int hessenberg_eigvals(int n, const double* H, double* wr, double* wi) {
  using cd = std::complex<double>;
  if (n < 1) return IRKMG_EINVAL;
  std::vector<cd> a((size_t)n * n);
  double scale = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      a[(size_t)i * n + j] = (j >= i - 1) ? cd(H[(size_t)i * n + j], 0.0) : cd(0.0, 0.0);
      scale = std::max(scale, std::fabs(H[(size_t)i * n + j]));
    }
  auto at = [&](int i, int j) -> cd& { return a[(size_t)i * n + j]; };
  const double eps = 1e-15;
  int hi = n - 1, its = 0, total = 0;
  while (hi >= 0) {
    if (hi == 0) {
      wr[0] = at(0, 0).real();
      wi[0] = at(0, 0).imag();
      break;
    }
    // deflate at the lowest negligible subdiagonal entry of the window
    int lo = hi;
    while (lo > 0) {
      const double s = std::abs(at(lo - 1, lo - 1)) + std::abs(at(lo, lo));
      if (std::abs(at(lo, lo - 1)) <= eps * (s > 0.0 ? s : scale)) {
        at(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // 1x1 block converged
      wr[hi] = at(hi, hi).real();
      wi[hi] = at(hi, hi).imag();
      --hi;
      its = 0;
      continue;
    }
    if (++total > 100 * n) return IRKMG_ENOCONV;
    ++its;
    // shift
    cd mu;
    if (its % 10 == 0) {
      mu = at(hi, hi) + std::abs(at(hi, hi - 1)) * 0.75;
    } else {
      const cd p = at(hi - 1, hi - 1), q = at(hi - 1, hi), r = at(hi, hi - 1), t = at(hi, hi);
      const cd half = 0.5 * (p - t);
      // eigenvalues of [[p, q], [r, t]]: (p + t)/2 ± sqrt(((p − t)/2)² + q r)
      const cd disc = std::sqrt(half * half + q * r);
      const cd e1 = 0.5 * (p + t) + disc, e2 = 0.5 * (p + t) - disc;
      mu = std::abs(e1 - t) < std::abs(e2 - t) ? e1 : e2;
    }
    // QR step on the window: H − μI = Q R by Givens rotations, then R Q + μI
    for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
    std::vector<cd> c(hi - lo), sn(hi - lo);
    for (int k = lo; k < hi; ++k) {
      const cd x = at(k, k), y = at(k + 1, k);
      const double rr = std::sqrt(std::norm(x) + std::norm(y));
      cd ck = 1.0, sk = 0.0;
      if (rr > 0.0) {
        ck = x / rr;
        sk = y / rr;
      }
      c[k - lo] = ck;
      sn[k - lo] = sk;
      // rows k, k+1 (columns k .. n-1) by G = [[conj(c), conj(s)], [-s, c]]
      for (int j = k; j < n; ++j) {
        const cd u = at(k, j), v = at(k + 1, j);
        at(k, j) = std::conj(ck) * u + std::conj(sk) * v;
        at(k + 1, j) = -sk * u + ck * v;
      }
    }
    for (int k = lo; k < hi; ++k) {
      const cd ck = c[k - lo], sk = sn[k - lo];
      // columns k, k+1 (rows 0 .. k+1) by Gᴴ
      for (int i = 0; i <= std::min(k + 1, hi); ++i) {
        const cd u = at(i, k), v = at(i, k + 1);
        at(i, k) = u * ck + v * sk;
        at(i, k + 1) = -u * std::conj(sk) + v * std::conj(ck);
      }
    }
    for (int i = lo; i <= hi; ++i) at(i, i) += mu;
  }
  return IRKMG_OK;
}

}  // namespace irkmg

// The fixed-point patch apply of one patch by one warp (the decoupled Vanka
// patch solves of Section 4.2 with exact integer dot products; see
// k_patch_fixed.cu for the number format), shared by the per-level apply
// kernels (k_patch_fixed.cu) and the batched persistent smoother (k_batch.cu).
#pragma once

#include <climits>
#include <cstdint>

#include "fx_math.h"
#include "irkmg_internal.h"

namespace irkmg {

constexpr int kFxWarps = 8;
constexpr int kFxMaxN = 63;    // rows of a block: no 64-bit accumulator overflows
constexpr int kFxPad = 16;     // zero limbs after each source: column batches need no mask
constexpr int kFxN2 = 39;      // interior 2D vertex star: 19 P2 nodes x 2 components + 1

struct __align__(8) Limbs {
  int32_t v1, v0;
};

struct FxApply {
  int s, nsrc, nt, nm;  // nsrc: source vectors built (ns, or nt for the transpose)
  int64_t m;
  double G[kKronMaxSrc * 3];
  double H[3 * kKronMaxTasks];
  int task_mat[kKronMaxTasks], task_src[kKronMaxTasks];
  const int32_t* np;
  const int64_t* fac_off;
  const int16_t* fexp;  // E of every stored row: [ordered patch][matrix][nmax]
  const double* r;
  double* out;
  double scale;
  int64_t first, count;
  int nmax;
  double* ybuf;  // one-launch mode (see KronApply)
  const int64_t* qoff;
  int64_t Q;
};

// Shared memory of one warp: limbs (nsrc·(nmax + kFxPad) × 8 B), residuals
// (s·nmax doubles), sources and then task results (max(nsrc, nt)·nmax
// doubles), exponents of the sources and of the matrices (2 · kKronMaxTasks
// int32), indices (nmax int32).
__host__ __device__ inline size_t fx_warp_bytes(int s, int nsrc, int nt, int nmax) {
  const int na = nsrc > nt ? nsrc : nt;
  size_t b = (size_t)nsrc * (nmax + kFxPad) * sizeof(Limbs) + (size_t)(s + na) * nmax * 8 +
             (size_t)2 * kKronMaxTasks * 4 + (size_t)nmax * 4;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ int64_t mad_wide(int32_t a, int32_t b, int64_t c) {
  int64_t d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// Bit pattern of the largest |x_i| over a warp's entries (i = lane, lane + 32,
// ... < n): non-negative doubles order like their bit patterns, so integer
// maxima suffice; a NaN or an infinity gives a pattern >= 0x7ff0000000000000.
__device__ __forceinline__ uint64_t warp_absmax_bits(const double* x, int n, int lane) {
  unsigned long long m = 0;
  for (int i = lane; i < n; i += 32)
    m = max(m, (unsigned long long)__double_as_longlong(x[i]) & 0x7fffffffffffffffull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One patch of the fixed-point apply.  N != 0: the patch size n is the
// compile-time N (divisions by constants, immediate load offsets, unrolled
// column batches); N == 0: n at run time.
// RL2: the residual is read through L2 only (ld.global.cg), for a residual
// written earlier by other CTAs of the same launch.
template <int N, int RC, int U, bool TR, bool RL2 = false>
__device__ __forceinline__ void fx_patch(const FxApply& P, const int2* __restrict__ fac,
                                         unsigned char* base, int lane, int64_t pi, int n_rt) {
  const int n = N ? N : n_rt;
  const int nmax = P.nmax;
  Limbs* s_lim = reinterpret_cast<Limbs*>(base);
  double* s_r = reinterpret_cast<double*>(s_lim + P.nsrc * (nmax + kFxPad));
  double* s_x = s_r + P.s * nmax;  // sources, then task results
  const int na = P.nsrc > P.nt ? P.nsrc : P.nt;
  int* s_F = reinterpret_cast<int*>(s_x + na * nmax);  // per source: F, or INT_MIN
  int* s_E = s_F + kKronMaxTasks;                       // transpose: max_j E_j per task
  int32_t* s_g = s_E + kKronMaxTasks;

  const int ls = n + kFxPad;  // limb stride of a source
  const int64_t nn = (int64_t)n * n;
  const int2* X = fac + P.fac_off[pi];
  const int32_t* gidx = reinterpret_cast<const int32_t*>(
      reinterpret_cast<const unsigned char*>(X) + (((int64_t)P.nm * nn * 8 + 15) & ~(int64_t)15));
  const int16_t* fe = P.fexp + pi * P.nm * nmax;
  for (int i = lane; i < n; i += 32) s_g[i] = gidx[i];
  if (TR)
    for (int c = 0; c < P.nsrc; ++c) {
      const int16_t* e = fe + P.task_mat[c] * nmax;
      int mx = INT_MIN;
      for (int i = lane; i < n; i += 32) mx = max(mx, (int)e[i]);
      mx = warp_max_int(mx);
      if (lane == 0) s_E[c] = mx;
    }
  __syncwarp();
  for (int idx = lane; idx < P.s * n; idx += 32) {
    const int t = idx / n, i = idx - t * n;
    s_r[idx] = RL2 ? __ldcg(P.r + t * P.m + s_g[i]) : P.r[t * P.m + s_g[i]];
  }
  __syncwarp();
  for (int idx = lane; idx < P.nsrc * n; idx += 32) {
    const int c = idx / n, i = idx - c * n;
    double a = 0.0;
    for (int t = 0; t < P.s; ++t)
      a += (TR ? P.H[t * kKronMaxTasks + c] : P.G[c * 3 + t]) * s_r[t * n + i];
    if (TR) a = ldexp(a, (int)fe[P.task_mat[c] * nmax + i] - s_E[c]);
    s_x[idx] = a;
  }
  __syncwarp();
  // each source to 58-bit integers with one exponent, split into two limbs
  for (int c = 0; c < P.nsrc; ++c) {
    const uint64_t mb = warp_absmax_bits(s_x + c * n, n, lane);
    const bool finite = mb < 0x7ff0000000000000ull;
    const int F = finite && mb != 0 ? fx_exponent(fx_from_bits(mb)) : 0;
    for (int i = lane; i < ls; i += 32) {
      const int64_t v = finite && i < n ? fx_scale_round(s_x[c * n + i], 58 - F) : 0;
      Limbs L;
      fx_split29(v, &L.v1, &L.v0);
      s_lim[c * ls + i] = L;
    }
    if (lane == 0) s_F[c] = finite ? F : INT_MIN;
  }
  __syncwarp();

  // (task, row) slots of this patch: lane + 32 k for k < RT, taken RC at a
  // time (four 64-bit accumulators per slot).  Columns go in batches of U,
  // the next batch's entries loaded before the current batch's products; the
  // last batch reads column n - 1 again past the end, against zero limbs.
  const int RT = (P.nt * n + 31) >> 5;
  const int nb = (n + U - 1) / U;
  const int64_t cstep = TR ? 1 : n;  // from one column to the next
  for (int k0 = 0; k0 < RT; k0 += RC) {
    const int2* mp[RC];
    const Limbs* lp[RC];
    int64_t acc[RC][4];
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int tau = lane + 32 * (k0 + k);
      const bool ok = k0 + k < RT && tau < P.nt * n;  // else: a valid address, result unused
      const int task = ok ? tau / n : 0;
      const int i = ok ? tau - task * n : 0;
      mp[k] = X + (int64_t)P.task_mat[task] * nn + (TR ? (int64_t)i * n : (int64_t)i);
      lp[k] = s_lim + (TR ? task : P.task_src[task]) * ls;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[k][q] = 0;
    }
    int2 qa[U][RC], qb[U][RC];
    // default-cached loads: rows 32..38 of a matrix are read by a later pass
    // of this warp, and an evict-first hint drops their lines from L2 first
    auto load = [&](int2 (&q)[U][RC], int b) {
      const int j0 = b * U;
      if (j0 + U <= n) {
#pragma unroll
        for (int k = 0; k < RC; ++k) {
          const int2* p = mp[k] + j0 * cstep;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            q[u][k] = __ldg(p);
            p += cstep;
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int k = 0; k < RC; ++k) q[u][k] = __ldg(mp[k] + min(j0 + u, n - 1) * cstep);
      }
    };
    auto mac = [&](const int2 (&q)[U][RC], int b) {
      const int j0 = b * U;
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < RC; ++k) {
          const Limbs L = lp[k][j0 + u];
          acc[k][0] = mad_wide(q[u][k].y, L.v1, acc[k][0]);
          acc[k][1] = mad_wide(q[u][k].y, L.v0, acc[k][1]);
          acc[k][2] = mad_wide(q[u][k].x, L.v1, acc[k][2]);
          acc[k][3] = mad_wide(q[u][k].x, L.v0, acc[k][3]);
        }
    };
    load(qa, 0);
    for (int b = 0; b < nb; b += 2) {
      if (b + 1 < nb) load(qb, b + 1);
      mac(qa, b);
      if (b + 1 < nb) {
        if (b + 2 < nb) load(qa, b + 2);
        mac(qb, b + 1);
      }
    }
    // s_x is free once the sources are in limbs: task results go there
#pragma unroll
    for (int k = 0; k < RC; ++k)
      if (k0 + k < RT && lane + 32 * (k0 + k) < P.nt * n) {
        const int tau = lane + 32 * (k0 + k);
        const int task = tau / n;
        const int i = tau - task * n;
        const int F = s_F[TR ? task : P.task_src[task]];
        const int ex = TR ? s_E[task] : (int)fe[P.task_mat[task] * nmax + i];
        s_x[tau] = F == INT_MIN ? __longlong_as_double(0x7ff8000000000000ll)
                                : fx_round(acc[k], ex + F - 115);
      }
  }
  __syncwarp();
  for (int idx = lane; idx < P.s * n; idx += 32) {
    const int t = idx / n, i = idx - t * n;
    double x = 0.0;
    for (int tau = 0; tau < P.nt; ++tau) {
      const double h = TR ? P.G[P.task_src[tau] * 3 + t] : P.H[t * kKronMaxTasks + tau];
      x += h * s_x[tau * n + i];
    }
    if (P.ybuf)
      P.ybuf[t * P.Q + P.qoff[pi] + i] = x;
    else
      P.out[t * P.m + s_g[i]] += P.scale * x;
  }
}

// The apply parameters of level L: colour >= 0, that colour's patches added
// into out (scaled); colour < 0, every patch into the context's result buffer
// (the one-launch relaxation).  k_patch_fixed.cu.
FxApply fx_params(Ctx& C, Level& L, int colour, const double* r, double* out, double scale,
                  int transpose);

}  // namespace irkmg

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
  int64_t ys;
  const int32_t* perm;
};

// Ordered patch index of the k-th patch a launch takes.
__device__ __forceinline__ int64_t fx_pi(const FxApply& P, int64_t k) {
  return P.perm ? (int64_t)P.perm[P.first + k] : P.first + k;
}

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

// c + a·b with the 32 × 32 → 64-bit product (a widening multiply-add).  Plain
// C++ rather than inline PTX: the compiler then updates the accumulators in
// place instead of moving them around each asm statement (measured: about
// one extra integer instruction per product with the asm form).  The callers'
// bounds keep every sum below 2^63.
__device__ __forceinline__ int64_t mad_wide(int32_t a, int32_t b, int64_t c) {
  return c + (int64_t)a * (int64_t)b;
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
      P.ybuf[t * P.Q + P.qoff[pi] + i * P.ys] = x;
    else
      P.out[t * P.m + s_g[i]] += P.scale * x;
  }
}


// ---------------------------------------------------------------------------
// Paired apply of one interior patch (n = kFxN2) in the complex layout, whose
// plan (host_kron.cpp) puts the complex pair first: matrices X = 0, Y = 1
// (tasks 0, 1 = X·w1, X·w2 and 2, 3 = Y·w1, Y·w2, sources w1 = 0, w2 = 1),
// then, for s = 3, the real block (matrix 2, task 4 = M2·w0, source 2).  A
// lane owns one row of X or Y and both of that matrix's tasks, so each loaded
// entry meets the limbs of w1 and w2 (one 16-byte shared-memory read) and
// feeds eight products; the rows of the real block run in the same passes
// against (w0, 0).  Rows of X and Y first, then those of the real block: with
// one, passes 0..2 hold 96 of the 117 rows (14 of pass 2's lanes on Y) and
// pass 3 the last 21 on the single-source path.  Per task and row the exact
// sum and its one rounding are those of fx_patch, so the results are
// bitwise the same.
// ---------------------------------------------------------------------------
constexpr int kFxPairLS = kFxN2 + kFxPad;  // limb entries per source (zero tail)

struct __align__(16) FxPairSmem {
  int4 pa[kFxPairLS];  // (v1, v0) of w1, then of w2
  int4 pb[kFxPairLS];  // (v1, v0) of w0, then zeros
  double r[3 * kFxN2];
  double x[kKronMaxTasks * kFxN2];  // sources, then task results
  int g[kFxN2 + 1];
  int F[kKronMaxSrc];
};

// The largest |x_i| over a source's entries as its exponent F (|x_i| < 2^F)
// and whether every entry is finite: the top words' maximum by one warp
// reduction when it is a normal number, else the 64-bit maximum.
__device__ __forceinline__ void fx_source_exponent(const double* x, int n, int lane, bool* finite,
                                                   int* F) {
  uint32_t hw = 0;
  for (int i = lane; i < n; i += 32)
    hw = max(hw, (uint32_t)((uint64_t)__double_as_longlong(x[i]) >> 32) & 0x7fffffffu);
  const uint32_t m = __reduce_max_sync(0xffffffffu, hw);
  if (m >= 0x00100000u) {  // exponent field of the maximum nonzero: the field alone gives F
    *finite = m < 0x7ff00000u;
    *F = (int)(m >> 20) - 1022;
  } else {
    const uint64_t mb = warp_absmax_bits(x, n, lane);
    *finite = true;
    *F = mb != 0 ? fx_exponent(fx_from_bits(mb)) : 0;
  }
}

// RL2: the residual is read through L2 only (written earlier in the launch).
template <int U, bool REAL, bool RL2 = false>
__device__ __forceinline__ void fx_patch_pair(const FxApply& P, const int2* __restrict__ fac,
                                              unsigned char* base, int lane, int64_t pi) {
  constexpr int N = kFxN2, NN = N * N, LS = kFxPairLS;
  constexpr int nb = (N + U - 1) / U;
  // stages, sources and tasks follow from the pair structure
  constexpr int S = REAL ? 3 : 2, NSRC = S, NT = REAL ? 5 : 4;
  FxPairSmem& sm = *reinterpret_cast<FxPairSmem*>(base);
  const int2* X = fac + P.fac_off[pi];
  // pass 0's first column batch (rows 0..31 of X) before the gathers
  int2 qa[U];
  {
    const int2* mp0 = X + lane;  // matrix X = 0
#pragma unroll
    for (int u = 0; u < U; ++u) qa[u] = __ldg(mp0 + u * N);
  }
  const int32_t* gidx = reinterpret_cast<const int32_t*>(
      reinterpret_cast<const unsigned char*>(X) + (((int64_t)P.nm * NN * 8 + 15) & ~(int64_t)15));
  for (int i = lane; i < N; i += 32) sm.g[i] = gidx[i];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (S * N + 31) / 32; ++k) {
    const int idx = lane + 32 * k;
    if (idx < S * N) {
      const int t = idx / N, i = idx - t * N;
      sm.r[idx] = RL2 ? __ldcg(P.r + t * P.m + sm.g[i]) : P.r[t * P.m + sm.g[i]];
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (NSRC * N + 31) / 32; ++k) {
    const int idx = lane + 32 * k;
    if (idx < NSRC * N) {
      const int c = idx / N, i = idx - c * N;
      double a = 0.0;
#pragma unroll
      for (int t = 0; t < S; ++t) a += P.G[c * 3 + t] * sm.r[t * N + i];
      sm.x[idx] = a;
    }
  }
  __syncwarp();
#pragma unroll
  for (int c = 0; c < NSRC; ++c) {
    bool finite;
    int F;
    fx_source_exponent(sm.x + c * N, N, lane, &finite, &F);
    int32_t* dst = c == 0 ? &sm.pa[0].x : c == 1 ? &sm.pa[0].z : &sm.pb[0].x;
#pragma unroll
    for (int k = 0; k < (LS + 31) / 32; ++k) {
      const int i = lane + 32 * k;
      if (i < LS) {
        const int64_t v = finite && i < N ? fx_scale_round(sm.x[c * N + i], 58 - F) : 0;
        int32_t v1, v0;
        fx_split29(v, &v1, &v0);
        dst[4 * i] = v1;
        dst[4 * i + 1] = v0;
        if (REAL && c == 2) {
          sm.pb[i].z = 0;
          sm.pb[i].w = 0;
        }
      }
    }
    if (lane == 0) sm.F[c] = finite ? F : INT_MIN;
  }
  __syncwarp();
  const int16_t* fe = P.fexp + pi * P.nm * P.nmax;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  // passes 0..2: rows of X (slots 0..38), Y (39..77), m0 (78..116, with a real block)
#pragma unroll 1
  for (int k0 = 0; k0 < 3; ++k0) {
    const int sl = 32 * k0 + lane;
    const int kind = sl < N ? 0 : sl < 2 * N ? 1 : 2;  // X, Y, real block (or idle)
    const bool ok = kind < 2 || (REAL && sl < 3 * N);
    const int row = ok ? sl - kind * N : 0;
    const int mat = ok ? kind : 0;  // matrix index = kind
    const int2* mp = X + (int64_t)mat * NN + row;
    const int4* lp = REAL && kind == 2 ? sm.pb : sm.pa;  // idle lanes: bounded limbs
    int64_t A[4] = {0, 0, 0, 0}, B[4] = {0, 0, 0, 0};
    int2 qb[U];
    if (k0 > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) qa[u] = __ldg(mp + u * N);
    }
    auto mac2 = [&](const int2 (&q)[U], int b) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int4 L = lp[b * U + u];
        A[0] = mad_wide(q[u].y, L.x, A[0]);
        A[1] = mad_wide(q[u].y, L.y, A[1]);
        A[2] = mad_wide(q[u].x, L.x, A[2]);
        A[3] = mad_wide(q[u].x, L.y, A[3]);
        B[0] = mad_wide(q[u].y, L.z, B[0]);
        B[1] = mad_wide(q[u].y, L.w, B[1]);
        B[2] = mad_wide(q[u].x, L.z, B[2]);
        B[3] = mad_wide(q[u].x, L.w, B[3]);
      }
    };
#pragma unroll
    for (int b = 0; b < nb; b += 2) {
      if (b + 1 < nb) {
#pragma unroll
        for (int u = 0; u < U; ++u) qb[u] = __ldg(mp + min((b + 1) * U + u, N - 1) * N);
      }
      mac2(qa, b);
      if (b + 1 < nb) {
        if (b + 2 < nb) {
#pragma unroll
          for (int u = 0; u < U; ++u) qa[u] = __ldg(mp + min((b + 2) * U + u, N - 1) * N);
        }
        mac2(qb, b + 1);
      }
    }
    if (ok) {
      const int ex = fe[mat * P.nmax + row];
      const int FA = sm.F[kind == 2 ? 2 : 0];  // w0 or w1
      sm.x[2 * kind * N + row] = FA == INT_MIN ? qnan : fx_round(A, ex + FA - 115);  // task 2·kind
      if (kind < 2) {
        const int FB = sm.F[1];  // w2
        sm.x[(2 * kind + 1) * N + row] = FB == INT_MIN ? qnan : fx_round(B, ex + FB - 115);
      }
    }
  }
  if (REAL) {  // pass 3: rows 18..38 of m0 against w0 alone
    const int row = 96 + lane - 2 * N;
    const bool ok = row < N;
    const int2* mp = X + 2 * NN + (ok ? row : 0);
    int64_t A[4] = {0, 0, 0, 0};
    int2 qb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) qa[u] = __ldg(mp + u * N);
    auto mac1 = [&](const int2 (&q)[U], int b) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int4 L = sm.pb[b * U + u];
        A[0] = mad_wide(q[u].y, L.x, A[0]);
        A[1] = mad_wide(q[u].y, L.y, A[1]);
        A[2] = mad_wide(q[u].x, L.x, A[2]);
        A[3] = mad_wide(q[u].x, L.y, A[3]);
      }
    };
#pragma unroll
    for (int b = 0; b < nb; b += 2) {
      if (b + 1 < nb) {
#pragma unroll
        for (int u = 0; u < U; ++u) qb[u] = __ldg(mp + min((b + 1) * U + u, N - 1) * N);
      }
      mac1(qa, b);
      if (b + 1 < nb) {
        if (b + 2 < nb) {
#pragma unroll
          for (int u = 0; u < U; ++u) qa[u] = __ldg(mp + min((b + 2) * U + u, N - 1) * N);
        }
        mac1(qb, b + 1);
      }
    }
    if (ok) {
      const int ex = fe[2 * P.nmax + row];
      const int F0 = sm.F[2];
      sm.x[4 * N + row] = F0 == INT_MIN ? qnan : fx_round(A, ex + F0 - 115);
    }
  }
  __syncwarp();
  const int64_t qo = P.ybuf ? P.qoff[pi] : 0;
#pragma unroll
  for (int k = 0; k < (S * N + 31) / 32; ++k) {
    const int idx = lane + 32 * k;
    if (idx < S * N) {
      const int t = idx / N, i = idx - t * N;
      double x = 0.0;
#pragma unroll
      for (int tau = 0; tau < NT; ++tau) x += P.H[t * kKronMaxTasks + tau] * sm.x[tau * N + i];
      if (P.ybuf)
        P.ybuf[t * P.Q + qo + i * P.ys] = x;
      else
        P.out[t * P.m + sm.g[i]] += P.scale * x;
    }
  }
}

// The apply parameters of level L: colour >= 0, that colour's patches added
// into out (scaled); colour < 0, every patch into the context's result buffer
// (the one-launch relaxation).  k_patch_fixed.cu.
FxApply fx_params(Ctx& C, Level& L, int colour, const double* r, double* out, double scale,
                  int transpose);


}  // namespace irkmg

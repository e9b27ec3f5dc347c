// Kronecker-decoupled Vanka patch solve (the Kronecker form of the stage
// system, Section 3, applied to the vertex-star patches of Section 4.2).
//
// With A = T D T⁻¹ (real block diagonal D) the patch inverse is
//     A_v⁻¹ = (T ⊗ I) (I ⊗ M̃ + Δt D ⊗ K̃)⁻¹ (T⁻¹ ⊗ I),
// so one colour launch does, for each of its patches (warp per patch):
//   1. gather the s stage residuals r_t (n spatial DoFs each) through the
//      patch's spatial index list (stage t adds t·m);
//   2. form the source vectors src_c = Σ_t G[c][t] r_t   (rows of T⁻¹ and, for
//      the three-product layout, their sums and differences);
//   3. nt dense n×n mat-vecs acc_τ = M_{mat τ} src_{src τ}, one (task, row)
//      pair per lane and slot, coalesced column-major loads streamed once;
//   4. x_t = Σ_τ H[t][τ] acc_τ (T and the complex recombination folded into H)
//      and out[S_v] += scale · x.
// Patches of one colour share no DoF, so the scatter needs no atomics.
// transpose = 1 applies (A_v⁻¹)ᵀ: the sources come from Hᵀ, each task reads
// its matrix transposed, and the stage results from Gᵀ.
#include <algorithm>

#include "irkmg_internal.h"
#include "tma.cuh"

namespace irkmg {

constexpr int kKronWarps = 8;
constexpr int kKronMaxSlots = 12;  // (task, row) pairs per lane: nt · n ≤ 384

struct KronApply {
  int s, ns, nt, nm;
  int64_t m;
  double G[kKronMaxSrc * 3];
  double H[3 * kKronMaxTasks];
  int task_mat[kKronMaxTasks], task_src[kKronMaxTasks];
  const int32_t* np;       // spatial n of each ordered patch
  const int64_t* fac_off;  // element offset of each ordered patch's block
  const double* r;
  double* out;
  double scale;
  int64_t first, count;  // ordered-patch range of this colour (or of all patches)
  int nmax;              // per-warp shared-memory stride
  // one-launch mode: the patch results go to ybuf[t·Q + qoff[p] + i·ys]
  // instead of out, and k_vanka_reduce adds them up per DoF afterwards; the
  // launch takes the ordered patches perm[0], perm[1], ... (vertex order)
  double* ybuf;
  const int64_t* qoff;
  int64_t Q;
  int64_t ys;
  const int32_t* perm;
  // tasks reading each stored matrix (at most two: the complex layout applies
  // X and Y to both sources of a pair), -1 if unused
  int mat_task[kKronMaxTasks][2];
  // G and H rounded to FP32, for the FP32-accumulating paired apply
  float Gf[kKronMaxSrc * 3], Hf[3 * kKronMaxTasks];
};

// Ordered patch index of the k-th patch a launch takes.
__device__ __forceinline__ int64_t kron_pi(const KronApply& P, int64_t k) {
  return P.perm ? (int64_t)P.perm[P.first + k] : P.first + k;
}

// The stage mixing around the patch solves (sources from the gathered
// residual by the rows of T⁻¹, results back by T) runs in the patch
// precision: FP64 for FP64 patches, FP32 for FP32 patches (the FP32 form
// accumulates in FP32 throughout the patch apply, and GB300's FP64 pipe is
// 1/62 of its FP32 rate).
template <typename T>
__device__ __forceinline__ T mix_g(const KronApply& P, int k) {
  if constexpr (sizeof(T) == 4) return P.Gf[k]; else return P.G[k];
}
template <typename T>
__device__ __forceinline__ T mix_h(const KronApply& P, int k) {
  if constexpr (sizeof(T) == 4) return P.Hf[k]; else return P.H[k];
}

// Shared memory of one warp: residuals (s·nmax doubles), task results
// (nt·nmax doubles), sources (max(ns, nt)·nmax of T), indices (nmax int32);
// FP32 patches keep the residuals and results as floats in the same slots.
__host__ __device__ inline size_t kron_warp_bytes(int s, int ns, int nt, int nmax, int tsize) {
  const int nsrc = ns > nt ? ns : nt;
  size_t b = (size_t)(s + nt) * nmax * 8 + (size_t)nsrc * nmax * tsize + (size_t)nmax * 4;
  return (b + 15) & ~(size_t)15;
}

// One patch by one warp (lanes over (task, row) slots, R slots per lane).
template <typename T, int R, bool TR>
__device__ __forceinline__ void kron_patch(const KronApply& P, const T* __restrict__ fac,
                                           unsigned char* base, int lane, int64_t pi) {
  const int nmax = P.nmax;
  double* s_r = reinterpret_cast<double*>(base);
  double* s_acc = s_r + P.s * nmax;
  T* s_src = reinterpret_cast<T*>(s_acc + P.nt * nmax);
  const int nsrc = TR ? P.nt : P.ns;
  int32_t* s_g = reinterpret_cast<int32_t*>(s_src + (P.ns > P.nt ? P.ns : P.nt) * nmax);

  const int n = P.np[pi];
  const int64_t nn = (int64_t)n * n;
  const T* X = fac + P.fac_off[pi];
  const int32_t* gidx = reinterpret_cast<const int32_t*>(
      reinterpret_cast<const unsigned char*>(X) +
      (((int64_t)P.nm * nn * (int64_t)sizeof(T) + 15) & ~(int64_t)15));
  T* s_rm = reinterpret_cast<T*>(s_r);
  T* s_accm = reinterpret_cast<T*>(s_acc);
  for (int i = lane; i < n; i += 32) s_g[i] = gidx[i];
  __syncwarp();
  for (int idx = lane; idx < P.s * n; idx += 32) {
    const int t = idx / n, i = idx - t * n;
    s_rm[idx] = (T)P.r[t * P.m + s_g[i]];
  }
  __syncwarp();
  for (int idx = lane; idx < nsrc * n; idx += 32) {
    const int c = idx / n, i = idx - c * n;
    T a = (T)0;
    for (int t = 0; t < P.s; ++t)
      a = fma(TR ? mix_h<T>(P, t * kKronMaxTasks + c) : mix_g<T>(P, c * 3 + t), s_rm[t * n + i], a);
    s_src[idx] = a;
  }
  __syncwarp();

  // (task, row) of every slot; column-major M[j n + i] (transposed: M[i n + j])
  const T* mp[R];
  const T* sp[R];
  T acc[R];
  bool ok[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int tau = lane + 32 * k;
    ok[k] = tau < P.nt * n;
    const int task = ok[k] ? tau / n : 0;
    const int i = ok[k] ? tau - task * n : 0;
    mp[k] = X + (int64_t)P.task_mat[task] * nn + (TR ? (int64_t)i * n : (int64_t)i);
    sp[k] = s_src + (TR ? task : P.task_src[task]) * n;
    acc[k] = (T)0;
  }
  const int64_t step = TR ? 1 : n;
#pragma unroll 2
  for (int j = 0; j < n; ++j) {
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (ok[k]) {
        const T m = TR ? mp[k][j] : __ldcs(mp[k]);
        acc[k] = fma(m, sp[k][j], acc[k]);
        if (!TR) mp[k] += step;
      }
  }
#pragma unroll
  for (int k = 0; k < R; ++k)
    if (ok[k]) s_accm[lane + 32 * k] = acc[k];
  __syncwarp();
  for (int idx = lane; idx < P.s * n; idx += 32) {
    const int t = idx / n, i = idx - t * n;
    T x = (T)0;
    for (int tau = 0; tau < P.nt; ++tau) {
      const T h = TR ? mix_g<T>(P, P.task_src[tau] * 3 + t) : mix_h<T>(P, t * kKronMaxTasks + tau);
      x = fma(h, s_accm[tau * n + i], x);
    }
    if (P.ybuf)
      P.ybuf[t * P.Q + P.qoff[pi] + i * P.ys] = (double)x;
    else
      P.out[t * P.m + s_g[i]] += P.scale * (double)x;
  }
}

template <typename T, int R, bool TR>
__global__ void __launch_bounds__(kKronWarps * 32) k_vanka_apply_kron(KronApply P,
                                                                      const T* __restrict__ fac) {
  extern __shared__ __align__(128) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kKronWarps + warp;
  if (w >= P.count) return;
  unsigned char* base = dyn + (size_t)warp * kron_warp_bytes(P.s, P.ns, P.nt, P.nmax, sizeof(T));
  kron_patch<T, R, TR>(P, fac, base, lane, kron_pi(P, w));
}

// ---------------------------------------------------------------------------
// Paired FP32 rows for the complex layout (pair first: X = 0, Y = 1 with
// tasks 0..3 on sources w1, w2 = 0, 1; the real block 2 with task 4 on
// source 2, for s = 3).  Interior patches (n = kFxN2 = 39): a lane owns a
// row of X or Y and both of its tasks, so every entry is loaded once and
// meets (w1[j], w2[j]) in one 8-byte shared-memory read; rows of the real
// block take (w0[j], 0).  Every (task, row) sum runs over the columns in the
// same order as kron_patch, so the results are bitwise those of kernel 4.
// Other patches go through kron_patch.
// ---------------------------------------------------------------------------
constexpr int kPairN = 39;
constexpr int kPair32U = 8;  // columns per load batch (two batches in flight)

struct __align__(16) KronPairSmem {
  float r[3 * kPairN];
  float acc[kKronMaxTasks * kPairN];
  float2 pa[kPairN];  // (w1, w2)
  float2 pb[kPairN];  // (w0, 0)
  int g[kPairN + 1];
};

__device__ __noinline__ void kron_patch_f32_generic(const KronApply& P, const float* __restrict__ fac,
                                                    unsigned char* base, int lane, int64_t pi) {
  // nt·n ≤ 5·39 slots: seven per lane (kKronMaxSlots would raise the whole
  // kernel's register count, and so cut its resident warps, for the few
  // boundary patches that come here)
  kron_patch<float, (kKronMaxTasks * kPairN + 31) / 32, false>(P, fac, base, lane, pi);
}

template <bool REAL>
__global__ void __launch_bounds__(kKronWarps * 32, 4) k_vanka_apply_kron_pair32(
    KronApply P, const float* __restrict__ fac, uint32_t warp_bytes) {
  constexpr int N = kPairN, NN = N * N, U = kPair32U, nb = (N + U - 1) / U;
  constexpr int S = REAL ? 3 : 2, NSRC = S, NT = REAL ? 5 : 4;
  extern __shared__ __align__(128) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kKronWarps + warp;
  if (w >= P.count) return;
  unsigned char* base = dyn + (size_t)warp * warp_bytes;
  const int64_t pi = kron_pi(P, w);
  if (P.np[pi] != N) {
    kron_patch_f32_generic(P, fac, base, lane, pi);
    return;
  }
  KronPairSmem& sm = *reinterpret_cast<KronPairSmem*>(base);
  const float* X = fac + P.fac_off[pi];
  float qa[U];
#pragma unroll
  for (int u = 0; u < U; ++u) qa[u] = __ldg(X + lane + u * N);  // pass 0: rows 0..31 of X
  const int32_t* gidx = reinterpret_cast<const int32_t*>(
      reinterpret_cast<const unsigned char*>(X) + (((int64_t)P.nm * NN * 4 + 15) & ~(int64_t)15));
  for (int i = lane; i < N; i += 32) sm.g[i] = gidx[i];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (S * N + 31) / 32; ++k) {
    const int idx = lane + 32 * k;
    if (idx < S * N) {
      const int t = idx / N, i = idx - t * N;
      sm.r[idx] = (float)P.r[t * P.m + sm.g[i]];
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (NSRC * N + 31) / 32; ++k) {
    const int idx = lane + 32 * k;
    if (idx < NSRC * N) {
      const int c = idx / N, i = idx - c * N;
      float f = 0.f;
#pragma unroll
      for (int t = 0; t < S; ++t) f = fmaf(P.Gf[c * 3 + t], sm.r[t * N + i], f);
      if (c == 0)
        sm.pa[i].x = f;
      else if (c == 1)
        sm.pa[i].y = f;
      else {
        sm.pb[i].x = f;
        sm.pb[i].y = 0.f;
      }
    }
  }
  __syncwarp();
#pragma unroll 1
  for (int k0 = 0; k0 < 3; ++k0) {  // rows of X, Y, then the real block (or idle)
    const int sl = 32 * k0 + lane;
    const int kind = sl < N ? 0 : sl < 2 * N ? 1 : 2;
    const bool ok = kind < 2 || (REAL && sl < 3 * N);
    const int row = ok ? sl - kind * N : 0;
    const int mat = ok ? kind : 0;
    const float* mp = X + mat * NN + row;
    const float2* lp = REAL && kind == 2 ? sm.pb : sm.pa;
    float A = 0.f, B = 0.f;
    float qb[U];
    if (k0 > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) qa[u] = __ldg(mp + u * N);
    }
#pragma unroll
    for (int b = 0; b < nb; b += 2) {
      if (b + 1 < nb) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if ((b + 1) * U + u < N) qb[u] = __ldg(mp + ((b + 1) * U + u) * N);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (b * U + u < N) {
          const float2 L = lp[b * U + u];
          A = fmaf(qa[u], L.x, A);
          B = fmaf(qa[u], L.y, B);
        }
      if (b + 1 < nb) {
        if (b + 2 < nb) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if ((b + 2) * U + u < N) qa[u] = __ldg(mp + ((b + 2) * U + u) * N);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if ((b + 1) * U + u < N) {
            const float2 L = lp[(b + 1) * U + u];
            A = fmaf(qb[u], L.x, A);
            B = fmaf(qb[u], L.y, B);
          }
      }
    }
    if (ok) {
      sm.acc[2 * kind * N + row] = A;  // task 0, 2 or 4
      if (kind < 2) sm.acc[(2 * kind + 1) * N + row] = B;
    }
  }
  if (REAL) {  // rows 18..38 of the real block against w0 alone
    const int row = 96 + lane - 2 * N;
    const bool ok = row < N;
    const float* mp = X + 2 * NN + (ok ? row : 0);
    float A = 0.f;
    float qb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) qa[u] = __ldg(mp + u * N);
#pragma unroll
    for (int b = 0; b < nb; b += 2) {
      if (b + 1 < nb) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if ((b + 1) * U + u < N) qb[u] = __ldg(mp + ((b + 1) * U + u) * N);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (b * U + u < N) A = fmaf(qa[u], sm.pb[b * U + u].x, A);
      if (b + 1 < nb) {
        if (b + 2 < nb) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if ((b + 2) * U + u < N) qa[u] = __ldg(mp + ((b + 2) * U + u) * N);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if ((b + 1) * U + u < N) A = fmaf(qb[u], sm.pb[(b + 1) * U + u].x, A);
      }
    }
    if (ok) sm.acc[4 * N + row] = A;
  }
  __syncwarp();
  const int64_t qo = P.ybuf ? P.qoff[pi] : 0;
#pragma unroll
  for (int k = 0; k < (S * N + 31) / 32; ++k) {
    const int idx = lane + 32 * k;
    if (idx < S * N) {
      const int t = idx / N, i = idx - t * N;
      float x = 0.f;
#pragma unroll
      for (int tau = 0; tau < NT; ++tau) x = fmaf(P.Hf[t * kKronMaxTasks + tau], sm.acc[tau * N + i], x);
      if (P.ybuf)
        P.ybuf[t * P.Q + qo + i * P.ys] = (double)x;
      else
        P.out[t * P.m + sm.g[i]] += P.scale * (double)x;
    }
  }
}

int kron_max_slots() { return kKronMaxSlots; }

// ---------------------------------------------------------------------------
// Decoupled apply for large patches (3D: n up to kKronBigMaxN per stage): one
// CTA per patch.  The gathered residual, the sources and the task results
// live in shared memory; thread t owns tasks (matrix, row) t, t + 256, ...,
// streaming each row's entries with coalesced loads (consecutive threads take
// consecutive rows of one column-major matrix), eight columns loaded before
// their multiply-adds.
// ---------------------------------------------------------------------------
constexpr int kKronBigThreads = 256;
constexpr int kKronBigMaxN = 256;

int kron_big_max_n() { return kKronBigMaxN; }

template <typename T>
__global__ void __launch_bounds__(kKronBigThreads)
    k_vanka_apply_kron_big(KronApply P, const T* __restrict__ fac) {
  __shared__ double s_r[3 * kKronBigMaxN];
  __shared__ T s_src[kKronMaxSrc * kKronBigMaxN];
  __shared__ double s_acc[kKronMaxTasks * kKronBigMaxN];
  __shared__ int32_t s_g[kKronBigMaxN];
  const int64_t w = blockIdx.x;
  if (w >= P.count) return;
  const int tid = threadIdx.x;
  const int64_t pi = kron_pi(P, w);
  const int n = P.np[pi];
  const int64_t nn = (int64_t)n * n;
  const T* X = fac + P.fac_off[pi];
  const int32_t* gidx = reinterpret_cast<const int32_t*>(
      reinterpret_cast<const unsigned char*>(X) +
      (((int64_t)P.nm * nn * (int64_t)sizeof(T) + 15) & ~(int64_t)15));
  T* s_rm = reinterpret_cast<T*>(s_r);
  T* s_accm = reinterpret_cast<T*>(s_acc);
  for (int i = tid; i < n; i += kKronBigThreads) s_g[i] = gidx[i];
  __syncthreads();
  for (int idx = tid; idx < P.s * n; idx += kKronBigThreads) {
    const int t = idx / n, i = idx - t * n;
    s_rm[idx] = (T)P.r[t * P.m + s_g[i]];
  }
  __syncthreads();
  for (int idx = tid; idx < P.ns * n; idx += kKronBigThreads) {
    const int c = idx / n, i = idx - c * n;
    T a = (T)0;
    for (int t = 0; t < P.s; ++t) a = fma(mix_g<T>(P, c * 3 + t), s_rm[t * n + i], a);
    s_src[idx] = a;
  }
  __syncthreads();
  // units (matrix b, row i): every stored entry is loaded once and feeds the
  // one or two tasks that read its matrix; thread t takes units t and t + 256
  // together, a batch of columns of each (16 FP32 or 8 FP64 entries) loaded
  // before their multiply-adds
  constexpr int kBatch = sizeof(T) == 4 ? 16 : 8;
  const int nunit = P.nm * n;
  for (int u0 = tid; u0 < nunit; u0 += 2 * kKronBigThreads) {
    const int u1 = u0 + kKronBigThreads;
    const bool has1 = u1 < nunit;
    const int b0 = u0 / n, i0 = u0 - b0 * n;
    const int b1 = has1 ? u1 / n : b0, i1 = has1 ? u1 - b1 * n : i0;
    const T* M0 = X + (int64_t)b0 * nn + i0;
    const T* M1 = X + (int64_t)b1 * nn + i1;
    const int t00 = P.mat_task[b0][0], t01 = P.mat_task[b0][1];
    const int t10 = P.mat_task[b1][0], t11 = P.mat_task[b1][1];
    const T* s00 = s_src + P.task_src[t00] * n;
    const T* s01 = s_src + P.task_src[t01 >= 0 ? t01 : t00] * n;
    const T* s10 = s_src + P.task_src[t10] * n;
    const T* s11 = s_src + P.task_src[t11 >= 0 ? t11 : t10] * n;
    T a00 = (T)0, a01 = (T)0, a10 = (T)0, a11 = (T)0;
    int j = 0;
    for (; j + kBatch <= n; j += kBatch) {
      T v0[kBatch], v1[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        v0[u] = __ldcs(M0 + (int64_t)(j + u) * n);
        if (has1) v1[u] = __ldcs(M1 + (int64_t)(j + u) * n);
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        a00 = fma(v0[u], s00[j + u], a00);
        a01 = fma(v0[u], s01[j + u], a01);
        if (has1) {
          a10 = fma(v1[u], s10[j + u], a10);
          a11 = fma(v1[u], s11[j + u], a11);
        }
      }
    }
    for (; j < n; ++j) {
      const T w0 = __ldcs(M0 + (int64_t)j * n);
      a00 = fma(w0, s00[j], a00);
      a01 = fma(w0, s01[j], a01);
      if (has1) {
        const T w1 = __ldcs(M1 + (int64_t)j * n);
        a10 = fma(w1, s10[j], a10);
        a11 = fma(w1, s11[j], a11);
      }
    }
    s_accm[t00 * n + i0] = a00;
    if (t01 >= 0) s_accm[t01 * n + i0] = a01;
    if (has1) {
      s_accm[t10 * n + i1] = a10;
      if (t11 >= 0) s_accm[t11 * n + i1] = a11;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < P.s * n; idx += kKronBigThreads) {
    const int t = idx / n, i = idx - t * n;
    T x = (T)0;
    for (int tau = 0; tau < P.nt; ++tau) x = fma(mix_h<T>(P, t * kKronMaxTasks + tau), s_accm[tau * n + i], x);
    if (P.ybuf)
      P.ybuf[t * P.Q + P.qoff[pi] + i * P.ys] = (double)x;
    else
      P.out[t * P.m + s_g[i]] += P.scale * (double)x;
  }
}

// ---------------------------------------------------------------------------
// TMA-staged decoupled apply (persistent over the patches of one colour).
// Each patch block (nm matrices + index list) is one contiguous 16-byte-aligned
// run, streamed into a ring of shared-memory stages by cp.async.bulk; the CTA
// works on one patch at a time from shared memory while the next blocks are
// in flight, so the latency of a patch is one pass over its block instead of
// one memory round trip per column.  The target values out[S_v] are read
// together with the residual (patches of one colour are disjoint, so no other
// CTA writes them during the launch).  Every mbarrier wait is bounded: on
// expiry the CTA records IRKMG_ETIMEOUT, waits (bounded) for its own copies
// still in flight and returns.
// ---------------------------------------------------------------------------
constexpr int kKronStagedThreads = 256;
constexpr int kKronMaxStages = 4;

struct KronStaged {
  KronApply a;
  int stages;
  uint32_t stage_bytes;  // bytes per stage (largest patch block, rounded to 128)
  uint32_t work_off;     // offset of the work arrays in dynamic shared memory
  int64_t spins;
  int* err;
};

template <typename T, bool TR>
__global__ void __launch_bounds__(kKronStagedThreads, 5)
    k_vanka_apply_kron_staged(KronStaged S, const T* __restrict__ fac) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar[kKronMaxStages];
  __shared__ int s_n[kKronMaxStages];  // patch size n of the block in each stage
  __shared__ int s_abort;
  const KronApply& P = S.a;
  const int tid = threadIdx.x;
  const int nmax = P.nmax;
  double* s_r = reinterpret_cast<double*>(dyn + S.work_off);  // s · nmax
  double* s_acc = s_r + P.s * nmax;                           // nt · nmax
  T* s_rm = reinterpret_cast<T*>(s_r);
  T* s_accm = reinterpret_cast<T*>(s_acc);
  T* s_src = reinterpret_cast<T*>(s_acc + P.nt * nmax);        // max(ns, nt) · nmax
  const int nsrc = TR ? P.nt : P.ns;
  const int64_t nmine = (P.count > blockIdx.x) ? (P.count - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int st = 0; st < S.stages; ++st) mbar_init(&bar[st], 1);
    s_abort = 0;
  }
  fence_proxy_async();
  __syncthreads();

  auto mats_bytes = [&](int n) -> int64_t {
    return ((int64_t)P.nm * n * n * (int64_t)sizeof(T) + 15) & ~(int64_t)15;
  };
  const uint64_t pol = l2_evict_first_policy();
  // Thread 0 issues the copies.  The size and offset of the next patch to be
  // issued are loaded one issue ahead (nx, ox), so no issue waits on a global
  // load; the size travels to the other threads through s_n.
  int nx = 0;
  int64_t ox = 0;
  auto meta = [&](int64_t k) {
    if (k < nmine) {
      const int64_t pi = kron_pi(P, blockIdx.x + k * gridDim.x);
      nx = P.np[pi];
      ox = P.fac_off[pi];
    }
  };
  auto issue = [&](int st) {  // the patch whose metadata is in (nx, ox)
    const uint32_t bytes = (uint32_t)(mats_bytes(nx) + (((int64_t)nx * 4 + 15) & ~(int64_t)15));
    s_n[st] = nx;
    mbar_expect_tx(&bar[st], bytes);
    bulk_g2s(dyn + (size_t)st * S.stage_bytes, fac + ox, bytes, &bar[st], pol);
  };
  if (tid == 0) {
    const int64_t pre = nmine < S.stages ? nmine : S.stages;
    for (int64_t k = 0; k < pre; ++k) {
      meta(k);
      issue((int)k);
    }
    meta(pre);
  }

  // Thread tid < s·n owns entry tid of the gathered stage residual: its global
  // index, the residual value and the current target value.  Patch k+1's
  // entries are loaded while patch k is computed (patches of one colour are
  // disjoint, so patch k's writes never touch them).
  int64_t gix = -1, qo = 0;
  double rv = 0.0, ov = 0.0;
  auto wait_stage = [&](int64_t k) {
    if (!mbar_wait_bounded(&bar[k % S.stages], (uint32_t)((k / S.stages) & 1), S.spins)) {
      s_abort = 1;
      atomicCAS(&S.err[0], 0, IRKMG_ETIMEOUT);
      return false;
    }
    return true;
  };
  auto gather = [&](int64_t k) {
    const int n = s_n[k % S.stages];
    const int32_t* G = reinterpret_cast<const int32_t*>(dyn + (size_t)(k % S.stages) * S.stage_bytes +
                                                        mats_bytes(n));
    gix = -1;
    if (tid < P.s * n) {
      const int t = tid / n, i = tid - t * n;
      gix = t * P.m + G[i];
      rv = P.r[gix];
      if (P.ybuf)
        qo = P.qoff[kron_pi(P, blockIdx.x + k * gridDim.x)];
      else
        ov = P.out[gix];
    }
  };
  // in flight after the prologue: copies 0 .. min(nmine, stages) - 1
  // copies issued and perhaps in flight: patches from .. upto - 1
  auto drain = [&](int64_t from, int64_t upto) {
    for (int64_t j = from; j < nmine && j < upto; ++j)
      mbar_drain(&bar[j % S.stages], (uint32_t)((j / S.stages) & 1));
  };
  __syncthreads();  // s_n of the first stages
  if (nmine > 0 && wait_stage(0)) gather(0);
  __syncthreads();
  if (s_abort) {
    drain(0, S.stages);
    return;
  }

  for (int64_t k = 0; k < nmine; ++k) {
    const int st = (int)(k % S.stages);
    const int n = s_n[st];
    const T* X = reinterpret_cast<const T*>(dyn + (size_t)st * S.stage_bytes);
    const int64_t nn = (int64_t)n * n;
    const int64_t gk = gix, qk = qo;
    const double ok_ = ov;
    if (gk >= 0) s_rm[tid] = (T)rv;
    __syncthreads();
    if (k + 1 < nmine && wait_stage(k + 1)) gather(k + 1);
    for (int idx = tid; idx < nsrc * n; idx += kKronStagedThreads) {
      const int c = idx / n, i = idx - c * n;
      T a = (T)0;
      for (int t = 0; t < P.s; ++t)
        a = fma(TR ? mix_h<T>(P, t * kKronMaxTasks + c) : mix_g<T>(P, c * 3 + t), s_rm[t * n + i], a);
      s_src[idx] = a;
    }
    __syncthreads();
    for (int tau = tid; tau < P.nt * n; tau += kKronStagedThreads) {
      const int task = tau / n, i = tau - task * n;
      const T* M = X + (int64_t)P.task_mat[task] * nn + (TR ? (int64_t)i * n : (int64_t)i);
      const T* src = s_src + (TR ? task : P.task_src[task]) * n;
      const int64_t step = TR ? 1 : n;
      T a0 = (T)0, a1 = (T)0;
      int j = 0;
#pragma unroll 4
      for (; j + 1 < n; j += 2) {
        a0 = fma(M[j * step], src[j], a0);
        a1 = fma(M[(j + 1) * step], src[j + 1], a1);
      }
      if (j < n) a0 = fma(M[j * step], src[j], a0);
      s_accm[tau] = a0 + a1;
    }
    __syncthreads();
    if (gk >= 0) {
      const int t = tid / n, i = tid - t * n;
      T x = (T)0;
      for (int tau = 0; tau < P.nt; ++tau) {
        const T h = TR ? mix_g<T>(P, P.task_src[tau] * 3 + t) : mix_h<T>(P, t * kKronMaxTasks + tau);
        x = fma(h, s_accm[tau * n + i], x);
      }
      if (P.ybuf)
        P.ybuf[t * P.Q + qk + i * P.ys] = (double)x;
      else
        P.out[gk] = ok_ + P.scale * (double)x;
    }
    fence_proxy_async();
    __syncthreads();  // stage st and the work arrays fully consumed
    if (s_abort) {  // patches up to k + stages - 1 were issued
      drain(k + 1, k + S.stages);
      return;
    }
    if (tid == 0 && k + S.stages < nmine) {
      issue(st);
      meta(k + S.stages + 1);
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised decoupled apply (persistent over the patches of a launch).
// Warp 0 is the producer: lane 0 streams patch blocks into a ring of stages
// with cp.async.bulk (completion on full[st]) and reuses a stage once its
// consumer has arrived on empty[st].  Warps 1..kWsConsumers each take every
// kWsConsumers-th patch of the CTA and work on it alone (warp-synchronous:
// gather, sources, matrix-centric units from the stage, results), so no
// CTA-wide barrier sits between patches.  The stage is released as soon as
// its matrices are consumed.  Every wait is bounded; on expiry the CTA
// records IRKMG_ETIMEOUT, the consumers leave and the producer waits (bounded)
// for the copies it issued before it returns.
// ---------------------------------------------------------------------------
constexpr int kWsConsumers = 7;
constexpr int kWsThreads = 32 * (kWsConsumers + 1);
constexpr int kWsMaxStages = 8;

struct KronWs {
  KronApply a;
  int stages;
  uint32_t stage_bytes;
  uint32_t work_off;    // per-warp work arrays after the stages
  uint32_t warp_bytes;  // bytes of one consumer's work arrays
  int64_t spins;
  int* err;
};

__host__ __device__ inline uint32_t ws_warp_bytes(int s, int ns, int nt, int nmax, int tsize) {
  const int nsrc = ns > nt ? ns : nt;
  const size_t b = (size_t)(s + nt) * nmax * 8 + (size_t)nsrc * nmax * tsize + (size_t)nmax * 4;
  return (uint32_t)((b + 15) & ~(size_t)15);
}

template <typename T, bool TR>
__global__ void __launch_bounds__(kWsThreads) k_vanka_apply_kron_ws(KronWs W, const T* __restrict__ fac) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ __align__(8) uint64_t full[kWsMaxStages];
  __shared__ __align__(8) uint64_t empty[kWsMaxStages];
  __shared__ int s_n[kWsMaxStages];
  __shared__ volatile long long s_seq[kWsMaxStages];  // patch index of each stage's current fill
  __shared__ volatile int s_abort;
  const KronApply& P = W.a;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nmine = (P.count > blockIdx.x) ? (P.count - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int S = W.stages;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
      s_seq[st] = -1;
    }
    s_abort = 0;
  }
  fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  auto mats_bytes = [&](int n) -> int64_t {
    return ((int64_t)P.nm * n * n * (int64_t)sizeof(T) + 15) & ~(int64_t)15;
  };
  if (warp == 0) {
    // ---- producer ----
    if (lane == 0) {
      const uint64_t pol = l2_evict_first_policy();
      int64_t issued = 0;
      for (int64_t k = 0; k < nmine; ++k) {
        const int st = (int)(k % S);
        if (k >= S && !mbar_wait_bounded(&empty[st], (uint32_t)(((k / S) - 1) & 1), W.spins)) {
          s_abort = 1;
          atomicCAS(&W.err[0], 0, IRKMG_ETIMEOUT);
        }
        if (s_abort) break;
        const int64_t pi = kron_pi(P, blockIdx.x + k * gridDim.x);
        const int n = P.np[pi];
        const uint32_t bytes = (uint32_t)(mats_bytes(n) + (((int64_t)n * 4 + 15) & ~(int64_t)15));
        s_n[st] = n;
        __threadfence_block();
        s_seq[st] = k;  // after this the stage's barrier is one phase behind patch k
        mbar_expect_tx(&full[st], bytes);
        bulk_g2s(dyn + (size_t)st * W.stage_bytes, fac + P.fac_off[pi], bytes, &full[st], pol);
        issued = k + 1;
      }
      if (s_abort)  // copies still in flight complete before the CTA leaves
        for (int64_t k = issued > S ? issued - S : 0; k < issued; ++k)
          mbar_drain(&full[k % S], (uint32_t)((k / S) & 1));
    }
    return;
  }
  // ---- consumers ----
  const int c = warp - 1;
  const int nmax = P.nmax;
  unsigned char* wb = dyn + W.work_off + (size_t)c * W.warp_bytes;
  double* s_r = reinterpret_cast<double*>(wb);
  double* s_acc = s_r + P.s * nmax;
  T* s_rm = reinterpret_cast<T*>(s_r);
  T* s_accm = reinterpret_cast<T*>(s_acc);
  T* s_src = reinterpret_cast<T*>(s_acc + P.nt * nmax);
  const int nsrc = TR ? P.nt : P.ns;
  int32_t* s_g = reinterpret_cast<int32_t*>(s_src + (P.ns > P.nt ? P.ns : P.nt) * nmax);
  for (int64_t k = c; k < nmine; k += kWsConsumers) {
    const int st = (int)(k % S);
    if (__any_sync(0xffffffffu, s_abort != 0)) return;  // the whole warp leaves together
    // Patches of one stage go to different consumers, so a consumer may reach
    // stage st before the fill for patch k - S has completed; a parity wait
    // would then match the older phase.  Waiting until the producer has
    // started patch k's fill (s_seq) leaves the barrier exactly one phase
    // behind, and the parity wait below is for patch k's copy.
    bool started = s_seq[st] == k;
    if (!started) {
      const uint64_t t0 = global_ns();
      for (int64_t it = 0; it < W.spins && !s_abort; ++it) {
        if (s_seq[st] == k) {
          started = true;
          break;
        }
        if ((it & 255) == 255 && global_ns() - t0 > 2000000000ull) break;
      }
    }
    const bool ok = started && mbar_wait_bounded(&full[st], (uint32_t)((k / S) & 1), W.spins);
    if (!__all_sync(0xffffffffu, ok)) {  // warp-uniform: the whole warp leaves together
      if (lane == 0) {
        s_abort = 1;
        atomicCAS(&W.err[0], 0, IRKMG_ETIMEOUT);
      }
      return;
    }
    const int64_t pi = kron_pi(P, blockIdx.x + k * gridDim.x);
    const int n = s_n[st];
    const int64_t nn = (int64_t)n * n;
    const T* X = reinterpret_cast<const T*>(dyn + (size_t)st * W.stage_bytes);
    const int32_t* G =
        reinterpret_cast<const int32_t*>(dyn + (size_t)st * W.stage_bytes + mats_bytes(n));
    for (int i = lane; i < n; i += 32) s_g[i] = G[i];
    __syncwarp();
    for (int idx = lane; idx < P.s * n; idx += 32) {
      const int t = idx / n, i = idx - t * n;
      s_rm[idx] = (T)P.r[t * P.m + s_g[i]];
    }
    __syncwarp();
    for (int idx = lane; idx < nsrc * n; idx += 32) {
      const int cc = idx / n, i = idx - cc * n;
      T a = (T)0;
      for (int t = 0; t < P.s; ++t)
        a = fma(TR ? mix_h<T>(P, t * kKronMaxTasks + cc) : mix_g<T>(P, cc * 3 + t), s_rm[t * n + i], a);
      s_src[idx] = a;
    }
    __syncwarp();
    // units (matrix b, row i); transposed: row i of Mᵀ is column i of M
    for (int u = lane; u < P.nm * n; u += 32) {
      const int b = u / n, i = u - b * n;
      const T* M = X + (int64_t)b * nn + (TR ? (int64_t)i * n : (int64_t)i);
      const int64_t step = TR ? 1 : n;
      const int t0 = P.mat_task[b][0], t1 = P.mat_task[b][1];
      const int t1s = t1 >= 0 ? t1 : t0;
      const T* q0 = s_src + (TR ? t0 : P.task_src[t0]) * n;
      const T* q1 = s_src + (TR ? t1s : P.task_src[t1s]) * n;
      T a0 = (T)0, a1 = (T)0;
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const T m = M[j * step];
        a0 = fma(m, q0[j], a0);
        a1 = fma(m, q1[j], a1);
      }
      s_accm[t0 * n + i] = a0;
      if (t1 >= 0) s_accm[t1 * n + i] = a1;
    }
    fence_proxy_async();  // the stage's reads before the producer's next copy into it
    __syncwarp();
    if (lane == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[st])) : "memory");
    for (int idx = lane; idx < P.s * n; idx += 32) {
      const int t = idx / n, i = idx - t * n;
      T x = (T)0;
      for (int tau = 0; tau < P.nt; ++tau) {
        const T h = TR ? mix_g<T>(P, P.task_src[tau] * 3 + t) : mix_h<T>(P, t * kKronMaxTasks + tau);
        x = fma(h, s_accm[tau * n + i], x);
      }
      if (P.ybuf)
        P.ybuf[t * P.Q + P.qoff[pi] + i * P.ys] = (double)x;
      else
        P.out[t * P.m + s_g[i]] += P.scale * (double)x;
    }
    __syncwarp();
  }
}

// Launch shape of the warp-specialised apply: two CTAs per SM when each holds
// at least four stages besides the consumers' work arrays, else one CTA with
// as many stages as fit (at least two).
struct WsShape {
  int stages;
  uint32_t stage_bytes, work_off, warp_bytes, dyn_bytes;
};

static bool kron_ws_config(const KronPlan& K, int nmax, int prec, WsShape* out) {
  const size_t w = prec == 64 ? 8 : 4;
  const size_t blk = (((size_t)K.nm * nmax * nmax * w + 15) & ~(size_t)15) +
                     (((size_t)nmax * 4 + 15) & ~(size_t)15);
  const size_t sb = (blk + 127) & ~(size_t)127;
  const uint32_t wbytes = ws_warp_bytes(K.s, K.ns, K.nt, nmax, (int)w);
  const size_t work = (size_t)kWsConsumers * wbytes;
  const size_t static_b = 256;
  for (int ctas = 2; ctas >= 1; --ctas) {
    const size_t lim = std::min((size_t)233472 / ctas - 1024, (size_t)232448);
    if (lim < static_b + work + 2 * sb) continue;
    int st = (int)((lim - static_b - work) / sb);
    if (st > kWsMaxStages) st = kWsMaxStages;
    if (ctas == 2 && st < 4) continue;
    out->stages = st;
    out->stage_bytes = (uint32_t)sb;
    out->work_off = (uint32_t)(st * sb);
    out->warp_bytes = wbytes;
    out->dyn_bytes = (uint32_t)(st * sb + work);
    return true;
  }
  return false;
}

bool kron_ws_fits(Ctx& C, Level& L) {
  WsShape shp;
  return kron_ws_config(C.kplan, L.kron_nmax, C.opt.patch_precision, &shp);
}

template <typename T, bool TR>
cudaError_t launch_kron_ws(const KronWs& W, const T* fac, const WsShape& shp, cudaStream_t st,
                           int* cap_cache) {
  auto kern = k_vanka_apply_kron_ws<T, TR>;
  static uint32_t limit[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (shp.dyn_bytes > limit[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shp.dyn_bytes);
    if (e != cudaSuccess) return e;
    limit[dev] = shp.dyn_bytes;
  }
  if (*cap_cache == 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWsThreads, shp.dyn_bytes);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *cap_cache = nsm * (per_sm < 1 ? 1 : per_sm);
  }
  const int64_t cap = *cap_cache;
  const int64_t ctas = W.a.count < cap ? W.a.count : cap;
  kern<<<(unsigned)ctas, kWsThreads, shp.dyn_bytes, st>>>(W, fac);
  return cudaGetLastError();
}

// Launch shapes of the staged decoupled apply for a level.  Shape 0: the most
// CTAs per SM (up to 5, the register bound) that leave room for three stages
// each (the block of patch k+1 is waited for while patch k is computed, so
// three stages keep one block of look-ahead in flight), else for two.  Shape
// 1: the most CTAs with two stages.  The autotuner times both.  False when
// s·n_max exceeds the CTA or not even one CTA with two stages fits.
struct KronShape {
  int stages, ctas_per_sm;
  uint32_t stage_bytes, work_off, dyn_bytes;
};

static bool kron_staged_config(const KronPlan& K, int nmax, int prec, int shape, KronShape* out) {
  if (K.s * nmax > kKronStagedThreads) return false;
  const size_t w = prec == 64 ? 8 : 4;
  const size_t blk = (((size_t)K.nm * nmax * nmax * w + 15) & ~(size_t)15) +
                     (((size_t)nmax * 4 + 15) & ~(size_t)15);
  const size_t sb = (blk + 127) & ~(size_t)127;
  const int nsrc = K.ns > K.nt ? K.ns : K.nt;
  const size_t work = (size_t)(K.s + K.nt) * nmax * 8 + (size_t)nsrc * nmax * w + 16;
  const size_t static_b = 128;
  const size_t per_sm = 233472, reserved = 1024, per_block = 232448;
  for (int want = shape == 0 ? 3 : 2; want >= 2; --want)
    for (int ctas = 5; ctas >= 1; --ctas) {
      const size_t lim = std::min(per_sm / ctas - reserved, per_block);
      if (lim < static_b + work + want * sb) continue;
      int st = (int)((lim - static_b - work) / sb);
      if (st > kKronMaxStages) st = kKronMaxStages;
      out->stages = st;
      out->ctas_per_sm = ctas;
      out->stage_bytes = (uint32_t)sb;
      out->work_off = (uint32_t)(st * sb);
      out->dyn_bytes = (uint32_t)(st * sb + work);
      return true;
    }
  return false;
}

bool kron_staged_fits(Ctx& C, Level& L, int shape) {
  KronShape shp;
  return kron_staged_config(C.kplan, L.kron_nmax, C.opt.patch_precision, shape, &shp);
}

// The kernel's dynamic shared-memory limit is a property of the function: it
// is only ever raised (per device), so launches of other levels with smaller
// shapes stay valid.  The residency for the level's shape is looked up once
// (cached in *cap); one CTA is launched per resident slot (at most one per
// patch).
template <typename T, bool TR>
cudaError_t launch_kron_staged(const KronStaged& S, const T* fac, const KronShape& shp,
                               cudaStream_t st, int* cap_cache) {
  auto kern = k_vanka_apply_kron_staged<T, TR>;
  static uint32_t limit[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (shp.dyn_bytes > limit[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shp.dyn_bytes);
    if (e != cudaSuccess) return e;
    limit[dev] = shp.dyn_bytes;
  }
  if (*cap_cache == 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kKronStagedThreads,
                                                      shp.dyn_bytes);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *cap_cache = nsm * (per_sm < 1 ? 1 : per_sm);
  }
  const int64_t cap = *cap_cache;
  const int64_t ctas = S.a.count < cap ? S.a.count : cap;
  kern<<<(unsigned)ctas, kKronStagedThreads, shp.dyn_bytes, st>>>(S, fac);
  return cudaGetLastError();
}

template <typename T, bool TR>
cudaError_t launch_kron_t(const KronApply& P, const T* fac, int R, unsigned grid, size_t smem,
                          cudaStream_t st) {
#define KRON_CASE(RR)                                                                         \
  case RR:                                                                                    \
    cudaFuncSetAttribute(k_vanka_apply_kron<T, RR, TR>,                                       \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
    k_vanka_apply_kron<T, RR, TR><<<grid, kKronWarps * 32, smem, st>>>(P, fac);               \
    break;
  if constexpr (TR) {  // the transposed apply (adjoint) is not tuned per size
    cudaFuncSetAttribute(k_vanka_apply_kron<T, kKronMaxSlots, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_vanka_apply_kron<T, kKronMaxSlots, true><<<grid, kKronWarps * 32, smem, st>>>(P, fac);
    return cudaGetLastError();
  } else {
  switch (R) {
    KRON_CASE(2)
    KRON_CASE(3)
    KRON_CASE(4)
    KRON_CASE(5)
    KRON_CASE(6)
    KRON_CASE(7)
    KRON_CASE(8)
    default:
      cudaFuncSetAttribute(k_vanka_apply_kron<T, kKronMaxSlots, TR>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_vanka_apply_kron<T, kKronMaxSlots, TR><<<grid, kKronWarps * 32, smem, st>>>(P, fac);
      break;
  }
  }
#undef KRON_CASE
  return cudaGetLastError();
}

cudaError_t launch_vanka_kron(Ctx& C, Level& L, int colour, const double* r, double* out,
                              double scale, int transpose) {
  const KronPlan& K = C.kplan;
  KronApply P{};
  P.s = C.s;
  P.ns = K.ns;
  P.nt = K.nt;
  P.nm = K.nm;
  P.m = L.m;
  for (int i = 0; i < kKronMaxSrc * 3; ++i) P.G[i] = K.G[i], P.Gf[i] = (float)K.G[i];
  for (int i = 0; i < 3 * kKronMaxTasks; ++i) P.H[i] = K.H[i], P.Hf[i] = (float)K.H[i];
  for (int i = 0; i < kKronMaxTasks; ++i) {
    P.task_mat[i] = K.task_mat[i];
    P.task_src[i] = K.task_src[i];
    P.mat_task[i][0] = P.mat_task[i][1] = -1;
  }
  for (int t = 0; t < K.nt; ++t) {
    int* mt = P.mat_task[K.task_mat[t]];
    if (mt[0] < 0)
      mt[0] = t;
    else
      mt[1] = t;
  }
  P.np = L.d_np;
  P.fac_off = L.d_fac_off;
  P.r = r;
  P.out = out;
  P.scale = scale;
  if (colour < 0) {  // one launch over all patches, results to the reduction buffer
    P.first = 0;
    P.count = L.nv;
    P.ybuf = C.d_Y;
    P.qoff = L.d_qoff;
    P.Q = L.Q;
    P.ys = L.ystride;
    P.perm = L.d_perm;
  } else {
    P.first = L.colour_start[colour];
    P.count = L.colour_start[colour + 1] - P.first;
    P.ybuf = nullptr;
    P.qoff = nullptr;
    P.Q = 0;
    P.ys = 1;
    P.perm = nullptr;
  }
  P.nmax = L.kron_nmax;
  if (P.count <= 0) return cudaSuccess;
  if (L.fixed)  // kernels 8, 9 and 10: the stored blocks are fixed point
    return launch_vanka_kron_fx(C, L, colour, r, out, scale, transpose);
  const int prec = C.opt.patch_precision;
  if (L.apply_kernel == 7) {
    WsShape wsh;
    if (!kron_ws_config(K, L.kron_nmax, prec, &wsh)) return cudaErrorInvalidConfiguration;
    KronWs W{};
    W.a = P;
    W.stages = wsh.stages;
    W.stage_bytes = wsh.stage_bytes;
    W.work_off = wsh.work_off;
    W.warp_bytes = wsh.warp_bytes;
    W.spins = C.opt.timeout_spins > 0 ? C.opt.timeout_spins : (int64_t)1 << 26;
    W.err = C.d_err;
    int* cap = &L.ws_cap[transpose ? 1 : 0];
    if (prec == 64) {
      const double* f = (const double*)L.d_fac;
      return transpose ? launch_kron_ws<double, true>(W, f, wsh, C.stream, cap)
                       : launch_kron_ws<double, false>(W, f, wsh, C.stream, cap);
    }
    const float* f = (const float*)L.d_fac;
    return transpose ? launch_kron_ws<float, true>(W, f, wsh, C.stream, cap)
                     : launch_kron_ws<float, false>(W, f, wsh, C.stream, cap);
  }
  if (L.apply_kernel == 6) {
    if (transpose) return cudaErrorNotSupported;
    if (prec == 64)
      k_vanka_apply_kron_big<double><<<(unsigned)P.count, kKronBigThreads, 0, C.stream>>>(
          P, (const double*)L.d_fac);
    else
      k_vanka_apply_kron_big<float><<<(unsigned)P.count, kKronBigThreads, 0, C.stream>>>(
          P, (const float*)L.d_fac);
    return cudaGetLastError();
  }
  KronShape shp;
  if (L.apply_kernel == 5 && kron_staged_config(K, L.kron_nmax, prec, L.kron_shape, &shp)) {
    KronStaged S{};
    S.a = P;
    S.stages = shp.stages;
    S.stage_bytes = shp.stage_bytes;
    S.work_off = shp.work_off;
    S.spins = C.opt.timeout_spins > 0 ? C.opt.timeout_spins : (int64_t)1 << 26;
    S.err = C.d_err;
    int* cap = &L.kron_cap[L.kron_shape][transpose ? 1 : 0];
    if (prec == 64) {
      const double* f = (const double*)L.d_fac;
      return transpose ? launch_kron_staged<double, true>(S, f, shp, C.stream, cap)
                       : launch_kron_staged<double, false>(S, f, shp, C.stream, cap);
    }
    const float* f = (const float*)L.d_fac;
    return transpose ? launch_kron_staged<float, true>(S, f, shp, C.stream, cap)
                     : launch_kron_staged<float, false>(S, f, shp, C.stream, cap);
  }
  const size_t smem =
      (size_t)kKronWarps * kron_warp_bytes(P.s, P.ns, P.nt, P.nmax, prec == 64 ? 8 : 4);
  const unsigned grid = (unsigned)((P.count + kKronWarps - 1) / kKronWarps);
  const int R = (K.nt * L.kron_nmax + 31) / 32;
  if (prec == 64) {
    const double* f = (const double*)L.d_fac;
    return transpose ? launch_kron_t<double, true>(P, f, R, grid, smem, C.stream)
                     : launch_kron_t<double, false>(P, f, R, grid, smem, C.stream);
  }
  const float* f = (const float*)L.d_fac;
  bool real = false;
  if (!transpose && L.kron_nmax == kPairN && fx_pair_plan(K, &real)) {  // paired FP32 rows
    const size_t wb = std::max(kron_warp_bytes(P.s, P.ns, P.nt, P.nmax, 4), sizeof(KronPairSmem));
    const size_t sm2 = (size_t)kKronWarps * wb;
    auto kern = real ? k_vanka_apply_kron_pair32<true> : k_vanka_apply_kron_pair32<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    kern<<<grid, kKronWarps * 32, sm2, C.stream>>>(P, f, (uint32_t)wb);
    return cudaGetLastError();
  }
  return transpose ? launch_kron_t<float, true>(P, f, R, grid, smem, C.stream)
                   : launch_kron_t<float, false>(P, f, R, grid, smem, C.stream);
}

}  // namespace irkmg

namespace irkmg {

// Deterministic gather of the one-launch patch results: for every stage t and
// spatial DoF d, out[t·m + d] += scale · Σ_e ybuf[t·Q + e] over the entries e
// of d (one per patch containing d, in the colour-ordered patch order).
// One spatial DoF per thread, all S stages: the contribution indices of a
// DoF are loaded eight at a time and their S·8 results issued together; each
// stage's sum still runs over the contributions in order (bitwise the sum of
// the batched smoother) and is added to out with one rounding.
template <int S, bool CHEB>
__global__ void __launch_bounds__(256) k_vanka_reduce(int64_t m, int64_t Q,
                                                      const int32_t* __restrict__ cptr,
                                                      const int32_t* __restrict__ cidx,
                                                      const double* __restrict__ y, double scale,
                                                      double* __restrict__ out, ChebFuse F) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= m) return;
  const int32_t e0 = cptr[d], e1 = cptr[d + 1];
  double a[S];
#pragma unroll
  for (int t = 0; t < S; ++t) a[t] = 0.0;
  for (int32_t e = e0; e < e1; e += 8) {
    int32_t c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = e + k < e1 ? cidx[e + k] : -1;
    double v[8][S];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int t = 0; t < S; ++t) v[k][t] = c[k] >= 0 ? y[t * Q + c[k]] : 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c[k] >= 0)
#pragma unroll
        for (int t = 0; t < S; ++t) a[t] += v[k][t];
  }
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const int64_t g = t * m + d;
    if (!CHEB) {
      out[g] = __fma_rn(scale, a[t], out[g]);
    } else {
      const double d2 = __fma_rn(scale, a[t], F.dzero ? 0.0 : __dmul_rn(F.c1, out[g]));
      out[g] = d2;
      F.x[g] = F.xadd ? __dadd_rn(d2, F.x[g]) : d2;
    }
  }
}

cudaError_t launch_vanka_reduce(Ctx& C, Level& L, double* out, double scale, const ChebFuse* f) {
  const unsigned grid = (unsigned)((L.m + 255) / 256);
  const ChebFuse F = f ? *f : ChebFuse{1.0, false, false, nullptr};
#define REDUCE_CASE(S_)                                                                     \
  case S_:                                                                                  \
    if (f)                                                                                  \
      k_vanka_reduce<S_, true><<<grid, 256, 0, C.stream>>>(L.m, L.Q, L.d_cptr, L.d_cidx,    \
                                                           C.d_Y, scale, out, F);           \
    else                                                                                    \
      k_vanka_reduce<S_, false><<<grid, 256, 0, C.stream>>>(L.m, L.Q, L.d_cptr, L.d_cidx,   \
                                                            C.d_Y, scale, out, F);          \
    break;
  switch (C.s) {
    REDUCE_CASE(1)
    REDUCE_CASE(2)
    REDUCE_CASE(3)
    default: return cudaErrorInvalidValue;
  }
#undef REDUCE_CASE
  return cudaGetLastError();
}

}  // namespace irkmg

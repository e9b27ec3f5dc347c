// Exact fixed-point apply of the decoupled FP64 patch inverses (the Vanka
// patch solves of Section 4.2 in the Kronecker-decoupled form).
//
// GB300 retires 2 FP64 FMAs per clock per SM and an order of magnitude more
// 32 × 32 → 64-bit integer multiply-adds with a 64-bit addend (mad.wide.s32),
// so four of those per matrix entry leave the decoupled mat-vecs bound by HBM
// instead of by the FP64 pipe.  Each row i of a stored inverse block M
// (column-major, n ≤ 63) is kept as 57-bit fixed point with its own power of
// two,
//     M_ij = q_ij 2^(E_i − 57),   |q_ij| ≤ 2^57,   q_ij = a1 2^29 + a0,
// a0 in [−2^28, 2^28) (two int32 per entry: eight bytes, as in FP64), and
// every source vector of a patch is scaled by one power of two to integers
//     x_j = v_j 2^(F − 58),   |v_j| ≤ 2^58,   v_j = v1 2^29 + v0,
// v0 in [−2^28, 2^28).  The four limb products a1·v1, a1·v0, a0·v1, a0·v0
// (each at most about 2^57) go to four 64-bit accumulators (n ≤ 63 terms
// cannot overflow), which are combined into the exact dot product
// Σ_j q_ij v_j (below 2^121) and rounded once to FP64:
//     y_i = round(Σ_j q_ij v_j) · 2^(E_i + F − 115).
// The only errors are the two conversions (at most 2^−57 of the row's largest
// entry, 2^−58 of the source's largest entry) and that one rounding; an FP64
// dot product rounds each of its n partial sums instead.
//
// The transposed apply (adjoint) sums down a column, across rows with
// different E_j; there the source entries are pre-scaled by the exact powers
// of two 2^(E_j − max_j E_j) before their conversion.
//
// Two kernels: warp per patch (k_vanka_apply_kron_fx; entries streamed into
// registers in column batches) and a TMA-staged persistent kernel
// (k_vanka_apply_kron_fx_staged); the set-up autotuner picks per level.
#include <algorithm>
#include <climits>

#include "fx_math.h"
#include "fx_patch.cuh"
#include "irkmg_internal.h"
#include "tma.cuh"

namespace irkmg {

namespace {

// One warp per (ordered patch, stored matrix), lanes over rows: the row
// exponent E_i (|M_ij| < 2^E_i for every j) and the entries rewritten in
// place as (a0, a1) pairs.  A non-finite entry reports IRKMG_ESINGULAR.
__global__ void k_patch_to_fixed(int nm, int nmax, int64_t npatch, const int32_t* __restrict__ np,
                                 const int64_t* __restrict__ fac_off,
                                 const int32_t* __restrict__ order, double* fac,
                                 int16_t* __restrict__ fexp, int* err) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= npatch * nm) return;
  const int64_t pi = w / nm;
  const int mat = (int)(w - pi * nm);
  const int n = np[pi];
  const int64_t nn = (int64_t)n * n;
  double* X = fac + fac_off[pi] + mat * nn;
  int2* Q = reinterpret_cast<int2*>(X);
  for (int i = lane; i < n; i += 32) {
    double mx = 0.0;
    bool finite = true;
    for (int j = 0; j < n; ++j) {
      const double a = X[(int64_t)j * n + i];
      finite = finite && isfinite(a);
      mx = fmax(mx, fabs(a));
    }
    int E = 0;
    if (!finite) {
      if (atomicCAS(&err[0], 0, IRKMG_ESINGULAR) == 0) err[1] = order[pi];
    } else if (mx > 0.0) {
      frexp(mx, &E);  // mx = f 2^E, f in [1/2, 1): every |M_ij| < 2^E
    }
    fexp[(pi * nm + mat) * nmax + i] = (int16_t)E;
    for (int j = 0; j < n; ++j) {
      const double a = X[(int64_t)j * n + i];
      const int64_t q = finite ? fx_scale_round(a, 57 - E) : 0;
      int32_t a1, a0;
      fx_split29(q, &a1, &a0);
      Q[(int64_t)j * n + i] = make_int2(a0, a1);
    }
  }
}

template <int RC, int U, int MB, bool TR>
__global__ void __launch_bounds__(kFxWarps * 32, MB) k_vanka_apply_kron_fx(FxApply P,
                                                                       const int2* __restrict__ fac) {
  extern __shared__ __align__(128) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kFxWarps + warp;
  if (w >= P.count) return;
  unsigned char* base = dyn + (size_t)warp * fx_warp_bytes(P.s, P.nsrc, P.nt, P.nmax);
  const int64_t pi = fx_pi(P, w);
  const int n = P.np[pi];
  if (n == kFxN2)
    fx_patch<kFxN2, RC, U, TR>(P, fac, base, lane, pi, n);
  else
    fx_patch<0, RC, U, TR>(P, fac, base, lane, pi, n);
}

// Boundary stars (n < kFxN2) of the paired kernel, out of line so that their
// registers do not count against the interior path's.
__device__ __noinline__ void fx_patch_boundary(const FxApply& P, const int2* __restrict__ fac,
                                               unsigned char* base, int lane, int64_t pi, int n) {
  fx_patch<0, 1, 8, false>(P, fac, base, lane, pi, n);
}

// The paired kernel (complex layout, non-transposed): interior patches by
// fx_patch_pair, the others by fx_patch.
template <int U, int MB, bool REAL>
__global__ void __launch_bounds__(kFxWarps * 32, MB) k_vanka_apply_kron_fx_pair(
    FxApply P, const int2* __restrict__ fac, uint32_t warp_bytes) {
  extern __shared__ __align__(128) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kFxWarps + warp;
  if (w >= P.count) return;
  unsigned char* base = dyn + (size_t)warp * warp_bytes;
  const int64_t pi = fx_pi(P, w);
  const int n = P.np[pi];
  if (n == kFxN2)
    fx_patch_pair<U, REAL>(P, fac, base, lane, pi);
  else
    fx_patch_boundary(P, fac, base, lane, pi, n);
}

// ---------------------------------------------------------------------------
// TMA-staged fixed-point apply (persistent over the patches of a launch): the
// patch blocks (stored fixed-point matrices + index list, one contiguous run)
// stream into a ring of shared-memory stages by cp.async.bulk while the CTA
// works on one patch at a time, so a block's latency is hidden behind the
// blocks ahead of it and no register holds data in flight.  Per patch: the
// gathered residual, the FP64 sources, their limbs (one warp per source),
// one (task, row) dot product per thread from the stage, the FP64
// recombination.  Every mbarrier wait is bounded: on expiry the CTA records
// IRKMG_ETIMEOUT, waits (bounded) for its own copies still in flight and
// returns.
// ---------------------------------------------------------------------------
constexpr int kFxStagedThreads = 256;
constexpr int kFxMaxStages = 4;

struct FxStaged {
  FxApply a;
  int stages;
  uint32_t stage_bytes;  // bytes per stage (largest patch block, rounded to 128)
  uint32_t work_off;     // offset of the work arrays in dynamic shared memory
  int64_t spins;
  int* err;
};

// residuals (s·nmax doubles), sources then task results (max(nsrc, nt)·nmax
// doubles), limbs (nsrc·nmax)
__host__ __device__ inline size_t fx_staged_work_bytes(int s, int nsrc, int nt, int nmax) {
  const int na = nsrc > nt ? nsrc : nt;
  return (size_t)(s + na) * nmax * 8 + (size_t)nsrc * nmax * sizeof(Limbs) + 16;
}

template <bool TR>
__global__ void __launch_bounds__(kFxStagedThreads, 1)
    k_vanka_apply_kron_fx_staged(FxStaged S, const int2* __restrict__ fac) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar[kFxMaxStages];
  __shared__ int s_n[kFxMaxStages];
  __shared__ int s_abort;
  __shared__ int s_F[kKronMaxTasks], s_E[kKronMaxTasks];
  const FxApply& P = S.a;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nmax = P.nmax;
  const int na = P.nsrc > P.nt ? P.nsrc : P.nt;
  double* s_r = reinterpret_cast<double*>(dyn + S.work_off);  // s · nmax
  double* s_x = s_r + P.s * nmax;                             // na · nmax
  Limbs* s_lim = reinterpret_cast<Limbs*>(s_x + na * nmax);   // nsrc · nmax
  const int64_t nmine = (P.count > blockIdx.x) ? (P.count - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int st = 0; st < S.stages; ++st) mbar_init(&bar[st], 1);
    s_abort = 0;
  }
  fence_proxy_async();
  __syncthreads();

  auto mats_bytes = [&](int n) -> int64_t { return ((int64_t)P.nm * n * n * 8 + 15) & ~(int64_t)15; };
  const uint64_t pol = l2_evict_first_policy();
  int nx = 0;
  int64_t ox = 0;
  auto meta = [&](int64_t k) {
    if (k < nmine) {
      const int64_t pi = fx_pi(P, blockIdx.x + k * gridDim.x);
      nx = P.np[pi];
      ox = P.fac_off[pi];
    }
  };
  auto issue = [&](int st) {
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
        qo = P.qoff[fx_pi(P, blockIdx.x + k * gridDim.x)];
      else
        ov = P.out[gix];
    }
  };
  // copies issued and perhaps in flight: patches from .. upto - 1
  auto drain = [&](int64_t from, int64_t upto) {
    for (int64_t j = from; j < nmine && j < upto; ++j)
      mbar_drain(&bar[j % S.stages], (uint32_t)((j / S.stages) & 1));
  };
  __syncthreads();
  if (nmine > 0 && wait_stage(0)) gather(0);
  __syncthreads();
  if (s_abort) {
    drain(0, S.stages);
    return;
  }

  for (int64_t k = 0; k < nmine; ++k) {
    const int st = (int)(k % S.stages);
    const int n = s_n[st];
    const int64_t pi = fx_pi(P, blockIdx.x + k * gridDim.x);
    const int2* X = reinterpret_cast<const int2*>(dyn + (size_t)st * S.stage_bytes);
    const int nn = n * n;
    const int16_t* fe = P.fexp + pi * P.nm * nmax;
    const int64_t gk = gix, qk = qo;
    const double ok_ = ov;
    if (gk >= 0) s_r[tid] = rv;
    if (TR && warp < P.nsrc) {  // max_j E_j of the matrix task `warp` reads
      const int16_t* e = fe + P.task_mat[warp] * nmax;
      int mx = INT_MIN;
      for (int i = lane; i < n; i += 32) mx = max(mx, (int)e[i]);
      mx = warp_max_int(mx);
      if (lane == 0) s_E[warp] = mx;
    }
    __syncthreads();
    if (k + 1 < nmine && wait_stage(k + 1)) gather(k + 1);
    for (int idx = tid; idx < P.nsrc * n; idx += kFxStagedThreads) {
      const int c = idx / n, i = idx - c * n;
      double a = 0.0;
      for (int t = 0; t < P.s; ++t)
        a += (TR ? P.H[t * kKronMaxTasks + c] : P.G[c * 3 + t]) * s_r[t * n + i];
      if (TR) a = ldexp(a, (int)fe[P.task_mat[c] * nmax + i] - s_E[c]);
      s_x[idx] = a;
    }
    __syncthreads();
    if (warp < P.nsrc) {  // source `warp` to 58-bit integers, two limbs
      const int c = warp;
      const uint64_t mb = warp_absmax_bits(s_x + c * n, n, lane);
      const bool finite = mb < 0x7ff0000000000000ull;
      const int F = finite && mb != 0 ? fx_exponent(fx_from_bits(mb)) : 0;
      for (int i = lane; i < n; i += 32) {
        const int64_t v = finite ? fx_scale_round(s_x[c * n + i], 58 - F) : 0;
        Limbs L;
        fx_split29(v, &L.v1, &L.v0);
        s_lim[c * n + i] = L;
      }
      if (lane == 0) s_F[c] = finite ? F : INT_MIN;
    }
    __syncthreads();
    for (int tau = tid; tau < P.nt * n; tau += kFxStagedThreads) {
      const int task = tau / n, i = tau - task * n;
      const int mat = P.task_mat[task];
      const int ex = TR ? s_E[task] : (int)fe[mat * nmax + i];
      const int2* M = X + mat * nn + (TR ? i * n : i);
      const int step = TR ? 1 : n;
      const Limbs* L = s_lim + (TR ? task : P.task_src[task]) * n;
      int64_t acc[4] = {0, 0, 0, 0};
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const int2 q = M[j * step];
        const Limbs v = L[j];
        acc[0] = mad_wide(q.y, v.v1, acc[0]);
        acc[1] = mad_wide(q.y, v.v0, acc[1]);
        acc[2] = mad_wide(q.x, v.v1, acc[2]);
        acc[3] = mad_wide(q.x, v.v0, acc[3]);
      }
      const int F = s_F[TR ? task : P.task_src[task]];
      s_x[tau] = F == INT_MIN ? __longlong_as_double(0x7ff8000000000000ll)
                              : fx_round(acc, ex + F - 115);
    }
    __syncthreads();
    if (gk >= 0) {
      const int t = tid / n, i = tid - t * n;
      double x = 0.0;
      for (int tau = 0; tau < P.nt; ++tau) {
        const double h = TR ? P.G[P.task_src[tau] * 3 + t] : P.H[t * kKronMaxTasks + tau];
        x += h * s_x[tau * n + i];
      }
      if (P.ybuf)
        P.ybuf[t * P.Q + qk + i * P.ys] = x;
      else
        P.out[gk] = ok_ + P.scale * x;
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

// Staged launch shapes: stages per CTA and resident CTAs per SM.
constexpr int kFxStagedShapes = 3;
constexpr int kFxStagedStages[kFxStagedShapes] = {4, 3, 2};
constexpr int kFxStagedCtas[kFxStagedShapes] = {1, 1, 2};

struct FxStagedShape {
  int stages, ctas;
  uint32_t stage_bytes, work_off, dyn_bytes;
};

bool fx_staged_config(const KronPlan& K, int s, int nmax, int shape, FxStagedShape* out) {
  if (shape < 0 || shape >= kFxStagedShapes || s * nmax > kFxStagedThreads) return false;
  const size_t blk = (((size_t)K.nm * nmax * nmax * 8 + 15) & ~(size_t)15) +
                     (((size_t)nmax * 4 + 15) & ~(size_t)15);
  const size_t sb = (blk + 127) & ~(size_t)127;
  const int nsrc = K.ns > K.nt ? K.ns : K.nt;
  const size_t work = fx_staged_work_bytes(s, nsrc, K.nt, nmax);
  const int stages = kFxStagedStages[shape], ctas = kFxStagedCtas[shape];
  const size_t dyn = stages * sb + work;
  const size_t static_b = 256, per_sm = 233472, reserved = 1024, per_block = 232448;
  if (dyn + static_b > per_block || ctas * (dyn + static_b + reserved) > per_sm) return false;
  out->stages = stages;
  out->ctas = ctas;
  out->stage_bytes = (uint32_t)sb;
  out->work_off = (uint32_t)(stages * sb);
  out->dyn_bytes = (uint32_t)dyn;
  return true;
}

template <bool TR>
cudaError_t launch_fx_staged(const FxStaged& S, const int2* fac, const FxStagedShape& shp,
                             cudaStream_t st, int* cap_cache) {
  auto kern = k_vanka_apply_kron_fx_staged<TR>;
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFxStagedThreads, shp.dyn_bytes);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm > shp.ctas) per_sm = shp.ctas;
    *cap_cache = nsm * (per_sm < 1 ? 1 : per_sm);
  }
  const int64_t cap = *cap_cache;
  const int64_t ctas = S.a.count < cap ? S.a.count : cap;
  kern<<<(unsigned)ctas, kFxStagedThreads, shp.dyn_bytes, st>>>(S, fac);
  return cudaGetLastError();
}

template <int RC, int U, int MB, bool TR>
cudaError_t launch_fx_t(const FxApply& P, const int2* fac, unsigned grid, size_t smem,
                        cudaStream_t st) {
  auto kern = k_vanka_apply_kron_fx<RC, U, MB, TR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kFxWarps * 32, smem, st>>>(P, fac);
  return cudaGetLastError();
}

// Paired kernel shapes (kernel 10): columns per load batch, resident CTAs.
constexpr int kFxPairShapes = 2;
constexpr int kFxPairU[kFxPairShapes] = {8, 2};

size_t fx_pair_warp_bytes(const FxApply& P) {
  const size_t g = fx_warp_bytes(P.s, P.nsrc > P.nt ? P.nsrc : P.nt, P.nt, P.nmax);
  return g > sizeof(FxPairSmem) ? g : sizeof(FxPairSmem);
}

template <int U, bool REAL>
cudaError_t launch_fx_pair_t(const FxApply& P, const int2* fac, cudaStream_t st) {
  auto kern = k_vanka_apply_kron_fx_pair<U, 4, REAL>;
  const size_t wb = fx_pair_warp_bytes(P);
  const size_t smem = (size_t)kFxWarps * wb;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((P.count + kFxWarps - 1) / kFxWarps);
  kern<<<grid, kFxWarps * 32, smem, st>>>(P, fac, (uint32_t)wb);
  return cudaGetLastError();
}

cudaError_t launch_fx_pair(const FxApply& P, const KronPlan& K, const int2* fac, int shape,
                           cudaStream_t st) {
  bool real = false;
  if (!fx_pair_plan(K, &real)) return cudaErrorInvalidConfiguration;
  if (shape == 0) return real ? launch_fx_pair_t<kFxPairU[0], true>(P, fac, st)
                              : launch_fx_pair_t<kFxPairU[0], false>(P, fac, st);
  if (shape == 1) return real ? launch_fx_pair_t<kFxPairU[1], true>(P, fac, st)
                              : launch_fx_pair_t<kFxPairU[1], false>(P, fac, st);
  return cudaErrorInvalidConfiguration;
}

// Launch shapes the set-up autotuner chooses from: slots per pass RC,
// columns per load batch U, resident CTAs per SM asked of the compiler MB.
constexpr int kFxShapes = 4;
constexpr int kFxShapeRC[kFxShapes] = {1, 1, 1, 1};
constexpr int kFxShapeU[kFxShapes] = {8, 4, 6, 8};
constexpr int kFxShapeMB[kFxShapes] = {3, 4, 3, 4};

template <bool TR>
cudaError_t launch_fx(const FxApply& P, const int2* fac, int shape, unsigned grid, size_t smem,
                      cudaStream_t st) {
#define FX_CASE(k)                                                                            \
  case k:                                                                                     \
    return launch_fx_t<kFxShapeRC[k], kFxShapeU[k], kFxShapeMB[k], TR>(P, fac, grid, smem, st);
  switch (shape) {
    FX_CASE(0)
    FX_CASE(1)
    FX_CASE(2)
    FX_CASE(3)
    default: return cudaErrorInvalidConfiguration;
  }
#undef FX_CASE
}

}  // namespace

int fixed_shapes() { return kFxShapes + kFxStagedShapes + kFxPairShapes; }

int fixed_shape_kernel(int shape) {
  return shape < kFxShapes ? 8 : shape < kFxShapes + kFxStagedShapes ? 9 : 10;
}

bool fx_pair_plan(const KronPlan& K, bool* real) {
  // complex layout, the pair first: X, Y = 0, 1 with tasks (0, w1) (0, w2)
  // (1, w1) (1, w2), w1, w2 = 0, 1; then at most one real block (2, 2)
  if (K.layout != 1 || K.nblk < 1 || K.nblk > 2 || K.blk_kind[0] != 1 || K.blk_mat[0] != 0)
    return false;
  const bool r = K.nblk == 2;
  if (r && (K.blk_kind[1] != 0 || K.blk_mat[1] != 2)) return false;
  const int tm[5] = {0, 0, 1, 1, 2}, ts[5] = {0, 1, 0, 1, 2};
  if (K.nt != (r ? 5 : 4) || K.ns != (r ? 3 : 2) || K.nm != (r ? 3 : 2) || K.s != (r ? 3 : 2))
    return false;
  for (int t = 0; t < K.nt; ++t)
    if (K.task_mat[t] != tm[t] || K.task_src[t] != ts[t]) return false;
  *real = r;
  return true;
}

bool fixed_shape_fits(Ctx& C, Level& L, int shape) {
  if (shape < 0 || shape >= fixed_shapes()) return false;
  if (shape < kFxShapes) return true;
  if (shape >= kFxShapes + kFxStagedShapes) {  // paired: complex pair, interior stars of 39
    bool real;
    return L.kron_nmax == kFxN2 && fx_pair_plan(C.kplan, &real) &&
           (size_t)kFxWarps * std::max(fx_warp_bytes(C.s, std::max(C.kplan.ns, C.kplan.nt),
                                                     C.kplan.nt, L.kron_nmax),
                                       sizeof(FxPairSmem)) <= 227 * 1024;
  }
  FxStagedShape shp;
  return fx_staged_config(C.kplan, C.s, L.kron_nmax, shape - kFxShapes, &shp);
}

bool fixed_fits(Ctx& C, Level& L) {
  const KronPlan& K = C.kplan;
  return C.opt.patch_precision == 64 && L.kron && !L.kron_big && L.kron_nmax <= kFxMaxN &&
         (size_t)kFxWarps * fx_warp_bytes(C.s, K.ns > K.nt ? K.ns : K.nt, K.nt, L.kron_nmax) <=
             227 * 1024;
}

cudaError_t launch_patch_to_fixed(Ctx& C, Level& L) {
  const int64_t warps = L.nv * C.kplan.nm;
  k_patch_to_fixed<<<(unsigned)((warps + 7) / 8), 256, 0, C.stream>>>(
      C.kplan.nm, L.kron_nmax, L.nv, L.d_np, L.d_fac_off, L.d_order, (double*)L.d_fac, L.d_fexp,
      C.d_err);
  return cudaGetLastError();
}

FxApply fx_params(Ctx& C, Level& L, int colour, const double* r, double* out, double scale,
                  int transpose) {
  const KronPlan& K = C.kplan;
  FxApply P{};
  P.s = C.s;
  P.nsrc = transpose ? K.nt : K.ns;
  P.nt = K.nt;
  P.nm = K.nm;
  P.m = L.m;
  for (int i = 0; i < kKronMaxSrc * 3; ++i) P.G[i] = K.G[i];
  for (int i = 0; i < 3 * kKronMaxTasks; ++i) P.H[i] = K.H[i];
  for (int i = 0; i < kKronMaxTasks; ++i) {
    P.task_mat[i] = K.task_mat[i];
    P.task_src[i] = K.task_src[i];
  }
  P.np = L.d_np;
  P.fac_off = L.d_fac_off;
  P.fexp = L.d_fexp;
  P.r = r;
  P.out = out;
  P.scale = scale;
  if (colour < 0) {
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
  return P;
}

cudaError_t launch_vanka_kron_fx(Ctx& C, Level& L, int colour, const double* r, double* out,
                                 double scale, int transpose) {
  const KronPlan& K = C.kplan;
  const FxApply P = fx_params(C, L, colour, r, out, scale, transpose);
  if (P.count <= 0) return cudaSuccess;
  if (L.kron_shape >= kFxShapes + kFxStagedShapes && !transpose)  // paired kernel
    return launch_fx_pair(P, K, (const int2*)L.d_fac, L.kron_shape - kFxShapes - kFxStagedShapes,
                          C.stream);
  if (L.kron_shape >= kFxShapes && L.kron_shape < kFxShapes + kFxStagedShapes) {  // TMA-staged
    FxStagedShape shp;
    if (!fx_staged_config(K, C.s, L.kron_nmax, L.kron_shape - kFxShapes, &shp))
      return cudaErrorInvalidConfiguration;
    FxStaged S{};
    S.a = P;
    S.stages = shp.stages;
    S.stage_bytes = shp.stage_bytes;
    S.work_off = shp.work_off;
    S.spins = C.opt.timeout_spins > 0 ? C.opt.timeout_spins : (int64_t)1 << 26;
    S.err = C.d_err;
    int* cap = &L.fx_cap[L.kron_shape - kFxShapes][transpose ? 1 : 0];
    const int2* f = (const int2*)L.d_fac;
    return transpose ? launch_fx_staged<true>(S, f, shp, C.stream, cap)
                     : launch_fx_staged<false>(S, f, shp, C.stream, cap);
  }
  const size_t smem = (size_t)kFxWarps * fx_warp_bytes(P.s, K.ns > K.nt ? K.ns : K.nt, P.nt, P.nmax);
  const unsigned grid = (unsigned)((P.count + kFxWarps - 1) / kFxWarps);
  const int2* f = (const int2*)L.d_fac;
  // the transposed apply of a level tuned to the paired kernel: shape 3
  const int shape = L.kron_shape < kFxShapes ? L.kron_shape : 3;
  return transpose ? launch_fx<true>(P, f, shape, grid, smem, C.stream)
                   : launch_fx<false>(P, f, shape, grid, smem, C.stream);
}

}  // namespace irkmg

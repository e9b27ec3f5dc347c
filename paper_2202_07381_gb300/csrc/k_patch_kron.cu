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
  int64_t first, count;  // ordered-patch range of this colour
  int nmax;              // per-warp shared-memory stride
};

// Shared memory of one warp: residuals (s·nmax doubles), task results
// (nt·nmax doubles), sources (max(ns, nt)·nmax of T), indices (nmax int32).
__host__ __device__ inline size_t kron_warp_bytes(int s, int ns, int nt, int nmax, int tsize) {
  const int nsrc = ns > nt ? ns : nt;
  size_t b = (size_t)(s + nt) * nmax * 8 + (size_t)nsrc * nmax * tsize + (size_t)nmax * 4;
  return (b + 15) & ~(size_t)15;
}

template <typename T, int R, bool TR>
__global__ void __launch_bounds__(kKronWarps * 32) k_vanka_apply_kron(KronApply P,
                                                                      const T* __restrict__ fac) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kKronWarps + warp;
  if (w >= P.count) return;
  const int nmax = P.nmax;
  unsigned char* base = dyn + (size_t)warp * kron_warp_bytes(P.s, P.ns, P.nt, nmax, sizeof(T));
  double* s_r = reinterpret_cast<double*>(base);
  double* s_acc = s_r + P.s * nmax;
  T* s_src = reinterpret_cast<T*>(s_acc + P.nt * nmax);
  const int nsrc = TR ? P.nt : P.ns;
  int32_t* s_g = reinterpret_cast<int32_t*>(s_src + (P.ns > P.nt ? P.ns : P.nt) * nmax);

  const int64_t pi = P.first + w;
  const int n = P.np[pi];
  const int64_t nn = (int64_t)n * n;
  const T* X = fac + P.fac_off[pi];
  const int32_t* gidx = reinterpret_cast<const int32_t*>(
      reinterpret_cast<const unsigned char*>(X) +
      (((int64_t)P.nm * nn * (int64_t)sizeof(T) + 15) & ~(int64_t)15));
  for (int i = lane; i < n; i += 32) s_g[i] = gidx[i];
  __syncwarp();
  for (int idx = lane; idx < P.s * n; idx += 32) {
    const int t = idx / n, i = idx - t * n;
    s_r[idx] = P.r[t * P.m + s_g[i]];
  }
  __syncwarp();
  for (int idx = lane; idx < nsrc * n; idx += 32) {
    const int c = idx / n, i = idx - c * n;
    double a = 0.0;
    for (int t = 0; t < P.s; ++t)
      a += (TR ? P.H[t * kKronMaxTasks + c] : P.G[c * 3 + t]) * s_r[t * n + i];
    s_src[idx] = (T)a;
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
    if (ok[k]) s_acc[lane + 32 * k] = (double)acc[k];
  __syncwarp();
  for (int idx = lane; idx < P.s * n; idx += 32) {
    const int t = idx / n, i = idx - t * n;
    double x = 0.0;
    for (int tau = 0; tau < P.nt; ++tau) {
      const double h = TR ? P.G[P.task_src[tau] * 3 + t] : P.H[t * kKronMaxTasks + tau];
      x += h * s_acc[tau * n + i];
    }
    P.out[t * P.m + s_g[i]] += P.scale * x;
  }
}

int kron_max_slots() { return kKronMaxSlots; }

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
  KronApply P;
  P.s = C.s;
  P.ns = K.ns;
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
  P.r = r;
  P.out = out;
  P.scale = scale;
  P.first = L.colour_start[colour];
  P.count = L.colour_start[colour + 1] - P.first;
  P.nmax = L.kron_nmax;
  if (P.count <= 0) return cudaSuccess;
  const int prec = C.opt.patch_precision;
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
  return transpose ? launch_kron_t<float, true>(P, f, R, grid, smem, C.stream)
                   : launch_kron_t<float, false>(P, f, R, grid, smem, C.stream);
}

}  // namespace irkmg

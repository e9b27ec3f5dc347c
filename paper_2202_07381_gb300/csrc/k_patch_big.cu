// Vanka patches too large for one shared-memory inverse (3D: up to 392 DoFs
// for s = 2, Section 4.2 with all stages in every patch).
//
//   k_patch_lu_big: gather A_v = R_v J R_vᵀ from the assembled operators into
//     the patch's block (column-major, in place) and factor it,
//     P A_v = L U, by a blocked right-looking LU with partial pivoting:
//     32-column panels factored in shared memory, row interchanges applied to
//     the rest of the matrix, a triangular solve for the U block row, and the
//     trailing update A22 -= L21 U12 from shared-memory tiles.
//   k_patch_inv_from_lu: X = A_v⁻¹ = U⁻¹ L⁻¹ P, by blocked forward and
//     backward substitution on all n_p columns of P at once (32-row blocks:
//     a per-column triangular solve of the diagonal block, then a shared-
//     memory tiled update of the remaining rows), in a per-CTA workspace;
//     X then overwrites the factors, so every apply is one dense mat-vec.
//   k_vanka_apply_big: out[S_v] += scale · X r|_{S_v}, one CTA per patch,
//     threads over rows, columns streamed with coalesced loads.
//     One launch per colour.
// Block layout of a patch: [n_p^2 values (LU factors, then the inverse)]
// [n_p int32 DoF indices][n_p int32 pivots], each part padded to 16 bytes.
//
// FP32 patches take the trailing update A22 -= L21 U12 on the 5th-generation
// tensor cores (tcgen05.mma kind::tf32, one elected thread, operands staged in
// shared memory, a 128x64 FP32 accumulator in tensor memory, read back with
// tcgen05.ld).  TF32 keeps 10 mantissa bits, so each operand is split as
// x = hi + lo (hi = x with its 13 low mantissa bits cleared, lo = x - hi
// exactly) and D = Lhi Uhi + Lhi Ulo + Llo Uhi: three MMAs per K step give
// FP32-level products ("3xTF32").
#include <cfloat>
#include <type_traits>

#include "irkmg_internal.h"
#include "tma.cuh"

namespace irkmg {

constexpr int kBigThreads = 256;
constexpr int kPanel = 32;
constexpr int kUChunk = 128;

struct BigParams {
  int s, dim;
  int tc;      // FP32 LU: 1 = tcgen05 trailing updates, 0 = CUDA cores
  int max_np;  // largest patch of the level (sizes the shared-memory panel)
  double A[9];
  double dt;
  int64_t nf, m;
  const int32_t *patch_ptr, *patch_nodes, *order, *np;
  const int64_t* fac_off;
  const int32_t *vptr, *vcol;
  const double *M, *K;
  const int32_t *bptr, *bcol;
  const double *Bx, *By, *Bz;
  int* err;
  // apply
  const double* r;
  double* out;
  double scale;
  int64_t first, count;
};

__device__ __forceinline__ int big_csr_find(const int32_t* __restrict__ col, int32_t b, int32_t e,
                                            int32_t key) {
  while (b < e) {
    int32_t mid = (b + e) >> 1;
    if (col[mid] < key)
      b = mid + 1;
    else
      e = mid;
  }
  return b;
}

// ---- tcgen05 helpers (trailing update of the FP32 patch LU) ----------------
// Tiles of 128 x 64 (two CTAs of the LU fit an SM with their operands).
constexpr int kTcM = 128, kTcN = 64, kTcK = 32;
constexpr int kTcOperandBytes = (kTcM + kTcN) * kTcK * 4 * 2;  // A and B tiles, hi and lo
constexpr uint32_t kTcCols = kTcN;                               // TMEM columns of the accumulator

// Element offset of (row m, k) in the K-major, unswizzled canonical layout:
// 8-row x 16-byte core matrices, rows 16 B apart; core matrices adjacent in K
// 128 B apart (leading-dimension offset), 8-row groups 1024 B apart (stride
// offset), for a rows x 32 FP32 tile.
__device__ __forceinline__ int tc_off(int m, int k) {
  return (m >> 3) * 256 + (k >> 2) * 32 + (m & 7) * 4 + (k & 3);
}
// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset 128, stride-dimension byte offset 1024 (all >> 4), descriptor
// version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_alloc(uint32_t* dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(kTcCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols)
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

template <typename T>
__device__ __forceinline__ int64_t big_x_bytes(int np) {
  return ((int64_t)np * np * (int64_t)sizeof(T) + 15) & ~(int64_t)15;
}
__device__ __forceinline__ int64_t big_i_bytes(int np) { return ((int64_t)np * 4 + 15) & ~(int64_t)15; }

// Static shared scratch of one big-patch factorisation.
struct BigLuShared {
  double red_v[kBigThreads];
  int red_i[kBigThreads];
  int piv[kPanel];
  double inv[kPanel];      // 1 / pivot of each panel column (scaling deferred to the panel's end)
  float invf[kPanel];      // the same for FP32 patches
  float red_f[kBigThreads / 32];
  int perm[kMaxBigNp];     // net row permutation of a panel's interchanges
  int chg[2 * kPanel];     // rows it moves
  int nchg;
  int32_t nodes[96];
  double thr;
  uint64_t mbar;
  uint32_t taddr;
  int abort;
};

// Zeroes the column-major np x np matrix A and gathers I_s ⊗ M̃ + dt Am ⊗ K̃ of
// patch v into it (s stages, Am with row stride 3, np = s (D L + 1)); S.nodes
// holds the patch's L free nodes.  Sets S.thr = 1e3 eps max|A| (singular-pivot
// threshold).  All threads of the block.
template <typename T>
__device__ void big_gather(const BigParams& P, int s, const double* Am, int32_t v, int L, T* A,
                           int np, BigLuShared& S) {
  const int tid = threadIdx.x;
  const int D = P.dim;
  const int q = D * L + 1;
  for (int64_t i = tid; i < (int64_t)np * np; i += kBigThreads) A[i] = (T)0;
  __syncthreads();
  // ---- gather A_v (Section 3.1 Kronecker blocks) ----
  double mx = 0.0;
  const double* Bc[3] = {P.Bx, P.By, P.Bz};
  for (int idx = tid; idx < L * L; idx += kBigThreads) {
    const int a = idx / L, b = idx % L;
    const int32_t ra = S.nodes[a], cb = S.nodes[b];
    const int32_t p0 = P.vptr[ra], p1 = P.vptr[ra + 1];
    const int32_t pos = big_csr_find(P.vcol, p0, p1, cb);
    double mab = 0.0, kab = 0.0;
    if (pos < p1 && P.vcol[pos] == cb) {
      mab = P.M[pos];
      kab = P.K[pos];
    }
    for (int t = 0; t < s; ++t)
      for (int u = 0; u < s; ++u) {
        const double val = (t == u ? mab : 0.0) + P.dt * Am[t * 3 + u] * kab;
        mx = fmax(mx, fabs(val));
        for (int d = 0; d < D; ++d)
          A[(int64_t)(u * q + d * L + b) * np + (t * q + d * L + a)] = (T)val;
      }
  }
  for (int a = tid; a < L; a += kBigThreads) {
    const int32_t ra = S.nodes[a];
    const int32_t p0 = P.bptr[ra], p1 = P.bptr[ra + 1];
    const int32_t pos = big_csr_find(P.bcol, p0, p1, v);
    double bv[3] = {0.0, 0.0, 0.0};
    if (pos < p1 && P.bcol[pos] == v)
      for (int d = 0; d < D; ++d) bv[d] = Bc[d][pos];
    for (int t = 0; t < s; ++t)
      for (int u = 0; u < s; ++u) {
        const double f = P.dt * Am[t * 3 + u];
        for (int d = 0; d < D; ++d) {
          mx = fmax(mx, fabs(f * bv[d]));
          A[(int64_t)(u * q + D * L) * np + (t * q + d * L + a)] = (T)(f * bv[d]);
          A[(int64_t)(u * q + d * L + a) * np + (t * q + D * L)] = (T)(f * bv[d]);
        }
      }
  }
  S.red_v[tid] = mx;
  __syncthreads();
  for (int o = kBigThreads / 2; o > 0; o >>= 1) {
    if (tid < o) S.red_v[tid] = fmax(S.red_v[tid], S.red_v[tid + o]);
    __syncthreads();
  }
  if (tid == 0) S.thr = 1e3 * DBL_EPSILON * S.red_v[0];
  __syncthreads();
}

// Blocked right-looking LU with partial pivoting of the column-major np x np
// matrix A in place (pivots to piv), for patch v (error reports).  dyn holds
// the panel (kPanel x pmax rows) and, after it (1024-aligned), either the
// U12 chunk or the tcgen05 operand tiles.  With tc the trailing updates run on
// the tensor cores with the TMEM accumulator at S.taddr (big_tc_begin).
template <typename T>
__device__ void big_lu(const BigParams& P, int32_t v, T* A, int np, int32_t* piv, int pmax,
                       unsigned char* dyn, BigLuShared& S, bool tc, uint32_t& tc_phase) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t taddr = S.taddr;
  T* Pn = reinterpret_cast<T*>(dyn);               // panel, [kPanel][np - k0]
  T* Ub = Pn + (size_t)kPanel * np;                // U12 chunk, [kPanel][kUChunk]
  const size_t tc_base = (((size_t)kPanel * pmax * sizeof(T)) + 1023) & ~(size_t)1023;
  float* tA_hi = reinterpret_cast<float*>(dyn + tc_base);
  float* tA_lo = tA_hi + kTcM * kTcK;
  float* tB_hi = tA_lo + kTcM * kTcK;
  float* tB_lo = tB_hi + kTcN * kTcK;
  // ---- blocked LU with partial pivoting ----
  for (int k0 = 0; k0 < np && !S.abort; k0 += kPanel) {
    const int kb = min(kPanel, np - k0), prow = np - k0;
    for (int idx = tid; idx < prow * kb; idx += kBigThreads) {
      const int l = idx / prow, r = idx - l * prow;
      Pn[l * prow + r] = A[(int64_t)(k0 + l) * np + k0 + r];
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
      // pivot: the largest |entry| of column j at or below row j, the lowest
      // row among equals (a selection, so the reduction order does not
      // matter): per thread, per warp by shuffles, then over the warps
      // compared in the patch's precision: the FP64 pipe is scarce, and
      // widening a float to double is exact, so the order is the same
      T best = (T)-1;
      int bi = j;
      for (int r = j + tid; r < prow; r += kBigThreads) {
        const T a = fabs(Pn[j * prow + r]);
        if (a > best) {
          best = a;
          bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T a = __shfl_xor_sync(0xffffffffu, best, o);
        const int ia = __shfl_xor_sync(0xffffffffu, bi, o);
        if (a > best || (a == best && ia < bi)) {
          best = a;
          bi = ia;
        }
      }
      if (lane == 0) {
        if constexpr (sizeof(T) == 4)
          S.red_f[warp] = best;
        else
          S.red_v[warp] = best;
        S.red_i[warp] = bi;
      }
      __syncthreads();
      T pbest;
      if constexpr (sizeof(T) == 4)
        pbest = S.red_f[0];
      else
        pbest = S.red_v[0];
      int p = S.red_i[0];
      for (int x = 1; x < kBigThreads / 32; ++x) {
        T a;
        if constexpr (sizeof(T) == 4)
          a = S.red_f[x];
        else
          a = S.red_v[x];
        const int ia = S.red_i[x];
        if (a > pbest || (a == pbest && ia < p)) {
          pbest = a;
          p = ia;
        }
      }
      const double pabs = (double)pbest;
      if (tid == 0) {
        S.piv[j] = p;
        piv[k0 + j] = k0 + p;
        if (!(pabs > S.thr) && atomicCAS(&P.err[0], 0, IRKMG_ESINGULAR) == 0) P.err[1] = v;
      }
      if (p != j)
        for (int l = tid; l < kb; l += kBigThreads) {
          const T x = Pn[l * prow + j];
          Pn[l * prow + j] = Pn[l * prow + p];
          Pn[l * prow + p] = x;
        }
      __syncthreads();
      // rank-1 update of the panel's trailing columns with the multipliers
      // l_r = a_rj / a_jj; column j itself is scaled at the panel's end (later
      // steps only swap its rows, which commutes with the scaling)
      const T pv = Pn[j * prow + j];
      const T inv = pbest > (T)0 ? (T)1 / pv : (T)0;
      if (tid == 0) {
        if constexpr (sizeof(T) == 4)
          S.invf[j] = inv;
        else
          S.inv[j] = inv;
      }
      for (int r = j + 1 + tid; r < prow; r += kBigThreads) {
        const T lr = Pn[j * prow + r] * inv;
        for (int l = j + 1; l < kb; ++l) Pn[l * prow + r] -= lr * Pn[l * prow + j];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < prow * kb; idx += kBigThreads) {
      const int l = idx / prow, r = idx - l * prow;
      if (r > l) {
        if constexpr (sizeof(T) == 4)
          Pn[l * prow + r] *= S.invf[l];
        else
          Pn[l * prow + r] *= S.inv[l];
      }
    }
    // net permutation of the panel's row interchanges (thread 0), and the
    // rows it moves
    if (tid == 0) {
      for (int r = 0; r < prow; ++r) S.perm[r] = r;
      for (int j = 0; j < kb; ++j) {
        const int p = S.piv[j], x = S.perm[j];
        S.perm[j] = S.perm[p];
        S.perm[p] = x;
      }
      int c = 0;
      for (int r = 0; r < prow; ++r)
        if (S.perm[r] != r) S.chg[c++] = r;
      S.nchg = c;
    }
    __syncthreads();
    for (int idx = tid; idx < prow * kb; idx += kBigThreads) {
      const int l = idx / prow, r = idx - l * prow;
      A[(int64_t)(k0 + l) * np + k0 + r] = Pn[l * prow + r];
    }
    // the interchanges applied to every other column: one warp per column,
    // all moved rows read, then written (row r takes old row perm[r])
    {
      const int nchg = S.nchg;
      for (int c = warp; c < np; c += kBigThreads / 32) {
        if (c >= k0 && c < k0 + kb) continue;
        T* col = A + (int64_t)c * np + k0;
        T x0 = (T)0, x1 = (T)0;
        if (lane < nchg) x0 = col[S.perm[S.chg[lane]]];
        if (lane + 32 < nchg) x1 = col[S.perm[S.chg[lane + 32]]];
        __syncwarp();
        if (lane < nchg) col[S.chg[lane]] = x0;
        if (lane + 32 < nchg) col[S.chg[lane + 32]] = x1;
      }
    }
    __syncthreads();
    // U12 = L11^{-1} A12 (unit lower L11 from the panel)
    const int ncol = np - k0 - kb;
    for (int c = tid; c < ncol; c += kBigThreads) {
      T* col = A + (int64_t)(k0 + kb + c) * np + k0;
      T x[kPanel];
#pragma unroll
      for (int l = 0; l < kPanel; ++l) x[l] = l < kb ? col[l] : (T)0;
#pragma unroll
      for (int l = 0; l < kPanel; ++l)
#pragma unroll
        for (int i = 0; i < kPanel; ++i)
          if (i > l && i < kb) x[i] -= Pn[l * prow + i] * x[l];
#pragma unroll
      for (int l = 0; l < kPanel; ++l)
        if (l < kb) col[l] = x[l];
    }
    __syncthreads();
    // A22 -= L21 U12
    const int mrow = prow - kb;
    if (tc) {
      // 128 x 64 tiles on the tensor cores: D = L21 U12 in TMEM (3xTF32),
      // then every thread subtracts its row of D from A22 in global memory
      for (int r0 = 0; r0 < mrow && !S.abort; r0 += kTcM)
        for (int c0 = 0; c0 < ncol && !S.abort; c0 += kTcN) {
          for (int idx = tid; idx < kTcM * kTcK; idx += kBigThreads) {
            const int k = idx / kTcM, m = idx - k * kTcM;
            const float x = (k < kb && r0 + m < mrow) ? (float)Pn[k * prow + kb + r0 + m] : 0.f;
            const float h = tf32_hi(x);
            tA_hi[tc_off(m, k)] = h;
            tA_lo[tc_off(m, k)] = x - h;
          }
          for (int idx = tid; idx < kTcN * kTcK; idx += kBigThreads) {
            const int n = idx / kTcK, k = idx - n * kTcK;
            const float x = (k < kb && c0 + n < ncol)
                                ? (float)A[(int64_t)(k0 + kb + c0 + n) * np + k0 + k]
                                : 0.f;
            const float h = tf32_hi(x);
            tB_hi[tc_off(n, k)] = h;
            tB_lo[tc_off(n, k)] = x - h;
          }
          fence_proxy_async();  // generic-proxy writes visible to the tensor core
          __syncthreads();
          if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(tA_hi), al = smem_u32(tA_lo);
            const uint32_t bh = smem_u32(tB_hi), bl = smem_u32(tB_lo);
#pragma unroll
            for (int ks = 0; ks < kTcK / 8; ++ks) {  // K = 8 per MMA: two core matrices
              const uint32_t o = ks * 256;
              tc_mma(taddr, tc_desc(ah + o), tc_desc(bh + o), ks > 0 ? 1u : 0u);
              tc_mma(taddr, tc_desc(ah + o), tc_desc(bl + o), 1u);
              tc_mma(taddr, tc_desc(al + o), tc_desc(bh + o), 1u);
            }
            tc_commit(&S.mbar);
          }
          if (!mbar_wait_bounded(&S.mbar, tc_phase, (int64_t)1 << 26)) {
            S.abort = 1;
            atomicCAS(&P.err[0], 0, IRKMG_ETIMEOUT);
          }
          tc_phase ^= 1u;
          __syncthreads();
          if (S.abort) {
            // the MMAs may still be in flight: one more bounded wait before
            // the tensor memory is released below
            mbar_wait_bounded(&S.mbar, tc_phase ^ 1u, (int64_t)1 << 26);
            break;
          }
          tc_fence_after();
          // warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows) and half
          // w / 4 of the tile's columns
          const int q = warp & 3, row = q * 32 + lane;
          const bool row_ok = r0 + row < mrow;
#pragma unroll 1
          for (int cc = 0; cc < kTcN / 32; ++cc) {
            const int col0 = (warp >> 2) * (kTcN / 2) + cc * 16;
            float v[16];
            tc_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = c0 + col0 + j;
              if (row_ok && c < ncol) A[(int64_t)(k0 + kb + c) * np + k0 + kb + r0 + row] -= (T)v[j];
            }
          }
          tc_fence_before();
          __syncthreads();  // TMEM and the operand tiles are reused by the next tile
        }
      __syncthreads();
      continue;
    }
    for (int cc0 = 0; cc0 < ncol; cc0 += kUChunk) {
      const int cw = min(kUChunk, ncol - cc0);
      for (int idx = tid; idx < kb * cw; idx += kBigThreads) {
        const int l = idx % kb, c = idx / kb;
        Ub[l * kUChunk + c] = A[(int64_t)(k0 + kb + cc0 + c) * np + k0 + l];
      }
      __syncthreads();
      for (int idx = tid; idx < mrow * cw; idx += kBigThreads) {
        const int i = idx % mrow, c = idx / mrow;
        T* a = A + (int64_t)(k0 + kb + cc0 + c) * np + k0 + kb + i;
        T acc = *a;
        for (int l = 0; l < kb; ++l) acc -= Pn[l * prow + kb + i] * Ub[l * kUChunk + c];
        *a = acc;
      }
      __syncthreads();
    }
  }
}

// TMEM for the tcgen05 trailing updates: warp 0 allocates kTcCols columns,
// thread 0 initialises the completion mbarrier.  All threads of the block.
__device__ void big_tc_begin(BigLuShared& S, bool tc) {
  const int tid = threadIdx.x;
  if (tid == 0) S.abort = 0;
  if (tc) {
    if (tid < 32) tc_alloc(&S.taddr);
    if (tid == 0) {
      mbar_init(&S.mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
  }
  __syncthreads();
  if (tc) tc_fence_after();
}

__device__ void big_tc_end(BigLuShared& S, bool tc) {
  if (!tc) return;
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tc_dealloc(S.taddr);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBigThreads) k_patch_lu_big(BigParams P, int64_t npatch, T* fac) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  __shared__ BigLuShared S;
  const int64_t pi = blockIdx.x;
  if (pi >= npatch) return;
  const int tid = threadIdx.x;
  const int32_t v = P.order[pi];
  const int32_t nb = P.patch_ptr[v], L = P.patch_ptr[v + 1] - nb;
  const int np = P.s * (P.dim * L + 1);
  T* A = fac + P.fac_off[pi];  // column-major: A[c * np + r]
  int32_t* piv = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(A) + big_x_bytes<T>(np) +
                                            big_i_bytes(np));
  const bool tc = std::is_same<T, float>::value && P.tc != 0;
  for (int i = tid; i < L; i += kBigThreads) S.nodes[i] = P.patch_nodes[nb + i];
  big_gather<T>(P, P.s, P.A, v, L, A, np, S);
  big_tc_begin(S, tc);
  uint32_t tc_phase = 0;
  big_lu<T>(P, v, A, np, piv, P.max_np, dyn, S, tc, tc_phase);
  big_tc_end(S, tc);
}


constexpr int kRowChunk = 128;

// Work on W (column-major np x ncols): W := L⁻¹ W (lower = true, unit
// diagonal) or W := U⁻¹ W (lower = false), with L / U the factors stored in A.
// Wb holds kPanel x ncols, Ms kPanel x kRowChunk, Ls kPanel x kPanel.
template <typename T>
__device__ void block_trsm(const T* __restrict__ A, T* W, int np, int ncols, bool lower, T* Ls,
                           T* Wb, T* Ms) {
  const int tid = threadIdx.x;
  const int nblk = (np + kPanel - 1) / kPanel;
  for (int bb = 0; bb < nblk; ++bb) {
    const int blk = lower ? bb : nblk - 1 - bb;
    const int k0 = blk * kPanel, kb = min(kPanel, np - k0);
    for (int idx = tid; idx < kb * kb; idx += kBigThreads) {
      const int l = idx / kb, i = idx % kb;
      Ls[l * kPanel + i] = A[(int64_t)(k0 + l) * np + k0 + i];
    }
    __syncthreads();
    // diagonal block: every column solved by one thread
    for (int c = tid; c < ncols; c += kBigThreads) {
      T* col = W + (int64_t)c * np + k0;
      T x[kPanel];
#pragma unroll
      for (int l = 0; l < kPanel; ++l) x[l] = l < kb ? col[l] : (T)0;
      if (lower) {
#pragma unroll
        for (int l = 0; l < kPanel; ++l)
#pragma unroll
          for (int i = 0; i < kPanel; ++i)
            if (i > l && i < kb) x[i] -= Ls[l * kPanel + i] * x[l];
      } else {
#pragma unroll
        for (int l = kPanel - 1; l >= 0; --l) {
          if (l < kb) x[l] = x[l] / Ls[l * kPanel + l];
#pragma unroll
          for (int i = 0; i < kPanel; ++i)
            if (i < l && l < kb) x[i] -= Ls[l * kPanel + i] * x[l];
        }
      }
#pragma unroll
      for (int l = 0; l < kPanel; ++l)
        if (l < kb) {
          col[l] = x[l];
          Wb[l * ncols + c] = x[l];
        }
    }
    __syncthreads();
    // remaining rows: W[r, :] -= A[r, k0:k0+kb] W[k0:k0+kb, :], rows below the
    // block for L, above it for U, in chunks of kRowChunk rows
    const int r0 = lower ? k0 + kb : 0, r1 = lower ? np : k0;
    for (int ch = r0; ch < r1; ch += kRowChunk) {
      const int mr = min(kRowChunk, r1 - ch);
      for (int idx = tid; idx < kb * mr; idx += kBigThreads) {
        const int l = idx / mr, i = idx % mr;
        Ms[l * kRowChunk + i] = A[(int64_t)(k0 + l) * np + ch + i];
      }
      __syncthreads();
      for (int idx = tid; idx < mr * ncols; idx += kBigThreads) {
        const int i = idx % mr, c = idx / mr;
        T* w = W + (int64_t)c * np + ch + i;
        T acc = *w;
        for (int l = 0; l < kb; ++l) acc -= Ms[l * kRowChunk + i] * Wb[l * ncols + c];
        *w = acc;
      }
      __syncthreads();
    }
  }
}

// Persistent: CTA b inverts patches b, b + gridDim.x, ...; its workspace is
// work + b * ws (ws >= np^2 for every patch of the level).
template <typename T>
__global__ void __launch_bounds__(kBigThreads) k_patch_inv_from_lu(BigParams P, int64_t npatch,
                                                                  T* fac, T* work, int64_t ws) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  __shared__ int32_t perm[kMaxBigNp];
  T* W = work + (int64_t)blockIdx.x * ws;
  const int tid = threadIdx.x;
  for (int64_t pi = blockIdx.x; pi < npatch; pi += gridDim.x) {
    const int np = P.np[pi];
    T* A = fac + P.fac_off[pi];
    const int32_t* piv = reinterpret_cast<const int32_t*>(
        reinterpret_cast<const unsigned char*>(A) + big_x_bytes<T>(np) + big_i_bytes(np));
    T* Ls = reinterpret_cast<T*>(dyn);                 // [kPanel][kPanel]
    T* Wb = Ls + kPanel * kPanel;                      // [kPanel][np]
    T* Ms = Wb + (size_t)kPanel * np;                  // [kPanel][kRowChunk]
    if (tid == 0) {
      for (int i = 0; i < np; ++i) perm[i] = i;
      for (int j = 0; j < np; ++j) {
        const int p = piv[j];
        if (p != j) {
          const int32_t x = perm[j];
          perm[j] = perm[p];
          perm[p] = x;
        }
      }
    }
    __syncthreads();
    // W = P (row i of P is e_{perm[i]})
    for (int64_t idx = tid; idx < (int64_t)np * np; idx += kBigThreads) {
      const int c = (int)(idx / np), r = (int)(idx % np);
      W[idx] = perm[r] == c ? (T)1 : (T)0;
    }
    __syncthreads();
    block_trsm<T>(A, W, np, np, true, Ls, Wb, Ms);
    block_trsm<T>(A, W, np, np, false, Ls, Wb, Ms);
    for (int64_t idx = tid; idx < (int64_t)np * np; idx += kBigThreads) A[idx] = W[idx];
    __syncthreads();
  }
}

// Decoupled factors of large patches (persistent: CTA b takes patches b,
// b + gridDim.x, ...).  For each block of the real block diagonalisation of A
// (one real eigenvalue, or a pair as [[α, β], [−β, α]]) the block system
// I ⊗ M̃ + dt D_b ⊗ K̃ (q·n DoFs) is gathered into the CTA's workspace, factored
// by the blocked LU, and the first n columns of its inverse are formed by the
// blocked triangular solves; they give the block's stored matrices (real: the
// inverse; pair: X, Y of its first block column, or X + Y, X, Y), written into
// the patch block like the shared-memory kernel does.  Workspace per CTA:
// pmax² (factors) + pmax·nmax (inverse columns) + pmax int32 (pivots).
template <typename T>
__global__ void __launch_bounds__(kBigThreads) k_patch_factor_kron_big(BigParams P, KronPlan K,
                                                                      int64_t npatch, T* fac, T* work,
                                                                      int64_t ws, int pmax, int nmax) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  __shared__ BigLuShared S;
  __shared__ int32_t perm[kMaxBigNp];
  const int tid = threadIdx.x;
  const bool tc = std::is_same<T, float>::value && P.tc != 0;
  big_tc_begin(S, tc);
  uint32_t tc_phase = 0;
  T* Wa = work + (int64_t)blockIdx.x * ws;
  T* W = Wa + (int64_t)pmax * pmax;
  int32_t* piv = reinterpret_cast<int32_t*>(W + (int64_t)pmax * nmax);
  T* Ls = reinterpret_cast<T*>(dyn);                 // [kPanel][kPanel]
  T* Wb = Ls + kPanel * kPanel;                      // [kPanel][nmax]
  T* Ms = Wb + (size_t)kPanel * nmax;                // [kPanel][kRowChunk]
  for (int64_t pi = blockIdx.x; pi < npatch && !S.abort; pi += gridDim.x) {
    const int32_t v = P.order[pi];
    const int32_t nb = P.patch_ptr[v], L = P.patch_ptr[v + 1] - nb;
    const int n = P.dim * L + 1;
    const int64_t nn = (int64_t)n * n;
    for (int i = tid; i < L; i += kBigThreads) S.nodes[i] = P.patch_nodes[nb + i];
    __syncthreads();
    T* base = fac + P.fac_off[pi];
    for (int b = 0; b < K.nblk && !S.abort; ++b) {
      const int q = K.blk_size[b], nq = q * n;
      double Am[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) Am[i * 3 + j] = K.blk[b][i * q + j];
      big_gather<T>(P, q, Am, v, L, Wa, nq, S);
      big_lu<T>(P, v, Wa, nq, piv, pmax, dyn, S, tc, tc_phase);
      __syncthreads();
      if (S.abort) break;
      // W = first n columns of the row-permuted identity: row r of P is e_perm[r]
      if (tid == 0) {
        for (int i = 0; i < nq; ++i) perm[i] = i;
        for (int j = 0; j < nq; ++j) {
          const int p = piv[j];
          if (p != j) {
            const int32_t x = perm[j];
            perm[j] = perm[p];
            perm[p] = x;
          }
        }
      }
      __syncthreads();
      for (int64_t idx = tid; idx < (int64_t)nq * n; idx += kBigThreads) {
        const int c = (int)(idx / nq), r = (int)(idx % nq);
        W[idx] = perm[r] == c ? (T)1 : (T)0;
      }
      __syncthreads();
      block_trsm<T>(Wa, W, nq, n, true, Ls, Wb, Ms);
      block_trsm<T>(Wa, W, nq, n, false, Ls, Wb, Ms);
      T* X = base + (int64_t)K.blk_mat[b] * nn;
      for (int64_t idx = tid; idx < nn; idx += kBigThreads) {
        const int c = (int)(idx / n), r = (int)(idx % n);  // column-major (r, c)
        const T x = W[(int64_t)c * nq + r];
        if (K.blk_kind[b] == 0) {
          X[idx] = x;
        } else {
          const T y = W[(int64_t)c * nq + n + r];
          if (K.blk_kind[b] == 1) {
            X[idx] = x;
            X[nn + idx] = y;
          } else {
            X[idx] = x + y;
            X[nn + idx] = x;
            X[2 * nn + idx] = y;
          }
        }
      }
      __syncthreads();
    }
  }
  big_tc_end(S, tc);
}

// out[S_v] += scale · X r|_{S_v} for large patches: one CTA per patch, thread t
// owns rows t and t + 256, columns streamed with coalesced loads.
template <typename T>
__global__ void __launch_bounds__(kBigThreads) k_vanka_apply_big(BigParams P, const T* __restrict__ fac) {
  __shared__ T y[kMaxBigNp];
  __shared__ int32_t g[kMaxBigNp];
  const int64_t w = blockIdx.x;
  if (w >= P.count) return;
  const int tid = threadIdx.x;
  const int64_t pi = P.first + w;
  const int np = P.np[pi];
  const T* X = fac + P.fac_off[pi];
  const int32_t* G = reinterpret_cast<const int32_t*>(reinterpret_cast<const unsigned char*>(X) +
                                                      big_x_bytes<T>(np));
  for (int i = tid; i < np; i += kBigThreads) {
    const int32_t gi = G[i];
    g[i] = gi;
    y[i] = (T)P.r[gi];
  }
  __syncthreads();
  // loads of kBatch columns are issued before their FMAs, so every thread
  // keeps kBatch (or 2 kBatch) independent loads in flight
  constexpr int kBatch = 8;
  const int i0 = tid, i1 = tid + kBigThreads;
  const bool has0 = i0 < np, has1 = i1 < np;
  T a0 = (T)0, b0 = (T)0, a1 = (T)0, b1 = (T)0;
  if (has0) {
    const T* x0 = X + i0;
    const T* x1 = X + (has1 ? i1 : i0);
    int j = 0;
    for (; j + kBatch <= np; j += kBatch) {
      T v0[kBatch], v1[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        v0[u] = __ldg(x0 + (int64_t)(j + u) * np);
        if (has1) v1[u] = __ldg(x1 + (int64_t)(j + u) * np);
      }
#pragma unroll
      for (int u = 0; u < kBatch; u += 2) {
        a0 = fma(v0[u], y[j + u], a0);
        b0 = fma(v0[u + 1], y[j + u + 1], b0);
        if (has1) {
          a1 = fma(v1[u], y[j + u], a1);
          b1 = fma(v1[u + 1], y[j + u + 1], b1);
        }
      }
    }
    for (; j < np; ++j) {
      a0 = fma(__ldg(x0 + (int64_t)j * np), y[j], a0);
      if (has1) a1 = fma(__ldg(x1 + (int64_t)j * np), y[j], a1);
    }
  }
  if (i0 < np) P.out[g[i0]] += P.scale * (double)(a0 + b0);
  if (i1 < np) P.out[g[i1]] += P.scale * (double)(a1 + b1);
}

static BigParams big_params(Ctx& C, Level& L) {
  BigParams P{};
  P.s = C.s;
  P.dim = L.dim;
  P.tc = C.opt.patch_lu_tc;
  P.max_np = L.max_np;
  for (int i = 0; i < 9; ++i) P.A[i] = 0.0;
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j) P.A[i * 3 + j] = C.A[i * C.s + j];
  P.dt = C.dt;
  P.nf = L.nf;
  P.m = L.m;
  P.patch_ptr = L.d_patch_ptr;
  P.patch_nodes = L.d_patch_nodes;
  P.order = L.d_order;
  P.np = L.d_np;
  P.fac_off = L.d_fac_off;
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.M = L.vel.v[0];
  P.K = L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.Bz = L.b.v[2];
  P.err = C.d_err;
  P.r = nullptr;
  P.out = nullptr;
  P.scale = 0.0;
  P.first = P.count = 0;
  return P;
}

// Shared memory of the LU: the panel (kPanel x max_np) and either the U12
// chunk (CUDA-core update) or the four tcgen05 operand tiles, 1024-aligned.
cudaError_t launch_patch_lu_big(Ctx& C, Level& L) {
  BigParams P = big_params(C, L);
  if (C.opt.patch_precision == 64) {
    const size_t smem = (size_t)kPanel * (L.max_np + kUChunk) * sizeof(double);
    cudaFuncSetAttribute(k_patch_lu_big<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_lu_big<double><<<(unsigned)L.nv, kBigThreads, smem, C.stream>>>(P, L.nv,
                                                                            (double*)L.d_fac);
  } else {
    size_t smem = (size_t)kPanel * (L.max_np + kUChunk) * sizeof(float);
    if (P.tc)
      smem = (((size_t)kPanel * L.max_np * sizeof(float) + 1023) & ~(size_t)1023) +
             (size_t)kTcOperandBytes;
    cudaFuncSetAttribute(k_patch_lu_big<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_lu_big<float><<<(unsigned)L.nv, kBigThreads, smem, C.stream>>>(P, L.nv,
                                                                           (float*)L.d_fac);
  }
  return cudaGetLastError();
}

cudaError_t launch_patch_inv_from_lu(Ctx& C, Level& L, void* work, int64_t ws, int ctas) {
  BigParams P = big_params(C, L);
  const int np = L.max_np;
  if (C.opt.patch_precision == 64) {
    const size_t smem = (size_t)(kPanel * kPanel + kPanel * np + kPanel * kRowChunk) * sizeof(double);
    cudaFuncSetAttribute(k_patch_inv_from_lu<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_inv_from_lu<double><<<(unsigned)ctas, kBigThreads, smem, C.stream>>>(
        P, L.nv, (double*)L.d_fac, (double*)work, ws);
  } else {
    const size_t smem = (size_t)(kPanel * kPanel + kPanel * np + kPanel * kRowChunk) * sizeof(float);
    cudaFuncSetAttribute(k_patch_inv_from_lu<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_inv_from_lu<float><<<(unsigned)ctas, kBigThreads, smem, C.stream>>>(
        P, L.nv, (float*)L.d_fac, (float*)work, ws);
  }
  return cudaGetLastError();
}

// Shared memory of the decoupled factorisation: the larger of the LU's needs
// (panel of pmax rows, then the U12 chunk or the tcgen05 tiles) and the
// triangular solves' (Ls, Wb, Ms).
static size_t kron_big_smem(int pmax, int nmax, size_t w, bool tc) {
  size_t lu = (size_t)kPanel * pmax * w;
  lu = tc ? ((lu + 1023) & ~(size_t)1023) + (size_t)kTcOperandBytes : lu + (size_t)kPanel * kUChunk * w;
  const size_t tr = (size_t)(kPanel * kPanel + kPanel * nmax + kPanel * kRowChunk) * w;
  return lu > tr ? lu : tr;
}

int64_t kron_big_workspace(int pmax, int nmax, int prec) {
  const int64_t w = prec == 64 ? 8 : 4;
  return (int64_t)pmax * pmax + (int64_t)pmax * nmax + ((int64_t)pmax * 4 + w - 1) / w;
}

cudaError_t launch_patch_factor_kron_big(Ctx& C, Level& L, void* work, int64_t ws, int ctas) {
  BigParams P = big_params(C, L);
  int q = 1;
  for (int b = 0; b < C.kplan.nblk; ++b) q = q > C.kplan.blk_size[b] ? q : C.kplan.blk_size[b];
  const int nmax = L.kron_nmax, pmax = q * nmax;
  if (C.opt.patch_precision == 64) {
    const size_t smem = kron_big_smem(pmax, nmax, 8, false);
    cudaFuncSetAttribute(k_patch_factor_kron_big<double>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_patch_factor_kron_big<double><<<(unsigned)ctas, kBigThreads, smem, C.stream>>>(
        P, C.kplan, L.nv, (double*)L.d_fac, (double*)work, ws, pmax, nmax);
  } else {
    const size_t smem = kron_big_smem(pmax, nmax, 4, P.tc != 0);
    cudaFuncSetAttribute(k_patch_factor_kron_big<float>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_patch_factor_kron_big<float><<<(unsigned)ctas, kBigThreads, smem, C.stream>>>(
        P, C.kplan, L.nv, (float*)L.d_fac, (float*)work, ws, pmax, nmax);
  }
  return cudaGetLastError();
}

cudaError_t launch_vanka_big(Ctx& C, Level& L, int colour, const double* r, double* out,
                             double scale) {
  BigParams P = big_params(C, L);
  P.r = r;
  P.out = out;
  P.scale = scale;
  P.first = L.colour_start[colour];
  P.count = L.colour_start[colour + 1] - P.first;
  if (P.count <= 0) return cudaSuccess;
  if (C.opt.patch_precision == 64)
    k_vanka_apply_big<double><<<(unsigned)P.count, kBigThreads, 0, C.stream>>>(
        P, (const double*)L.d_fac);
  else
    k_vanka_apply_big<float><<<(unsigned)P.count, kBigThreads, 0, C.stream>>>(
        P, (const float*)L.d_fac);
  return cudaGetLastError();
}

}  // namespace irkmg

// Exact fixed-point stage operator (Section 3.1: the residual r = F - J k of
// J = I_s ⊗ [[M,0],[0,0]] + dt A ⊗ [[K,B],[Bᵀ,0]]) for 2D levels, the
// non-transposed Stokes / Oseen operator.
//
// GB300 retires 2 FP64 FMAs per clock per SM: the FP64 operator (12 FMAs per
// stored velocity entry for s = 3) is bound by the FP64 pipe at a fifth of
// HBM bandwidth.  Here every stored row of M, K, B_x, B_y (velocity rows) and
// of Bᵀ (pressure rows, both components under one exponent) is kept as
// 57-bit fixed point with its own power of two,
//     A_rj = q_rj 2^(E_r − 57),   |q_rj| ≤ 2^57,
// and one application runs in three launches:
//   1. the largest |x| of every (stage, velocity / pressure) block;
//   2. x_t,j = v_t,j 2^(F_g − 58) as two 29-bit limbs, one exponent F_g per
//      group g (velocity or pressure, the largest over the stages);
//   3. a thread per (velocity row, component c) forms, for every stage t,
//      the exact sums M x_t,c, K x_t,c and B^c p_t (32 × 32 → 64-bit
//      multiply-adds into three 64-bit accumulators), each rounded once to
//      FP64, and applies the stage mixing in FP64 as the FP64 operator does:
//      y_i,c = (M x_i,c) + Σ_t (dt a_it) (K x_t,c + B^c p_t);  a thread per
//      pressure row forms Bᵀ_v u_t exactly for every stage and mixes likewise.
//      r = F − y.
// The errors are the conversions (2^−57 of a row's largest entry, 2^−58 of a
// group's largest |x|), one rounding per product sum and the FP64 mixing; an
// FP64 dot product instead rounds every partial sum.  A non-finite entry
// anywhere in x makes every output NaN.
#include <algorithm>
#include <climits>
#include <cmath>

#include "fx_math.h"
#include "fx_patch.cuh"
#include "irkmg_internal.h"

namespace irkmg {

namespace {

constexpr int kOpThreads = 256;

// Row r of a SELL matrix (ncomp value arrays sharing the row exponent): E_r
// with every |a_rj| < 2^E_r, the entries as (a0, a1) limbs of
// round(a 2^(57 − E_r)).  A non-finite entry reports IRKMG_ESINGULAR.
__global__ void k_sell_to_fixed(int64_t nrows, const int64_t* __restrict__ ptr, int ncomp,
                                const double* __restrict__ v0, const double* __restrict__ v1,
                                int2* __restrict__ q0, int2* __restrict__ q1,
                                int16_t* __restrict__ ex, int* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int64_t sl = r >> 5, lane = r & 31;
  const int64_t b0 = ptr[sl], b1 = ptr[sl + 1];
  double mx = 0.0;
  bool finite = true;
  for (int64_t e = b0 + lane; e < b1; e += 32) {
    const double a = v0[e];
    finite = finite && isfinite(a);
    mx = fmax(mx, fabs(a));
    if (ncomp > 1) {
      const double b = v1[e];
      finite = finite && isfinite(b);
      mx = fmax(mx, fabs(b));
    }
  }
  int E = 0;
  if (!finite) {
    if (atomicCAS(&err[0], 0, IRKMG_ESINGULAR) == 0) err[1] = (int)r;
  } else if (mx > 0.0) {
    frexp(mx, &E);
  }
  ex[r] = (int16_t)E;
  for (int64_t e = b0 + lane; e < b1; e += 32) {
    int32_t a1, a0;
    fx_split29(finite ? fx_scale_round(v0[e], 57 - E) : 0, &a1, &a0);
    q0[e] = make_int2(a0, a1);
    if (ncomp > 1) {
      fx_split29(finite ? fx_scale_round(v1[e], 57 - E) : 0, &a1, &a0);
      q1[e] = make_int2(a0, a1);
    }
  }
}

// 1. Largest |x| of every (stage t, group g) block as a bit pattern (bmax
// zeroed before): g = 0 on the velocity entries [0, nu) of a stage, 1 on
// the pressure entries.
template <int S>
__global__ void __launch_bounds__(kOpThreads) k_block_absmax(const double* __restrict__ x,
                                                             int64_t m, int64_t nu,
                                                             unsigned long long* bmax) {
  unsigned long long mx[2 * S];
#pragma unroll
  for (int k = 0; k < 2 * S; ++k) mx[k] = 0;
  const int64_t n = S * m;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = id / m, j = id - t * m;
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(x[id]) & 0x7fffffffffffffffull;
    const int k = 2 * (int)t + (j < nu ? 0 : 1);
#pragma unroll
    for (int q = 0; q < 2 * S; ++q)
      if (q == k) mx[q] = max(mx[q], b);
  }
  __shared__ unsigned long long s_mx[2 * S];
  if (threadIdx.x < 2 * S) s_mx[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2 * S; ++q) {
    unsigned long long v = mx[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v != 0) atomicMax(&s_mx[q], v);
  }
  __syncthreads();
  if (threadIdx.x < 2 * S && s_mx[threadIdx.x] != 0) atomicMax(&bmax[threadIdx.x], s_mx[threadIdx.x]);
}

// The 58-convention exponent of x in group g from the block maxima: INT_MIN
// when a block holds a non-finite value.
template <int S>
__device__ __forceinline__ int group_exponent(const unsigned long long* bmax, int g) {
  unsigned long long mb = 0;
#pragma unroll
  for (int t = 0; t < S; ++t) mb = max(mb, bmax[2 * t + g]);
  if (mb >= 0x7ff0000000000000ull) return INT_MIN;
  return mb ? fx_exponent(fx_from_bits(mb)) : 0;
}

// 2. x as 58-bit limbs (the layout of x).
template <int S>
__global__ void __launch_bounds__(kOpThreads) k_op_convert(const double* __restrict__ x,
                                                           int64_t m, int64_t nu,
                                                           const unsigned long long* __restrict__ bmax,
                                                           int2* __restrict__ xl) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= S * m) return;
  const int64_t t = id / m, j = id - t * m;
  const int F = group_exponent<S>(bmax, j < nu ? 0 : 1);
  int32_t v1, v0;
  fx_split29(F == INT_MIN ? 0 : fx_scale_round(x[id], 58 - F), &v1, &v0);
  xl[id] = make_int2(v0, v1);
}

struct OpFx {
  int64_t nf, nv, m, nf_pad;
  const int64_t *svp, *sbp, *sbtp;
  const int32_t *svc, *sbc, *sbtc;
  const int2 *qM, *qK, *qB0, *qB1, *qT0, *qT1;
  const int16_t *eM, *eK, *eB0, *eB1, *eT;
  double mix[9];  // dt a_it, row-major 3 × 3
};

// Three 64-bit accumulators per exact product sum: high × high, the two
// mixed products together (each at most 1.5·2^57 in magnitude, so a row of
// up to kOpMaxRow products cannot overflow), low × low.
constexpr int kOpMaxRow = 42;
__device__ __forceinline__ void fx_mac3(int64_t (&a)[3], int2 q, int2 v) {
  a[0] = mad_wide(q.y, v.y, a[0]);
  a[1] = mad_wide(q.y, v.x, a[1]);
  a[1] = mad_wide(q.x, v.y, a[1]);
  a[2] = mad_wide(q.x, v.x, a[2]);
}
__device__ __forceinline__ double fx_round3(const int64_t (&a)[3], int e) {
  const int64_t b[4] = {a[0], a[1], 0, a[2]};
  return fx_round(b, e);
}

// 3. The operator: threads [0, 2 nf_pad) take (velocity row, component),
// the two warps of a SELL slice next to each other (components 0, 1) so that
// the second reads the slice's matrix entries from L1; the rest pressure
// rows.  r = F − J x, or r = J x when F is null.
template <int S>
__global__ void __launch_bounds__(kOpThreads, 4) k_residual_fx(OpFx P,
                                                            const unsigned long long* __restrict__ bmax,
                                                            const int2* __restrict__ xl,
                                                            const double* __restrict__ F,
                                                            double* __restrict__ r) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nf = P.nf, m = P.m;
  int Fu = group_exponent<S>(bmax, 0), Fp = group_exponent<S>(bmax, 1);
  const bool finite = Fu != INT_MIN && Fp != INT_MIN;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (!finite) Fu = Fp = 0;  // only NaN is written then
  if (tid < 2 * P.nf_pad) {
    const int64_t gw = tid >> 5;  // global warp: slice gw / 2, component gw % 2
    const int c = (int)(gw & 1);
    const int64_t row = ((gw >> 1) << 5) + (tid & 31);
    if (row >= nf) return;
    const int64_t sl = row >> 5, lane = row & 31;
    const int2* xc = xl + c * nf;
    const int64_t e0 = P.svp[sl] + lane, e1 = P.svp[sl + 1];
    double ym[S], kb[S];
    {  // M x_t,c for every stage (a first pass over the row)
      int64_t a[S][3];
#pragma unroll
      for (int t = 0; t < S; ++t) a[t][0] = a[t][1] = a[t][2] = 0;
            for (int64_t e = e0; e < e1; e += 32) {
        const int32_t j = P.svc[e];
        const int2 q = P.qM[e];
#pragma unroll
        for (int t = 0; t < S; ++t) fx_mac3(a[t], q, xc[t * m + j]);
      }
      const int em = (int)P.eM[row] + Fu - 115;
#pragma unroll
      for (int t = 0; t < S; ++t) ym[t] = fx_round3(a[t], em);
    }
    {  // K x_t,c (a second pass: the row's indices and x come from L1)
      int64_t a[S][3];
#pragma unroll
      for (int t = 0; t < S; ++t) a[t][0] = a[t][1] = a[t][2] = 0;
            for (int64_t e = e0; e < e1; e += 32) {
        const int32_t j = P.svc[e];
        const int2 q = P.qK[e];
#pragma unroll
        for (int t = 0; t < S; ++t) fx_mac3(a[t], q, xc[t * m + j]);
      }
      const int ek = (int)P.eK[row] + Fu - 115;
#pragma unroll
      for (int t = 0; t < S; ++t) kb[t] = fx_round3(a[t], ek);
    }
    int64_t ab[S][3];
#pragma unroll
    for (int t = 0; t < S; ++t) ab[t][0] = ab[t][1] = ab[t][2] = 0;
    const int2* qB = c == 0 ? P.qB0 : P.qB1;
        for (int64_t e = P.sbp[sl] + lane; e < P.sbp[sl + 1]; e += 32) {
      const int2 qb = qB[e];
      const int64_t vtx = 2 * nf + P.sbc[e];
#pragma unroll
      for (int t = 0; t < S; ++t) fx_mac3(ab[t], qb, xl[t * m + vtx]);
    }
    const int eb = (int)(c == 0 ? P.eB0 : P.eB1)[row] + Fp - 115;
#pragma unroll
    for (int t = 0; t < S; ++t) kb[t] += fx_round3(ab[t], eb);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double y = ym[i];
#pragma unroll
      for (int t = 0; t < S; ++t) y = fma(P.mix[i * 3 + t], kb[t], y);
      const int64_t g = i * m + c * nf + row;
      const double yv = finite ? y : nan;
      r[g] = F ? F[g] - yv : yv;
    }
  } else {
    const int64_t v = tid - 2 * P.nf_pad;
    if (v >= P.nv) return;
    const int64_t sl = v >> 5, lane = v & 31;
    int64_t a[S][3];
#pragma unroll
    for (int t = 0; t < S; ++t) a[t][0] = a[t][1] = a[t][2] = 0;
        for (int64_t e = P.sbtp[sl] + lane; e < P.sbtp[sl + 1]; e += 32) {
      const int32_t j = P.sbtc[e];
      const int2 q0 = P.qT0[e], q1 = P.qT1[e];
#pragma unroll
      for (int t = 0; t < S; ++t) {
        fx_mac3(a[t], q0, xl[t * m + j]);
        fx_mac3(a[t], q1, xl[t * m + nf + j]);
      }
    }
    const int et = (int)P.eT[v] + Fu - 115;
    double bt[S];
#pragma unroll
    for (int t = 0; t < S; ++t) bt[t] = fx_round3(a[t], et);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double y = 0.0;
#pragma unroll
      for (int t = 0; t < S; ++t) y = fma(P.mix[i * 3 + t], bt[t], y);
      const int64_t g = i * m + 2 * nf + v;
      const double yv = finite ? y : nan;
      r[g] = F ? F[g] - yv : yv;
    }
  }
}

}  // namespace

// The longest stored row (SELL slice width) of a level's operator, in
// products per exact sum (Bᵀ rows sum both components).
static int64_t longest_row(const HostCSR& A, int per_entry) {
  int64_t w = 0;
  for (int64_t r = 0; r < A.nrows; ++r) w = std::max<int64_t>(w, A.ptr[r + 1] - A.ptr[r]);
  return w * per_entry;
}

bool op_fixed_fits(Ctx& C, Level& L) {
  return C.opt.op_fixed == 1 && L.dim == 2 && C.s >= 1 && C.s <= 3 &&
         longest_row(L.hops.vel, 1) <= kOpMaxRow && longest_row(L.hops.b, 1) <= kOpMaxRow &&
         longest_row(L.hops.bt, 2) <= kOpMaxRow;
}

cudaError_t launch_op_fixed_convert(Ctx& C, Level& L) {
  FxOpLevel& X = L.fxop;
  const unsigned bv = (unsigned)((L.nf + 255) / 256), bp = (unsigned)((L.nv + 255) / 256);
  k_sell_to_fixed<<<bv, 256, 0, C.stream>>>(L.nf, L.svel.ptr, 1, L.svel.v[0], nullptr, X.qM,
                                            nullptr, X.eM, C.d_err);
  k_sell_to_fixed<<<bv, 256, 0, C.stream>>>(L.nf, L.svel.ptr, 1, L.svel.v[1], nullptr, X.qK,
                                            nullptr, X.eK, C.d_err);
  k_sell_to_fixed<<<bv, 256, 0, C.stream>>>(L.nf, L.sb.ptr, 1, L.sb.v[0], nullptr, X.qB[0],
                                            nullptr, X.eB[0], C.d_err);
  k_sell_to_fixed<<<bv, 256, 0, C.stream>>>(L.nf, L.sb.ptr, 1, L.sb.v[1], nullptr, X.qB[1],
                                            nullptr, X.eB[1], C.d_err);
  k_sell_to_fixed<<<bp, 256, 0, C.stream>>>(L.nv, L.sbt.ptr, 2, L.sbt.v[0], L.sbt.v[1],
                                            X.qT[0], X.qT[1], X.eT, C.d_err);
  return cudaGetLastError();
}

cudaError_t launch_residual_fx(Ctx& C, Level& L, const double* F, const double* x, double* r) {
  FxOpLevel& X = L.fxop;
  cudaError_t e = cudaMemsetAsync(X.bmax, 0, sizeof(unsigned long long) * 6, C.stream);
  if (e != cudaSuccess) return e;
  const int64_t nu = 2 * L.nf, n = C.s * L.m;
  const unsigned gm = (unsigned)std::min<int64_t>((n + kOpThreads - 1) / kOpThreads, 2 * 152);
  const unsigned gc = (unsigned)((n + kOpThreads - 1) / kOpThreads);
  OpFx P{};
  P.nf = L.nf;
  P.nv = L.nv;
  P.m = L.m;
  P.nf_pad = (L.nf + 31) / 32 * 32;
  P.svp = L.svel.ptr;
  P.svc = L.svel.col;
  P.sbp = L.sb.ptr;
  P.sbc = L.sb.col;
  P.sbtp = L.sbt.ptr;
  P.sbtc = L.sbt.col;
  P.qM = X.qM;
  P.qK = X.qK;
  P.qB0 = X.qB[0];
  P.qB1 = X.qB[1];
  P.qT0 = X.qT[0];
  P.qT1 = X.qT[1];
  P.eM = X.eM;
  P.eK = X.eK;
  P.eB0 = X.eB[0];
  P.eB1 = X.eB[1];
  P.eT = X.eT;
  for (int i = 0; i < 9; ++i) P.mix[i] = 0.0;
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j) P.mix[i * 3 + j] = C.dt * C.A[i * C.s + j];
  const int64_t threads = 2 * P.nf_pad + L.nv;
  const unsigned go = (unsigned)((threads + kOpThreads - 1) / kOpThreads);
  switch (C.s) {
    case 1:
      k_block_absmax<1><<<gm, kOpThreads, 0, C.stream>>>(x, L.m, nu, X.bmax);
      k_op_convert<1><<<gc, kOpThreads, 0, C.stream>>>(x, L.m, nu, X.bmax, X.xl);
      k_residual_fx<1><<<go, kOpThreads, 0, C.stream>>>(P, X.bmax, X.xl, F, r);
      break;
    case 2:
      k_block_absmax<2><<<gm, kOpThreads, 0, C.stream>>>(x, L.m, nu, X.bmax);
      k_op_convert<2><<<gc, kOpThreads, 0, C.stream>>>(x, L.m, nu, X.bmax, X.xl);
      k_residual_fx<2><<<go, kOpThreads, 0, C.stream>>>(P, X.bmax, X.xl, F, r);
      break;
    default:
      k_block_absmax<3><<<gm, kOpThreads, 0, C.stream>>>(x, L.m, nu, X.bmax);
      k_op_convert<3><<<gc, kOpThreads, 0, C.stream>>>(x, L.m, nu, X.bmax, X.xl);
      k_residual_fx<3><<<go, kOpThreads, 0, C.stream>>>(P, X.bmax, X.xl, F, r);
      break;
  }
  return cudaGetLastError();
}

}  // namespace irkmg

// Stage operator, transfers, stage right-hand side / update and the vector
// kernels of FGMRES.
//
//   stage residual (Section 3.1):  r = F - J x,
//     J = I_s ⊗ [[M,0],[0,0]] + dt A ⊗ [[K,B],[Bᵀ,0]],
//   evaluated row by row on SELL-32 copies of the operators: one pass over the
//   scalar P2 pattern (M and K share it) and the B / Bᵀ rows gathers every
//   stage and both velocity components of a neighbour at once, and the s×s
//   stage mixing is applied per row.
//   Jᵀ swaps A for Aᵀ and K for Kᵀ (the B blocks are unchanged).
//   transfers (Section 4.1): I_s ⊗ diag(P_u, P_u, P_p) and its transpose.
//   reductions are two-pass with a fixed block count, so sums are bitwise
//   reproducible run to run.
#include "irkmg_internal.h"
#include "op_sell.cuh"

namespace irkmg {

// The stage operator on SELL-32 storage, one thread per row (op_sell.cuh).
template <int S, int D>
__global__ void __launch_bounds__(256) k_residual_sell(OpParams P, const double* __restrict__ F,
                                                       const double* __restrict__ x,
                                                       double* __restrict__ r) {
  residual_sell_row<S, D>(P, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, F, x, r);
}

OpParams op_params(Ctx& C, Level& L, int transpose) {
  OpParams P{};
  P.nf = L.nf;
  P.nv = L.nv;
  P.m = L.m;
  for (int i = 0; i < 9; ++i) P.mix[i] = 0.0;
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j)
      P.mix[i * 3 + j] = C.dt * (transpose ? C.A[j * C.s + i] : C.A[i * C.s + j]);
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.M = L.vel.v[0];
  P.K = transpose ? L.vel.v[2] : L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.btptr = L.bt.ptr;
  P.btcol = L.bt.col;
  P.BTx = L.bt.v[0];
  P.BTy = L.bt.v[1];
  P.nf_pad = (L.nf + 31) / 32 * 32;
  P.svp = L.svel.ptr;
  P.svc = L.svel.col;
  P.sM = L.svel.v[0];
  P.sK = transpose ? L.svel.v[2] : L.svel.v[1];
  P.sbp = L.sb.ptr;
  P.sbc = L.sb.col;
  P.sBx = L.sb.v[0];
  P.sBy = L.sb.v[1];
  P.sbtp = L.sbt.ptr;
  P.sbtc = L.sbt.col;
  P.sBTx = L.sbt.v[0];
  P.sBTy = L.sbt.v[1];
  P.sBz = L.sb.v[2];
  P.sBTz = L.sbt.v[2];
  P.Bz = L.b.v[2];
  P.ns_on = (C.ns && C.ns_active && !transpose) ? 1 : 0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) P.sW[i][k] = L.d_ns_sell[i][k];
  return P;
}

cudaError_t launch_residual(Ctx& C, Level& L, const double* F, const double* x, double* r,
                            int transpose) {
  if (L.fxop_on && !transpose && !(C.ns && C.ns_active))
    return launch_residual_fx(C, L, F, x, r);  // exact fixed point (k_op_fixed.cu)
  OpParams P = op_params(C, L, transpose);
  const int64_t rows = P.nf_pad + L.nv;
  const unsigned grid = (unsigned)((rows + 255) / 256);
  if (L.dim == 2) {
    switch (C.s) {
      case 1: k_residual_sell<1, 2><<<grid, 256, 0, C.stream>>>(P, F, x, r); break;
      case 2: k_residual_sell<2, 2><<<grid, 256, 0, C.stream>>>(P, F, x, r); break;
      default: k_residual_sell<3, 2><<<grid, 256, 0, C.stream>>>(P, F, x, r); break;
    }
  } else {
    switch (C.s) {
      case 1: k_residual_sell<1, 3><<<grid, 256, 0, C.stream>>>(P, F, x, r); break;
      case 2: k_residual_sell<2, 3><<<grid, 256, 0, C.stream>>>(P, F, x, r); break;
      default: k_residual_sell<3, 3><<<grid, 256, 0, C.stream>>>(P, F, x, r); break;
    }
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Transfers.  Rows: nf free P2 nodes (both components, every stage), then nv
// vertices (pressure, every stage).
// ---------------------------------------------------------------------------
struct XferParams {
  int s, dim;
  int64_t nf_out, nv_out, m_out, nf_in, m_in;
  int64_t nf_pad;  // velocity rows rounded up to whole slices
  const int64_t* uptr;
  const int32_t* ucol;
  const double* uw;
  const int64_t* pptr;
  const int32_t* pcol;
  const double* pw;
};

// One output row per thread on SELL-32 copies of the transfer matrices (a
// warp is one slice, so index and weight reads are coalesced; a row ends at
// its first column −1): S stages × D velocity components (or S pressure
// values) of that row, accumulated in registers in the row's entry order.
template <int S, int D>
__global__ void __launch_bounds__(256) k_transfer(XferParams P, const double* __restrict__ in,
                                                  double* __restrict__ out, int add) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < P.nf_pad) {
    const int64_t row = tid;
    if (row >= P.nf_out) return;
    double acc[S][D];
#pragma unroll
    for (int t = 0; t < S; ++t)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[t][c] = 0.0;
    const int64_t sl = row >> 5, e1 = P.uptr[sl + 1];
    for (int64_t e = P.uptr[sl] + (row & 31); e < e1; e += 32) {
      const int32_t j = P.ucol[e];
      if (j < 0) break;
      const double w = P.uw[e];
#pragma unroll
      for (int t = 0; t < S; ++t)
#pragma unroll
        for (int c = 0; c < D; ++c)
          acc[t][c] = fma(w, in[t * P.m_in + c * P.nf_in + j], acc[t][c]);
    }
#pragma unroll
    for (int t = 0; t < S; ++t)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const int64_t g = t * P.m_out + c * P.nf_out + row;
        out[g] = add ? out[g] + acc[t][c] : acc[t][c];
      }
  } else if (tid < P.nf_pad + P.nv_out) {
    const int64_t v = tid - P.nf_pad;
    double acc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) acc[t] = 0.0;
    const int64_t sl = v >> 5, e1 = P.pptr[sl + 1];
    for (int64_t e = P.pptr[sl] + (v & 31); e < e1; e += 32) {
      const int32_t j = P.pcol[e];
      if (j < 0) break;
      const double w = P.pw[e];
#pragma unroll
      for (int t = 0; t < S; ++t) acc[t] = fma(w, in[t * P.m_in + D * P.nf_in + j], acc[t]);
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int64_t g = t * P.m_out + D * P.nf_out + v;
      out[g] = add ? out[g] + acc[t] : acc[t];
    }
  }
}

cudaError_t launch_transfer(const XferParams& P, const double* in, double* out, int add,
                            cudaStream_t st) {
  const int64_t rows = P.nf_pad + P.nv_out;
  const unsigned grid = (unsigned)((rows + 255) / 256);
#define XFER_CASE(S_, D_)                                                   \
  if (P.s == S_ && P.dim == D_) {                                         \
    k_transfer<S_, D_><<<grid, 256, 0, st>>>(P, in, out, add);            \
    return cudaGetLastError();                                            \
  }
  XFER_CASE(1, 2) XFER_CASE(2, 2) XFER_CASE(3, 2) XFER_CASE(1, 3) XFER_CASE(2, 3) XFER_CASE(3, 3)
#undef XFER_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_restrict(Ctx& C, Level& Lf, const double* fine, double* coarse) {
  Level& Lc = *(&Lf - 1);
  XferParams P{};
  P.s = C.s;
  P.dim = Lf.dim;
  P.nf_out = Lc.nf;
  P.nv_out = Lc.nv;
  P.nf_pad = (P.nf_out + 31) / 32 * 32;
  P.m_out = Lc.m;
  P.nf_in = Lf.nf;
  P.m_in = Lf.m;
  P.uptr = Lf.put.ptr;
  P.ucol = Lf.put.col;
  P.uw = Lf.put.v[0];
  P.pptr = Lf.ppt.ptr;
  P.pcol = Lf.ppt.col;
  P.pw = Lf.ppt.v[0];
  return launch_transfer(P, fine, coarse, 0, C.stream);
}

cudaError_t launch_prolong(Ctx& C, Level& Lf, const double* coarse, double* fine, int add) {
  Level& Lc = *(&Lf - 1);
  XferParams P{};
  P.s = C.s;
  P.dim = Lf.dim;
  P.nf_out = Lf.nf;
  P.nv_out = Lf.nv;
  P.nf_pad = (P.nf_out + 31) / 32 * 32;
  P.m_out = Lf.m;
  P.nf_in = Lc.nf;
  P.m_in = Lc.m;
  P.uptr = Lf.pu.ptr;
  P.ucol = Lf.pu.col;
  P.uw = Lf.pu.v[0];
  P.pptr = Lf.pp.ptr;
  P.pcol = Lf.pp.col;
  P.pw = Lf.pp.v[0];
  return launch_transfer(P, coarse, fine, add, C.stream);
}

// ---------------------------------------------------------------------------
// Vector kernels
// ---------------------------------------------------------------------------
__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b,
                        int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

__global__ void k_fill(double* __restrict__ y, double v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = v;
}

static unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

cudaError_t launch_axpby(double* y, const double* x, double a, double b, int64_t n,
                         cudaStream_t st) {
  k_axpby<<<grid_for(n), 256, 0, st>>>(y, x, a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* y, double v, int64_t n, cudaStream_t st) {
  k_fill<<<grid_for(n), 256, 0, st>>>(y, v, n);
  return cudaGetLastError();
}

__global__ void k_fill_sin(double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = sin((double)(i + 1));
}

cudaError_t launch_fill_sin(double* y, int64_t n, cudaStream_t st) {
  k_fill_sin<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, n);
  return cudaGetLastError();
}

// part[b*k + j] = partial sum over block b's contiguous chunk of V_j . w
// Partial dot products of w with k columns of V over fixed contiguous chunks
// (one chunk per block, a fixed tree per block), KMAX columns per pass over
// the chunk (w is read once per pass).  Each thread's elements i, i + 256,
// ... are taken U at a time: all their loads are issued before the
// multiply-adds, which then run in ascending i, so every column's sum has the
// order of one element at a time.
template <int KMAX, int U>
__global__ void __launch_bounds__(256, 2) k_multidot_part(const double* __restrict__ V, int64_t ldv,
                                                          int k, const double* __restrict__ w,
                                                          int64_t n, double* __restrict__ part) {
  __shared__ double red[8][256];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(n, b0 + chunk);
  const int64_t st = blockDim.x;
  for (int p0 = 0; p0 < k; p0 += KMAX) {
    const int nj = min(KMAX, k - p0);
    const double* Vp = V + (int64_t)p0 * ldv;
    double acc[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) acc[q] = 0.0;
    int64_t i = b0 + threadIdx.x;
    for (; i + (U - 1) * st < b1; i += U * st) {
      double wv[U], vv[U][KMAX];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wv[u] = w[i + u * st];
#pragma unroll
        for (int q = 0; q < KMAX; ++q)
          if (q < nj) vv[u][q] = Vp[(int64_t)q * ldv + i + u * st];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < KMAX; ++q)
          if (q < nj) acc[q] = fma(vv[u][q], wv[u], acc[q]);
    }
    for (; i < b1; i += st) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < KMAX; ++q)
        if (q < nj) acc[q] = fma(Vp[(int64_t)q * ldv + i], wi, acc[q]);
    }
    constexpr int QN = KMAX < 8 ? KMAX : 8;  // columns per block tree
#pragma unroll
    for (int j0 = 0; j0 < KMAX; j0 += QN) {
      if (j0 < nj) {
#pragma unroll
        for (int q = 0; q < QN; ++q) red[q][threadIdx.x] = acc[j0 + q];
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
          if (threadIdx.x < (unsigned)o)
#pragma unroll
            for (int q = 0; q < QN; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
          __syncthreads();
        }
        if (threadIdx.x < QN && j0 + (int)threadIdx.x < nj)
          part[(int64_t)blockIdx.x * k + p0 + j0 + threadIdx.x] = red[threadIdx.x][0];
        __syncthreads();
      }
    }
  }
}

// The sums of the partials, column j in block j: a fixed tree over the blocks'
// partials (strided per thread, then halved), the same order on every call.
__global__ void __launch_bounds__(256) k_multidot_final(const double* __restrict__ part,
                                                        int nblocks, int k,
                                                        double* __restrict__ out) {
  __shared__ double red[256];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(int64_t)b * k + j];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

cudaError_t launch_multidot(const double* V, int64_t ldv, int k, const double* w, int64_t n,
                            double* part, double* out, cudaStream_t st) {
  if (k < 1 || k > 64) return cudaErrorInvalidValue;
  if (k <= 4)
    k_multidot_part<4, 4><<<kMultidotBlocks, 256, 0, st>>>(V, ldv, k, w, n, part);
  else if (k <= 8)
    k_multidot_part<8, 2><<<kMultidotBlocks, 256, 0, st>>>(V, ldv, k, w, n, part);
  else
    k_multidot_part<16, 1><<<kMultidotBlocks, 256, 0, st>>>(V, ldv, k, w, n, part);
  k_multidot_final<<<k, 256, 0, st>>>(part, kMultidotBlocks, k, out);
  return cudaGetLastError();
}

__global__ void k_multiaxpy(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int k,
                            const double* __restrict__ h, double sign, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    int j = 0;
    for (; j + 4 <= k; j += 4) {  // four loads issued together, the same FMA order
      const double v0 = V[(int64_t)j * ldv + i], v1 = V[(int64_t)(j + 1) * ldv + i];
      const double v2 = V[(int64_t)(j + 2) * ldv + i], v3 = V[(int64_t)(j + 3) * ldv + i];
      acc = fma(h[j], v0, acc);
      acc = fma(h[j + 1], v1, acc);
      acc = fma(h[j + 2], v2, acc);
      acc = fma(h[j + 3], v3, acc);
    }
    for (; j < k; ++j) acc = fma(h[j], V[(int64_t)j * ldv + i], acc);
    w[i] = fma(sign, acc, w[i]);
  }
}

cudaError_t launch_multiaxpy(double* w, const double* V, int64_t ldv, int k, const double* h,
                             double sign, int64_t n, cudaStream_t st) {
  k_multiaxpy<<<grid_for(n), 256, 0, st>>>(w, V, ldv, k, h, sign, n);
  return cudaGetLastError();
}

// One classical Gram–Schmidt update fused with the next reduction: w ←
// w + sign·V h (k_multiaxpy's FMA order), then the partial dot products of
// the updated w with the k columns of V (NORM: with itself) over
// k_multidot_part's chunks, in its per-thread order and block tree.  The
// results are bitwise those of k_multiaxpy followed by launch_multidot; V and
// w are read once instead of twice.
template <int KMAX, int U, bool NORM>
__global__ void __launch_bounds__(256, 2) k_multiaxpy_dot(double* __restrict__ w,
                                                       const double* __restrict__ V, int64_t ldv,
                                                       int k, const double* __restrict__ h,
                                                       double sign, int64_t n,
                                                       double* __restrict__ part) {
  constexpr int ND = NORM ? 1 : KMAX;
  __shared__ double red[8][256];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(n, b0 + chunk);
  __shared__ double s_h[KMAX];
  if (threadIdx.x < KMAX) s_h[threadIdx.x] = (int)threadIdx.x < k ? h[threadIdx.x] : 0.0;
  __syncthreads();
  double d[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) d[q] = 0.0;
  // U elements per thread at a time, loads first, then the updates
  // and the partial sums in ascending i (the order of one at a time)
  const int64_t st = blockDim.x;
  int64_t i = b0 + threadIdx.x;
  for (; i + (U - 1) * st < b1; i += U * st) {
    double v[U][KMAX], wo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wo[u] = w[i + u * st];
#pragma unroll
      for (int q = 0; q < KMAX; ++q)
        if (q < k) v[u][q] = V[(int64_t)q * ldv + i + u * st];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < KMAX; ++q)
        if (q < k) acc = fma(s_h[q], v[u][q], acc);
      const double wn = fma(sign, acc, wo[u]);
      w[i + u * st] = wn;
      if (NORM) {
        d[0] = fma(wn, wn, d[0]);
      } else {
#pragma unroll
        for (int q = 0; q < ND; ++q)
          if (q < k) d[q] = fma(v[u][q], wn, d[q]);
      }
    }
  }
  for (; i < b1; i += st) {
    double v[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < k) v[q] = V[(int64_t)q * ldv + i];
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < k) acc = fma(s_h[q], v[q], acc);
    const double wn = fma(sign, acc, w[i]);
    w[i] = wn;
    if (NORM) {
      d[0] = fma(wn, wn, d[0]);
    } else {
#pragma unroll
      for (int q = 0; q < ND; ++q)
        if (q < k) d[q] = fma(v[q], wn, d[q]);
    }
  }
  const int kk = NORM ? 1 : k;
  constexpr int QN = ND < 8 ? ND : 8;  // columns per block tree
#pragma unroll
  for (int j0 = 0; j0 < ND; j0 += QN) {
    if (j0 < kk) {
#pragma unroll
      for (int q = 0; q < QN; ++q) red[q][threadIdx.x] = d[j0 + q];
      __syncthreads();
      for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o)
#pragma unroll
          for (int q = 0; q < QN; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
        __syncthreads();
      }
      if (threadIdx.x < QN && j0 + (int)threadIdx.x < kk)
        part[(int64_t)blockIdx.x * kk + j0 + threadIdx.x] = red[threadIdx.x][0];
      __syncthreads();
    }
  }
}

cudaError_t launch_multiaxpy_dot(double* w, const double* V, int64_t ldv, int k, const double* h,
                                 double sign, int64_t n, double* part, double* out, bool norm,
                                 cudaStream_t st) {
  if (k < 1 || k > 16) {  // more columns than registers: the two launches
    cudaError_t e = launch_multiaxpy(w, V, ldv, k, h, sign, n, st);
    if (e != cudaSuccess) return e;
    return norm ? launch_multidot(w, 0, 1, w, n, part, out, st)
                : launch_multidot(V, ldv, k, w, n, part, out, st);
  }
  const int kk = norm ? 1 : k;
  // fewer columns, more elements per thread in flight
  if (norm) {
    if (k <= 4)
      k_multiaxpy_dot<4, 4, true><<<kMultidotBlocks, 256, 0, st>>>(w, V, ldv, k, h, sign, n, part);
    else if (k <= 8)
      k_multiaxpy_dot<8, 2, true><<<kMultidotBlocks, 256, 0, st>>>(w, V, ldv, k, h, sign, n, part);
    else
      k_multiaxpy_dot<16, 1, true><<<kMultidotBlocks, 256, 0, st>>>(w, V, ldv, k, h, sign, n, part);
  } else {
    if (k <= 4)
      k_multiaxpy_dot<4, 4, false><<<kMultidotBlocks, 256, 0, st>>>(w, V, ldv, k, h, sign, n, part);
    else if (k <= 8)
      k_multiaxpy_dot<8, 2, false><<<kMultidotBlocks, 256, 0, st>>>(w, V, ldv, k, h, sign, n, part);
    else
      k_multiaxpy_dot<16, 1, false><<<kMultidotBlocks, 256, 0, st>>>(w, V, ldv, k, h, sign, n, part);
  }
  k_multidot_final<<<kk, 256, 0, st>>>(part, kMultidotBlocks, kk, out);
  return cudaGetLastError();
}

// Per-stage pressure mean removal in two launches: kMeanBlocks blocks per
// stage sum fixed contiguous chunks (a fixed tree per block), then every
// block adds the partial sums of its stage in block order and subtracts the
// mean from its chunk.  The same order on every call: reproducible bitwise.
constexpr int kMeanBlocks = 152;

__global__ void __launch_bounds__(256) k_pressure_part(const double* __restrict__ x, int64_t m,
                                                       int64_t off, int64_t nv,
                                                       double* __restrict__ part) {
  __shared__ double red[256];
  const int t = blockIdx.y;
  const double* p = x + t * m + off;
  const int64_t chunk = (nv + kMeanBlocks - 1) / kMeanBlocks;
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(nv, b0 + chunk);
  double s = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += p[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[t * kMeanBlocks + blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_pressure_sub(double* __restrict__ x, int64_t m,
                                                      int64_t off, int64_t nv,
                                                      const double* __restrict__ part) {
  __shared__ double mean;
  const int t = blockIdx.y;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < kMeanBlocks; ++b) s += part[t * kMeanBlocks + b];
    mean = s / (double)nv;
  }
  __syncthreads();
  double* p = x + t * m + off;
  const int64_t chunk = (nv + kMeanBlocks - 1) / kMeanBlocks;
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(nv, b0 + chunk);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) p[i] -= mean;
}

cudaError_t launch_pressure_mean_remove(Ctx& C, Level& L, double* x) {
  const dim3 grid(kMeanBlocks, (unsigned)C.s);
  k_pressure_part<<<grid, 256, 0, C.stream>>>(x, L.m, L.dim * L.nf, L.nv, C.d_part);
  k_pressure_sub<<<grid, 256, 0, C.stream>>>(x, L.m, L.dim * L.nf, L.nv, C.d_part);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stage right-hand side and update (Section 3.1)
// ---------------------------------------------------------------------------
struct RhsParams {
  int s, dim;
  int64_t nf, nv, np2, m;
  const int32_t *aptr, *acol;
  const double* Mall;
  const int32_t *vptr, *vcol;
  const double* K;
  const int32_t *bptr, *bcol;
  const double *Bx, *By;
  const int32_t *btptr, *btcol;
  const double *BTx, *BTy;
  const double *Bz, *BTz;
};

__global__ void k_stage_rhs(RhsParams P, const double* __restrict__ un, const double* __restrict__ pn,
                            const double* __restrict__ f, double* __restrict__ F) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nf = P.nf;
  const int D = P.dim;
  const double* Bc[3] = {P.Bx, P.By, P.Bz};
  const double* BTc[3] = {P.BTx, P.BTy, P.BTz};
  if (row < nf) {
    double kc[3] = {0.0, 0.0, 0.0};
    for (int32_t p = P.vptr[row]; p < P.vptr[row + 1]; ++p) {
      const int32_t j = P.vcol[p];
      for (int c = 0; c < D; ++c) kc[c] = fma(P.K[p], un[c * nf + j], kc[c]);
    }
    for (int32_t p = P.bptr[row]; p < P.bptr[row + 1]; ++p) {
      const double pv = pn[P.bcol[p]];
      for (int c = 0; c < D; ++c) kc[c] = fma(Bc[c][p], pv, kc[c]);
    }
    for (int t = 0; t < P.s; ++t)
      for (int c = 0; c < D; ++c) {
        double mc = 0.0;
        const double* fc = f + ((int64_t)t * D + c) * P.np2;
        for (int32_t p = P.aptr[row]; p < P.aptr[row + 1]; ++p) mc = fma(P.Mall[p], fc[P.acol[p]], mc);
        F[t * P.m + c * nf + row] = mc - kc[c];
      }
  } else if (row < nf + P.nv) {
    const int64_t v = row - nf;
    double a = 0.0;
    for (int32_t p = P.btptr[v]; p < P.btptr[v + 1]; ++p) {
      const int32_t j = P.btcol[p];
      for (int c = 0; c < D; ++c) a = fma(BTc[c][p], un[c * nf + j], a);
    }
    for (int t = 0; t < P.s; ++t) F[t * P.m + D * nf + v] = -a;
  }
}

cudaError_t launch_stage_rhs(Ctx& C, const double* un, const double* pn, const double* f,
                             double* F) {
  Level& L = C.L.back();
  RhsParams P;
  P.s = C.s;
  P.dim = L.dim;
  P.Bz = L.b.v[2];
  P.BTz = L.bt.v[2];
  P.nf = L.nf;
  P.nv = L.nv;
  P.np2 = L.np2;
  P.m = L.m;
  P.aptr = L.mall.ptr;
  P.acol = L.mall.col;
  P.Mall = L.mall.v[0];
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.K = L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.btptr = L.bt.ptr;
  P.btcol = L.bt.col;
  P.BTx = L.bt.v[0];
  P.BTy = L.bt.v[1];
  const int64_t rows = L.nf + L.nv;
  k_stage_rhs<<<(unsigned)((rows + 255) / 256), 256, 0, C.stream>>>(P, un, pn, f, F);
  return cudaGetLastError();
}

// Stage right-hand side with u^n given at every P2 node (boundary values
// included, e.g. a moving lid): F_i = [M f_i - K u^n - B p^n; -Bᵀ u^n] with K
// and Bᵀ taken over every velocity column.
__global__ void k_stage_rhs_full(RhsParams P, const int32_t* __restrict__ btaptr,
                                 const int32_t* __restrict__ btacol, const double* btax,
                                 const double* btay, const double* btaz,
                                 const double* __restrict__ Kall, const double* __restrict__ un,
                                 const double* __restrict__ pn, const double* __restrict__ f,
                                 double* __restrict__ F) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nf = P.nf, np2 = P.np2;
  const int D = P.dim;
  const double* Bc[3] = {P.Bx, P.By, P.Bz};
  const double* BTA[3] = {btax, btay, btaz};
  if (row < nf) {
    double kc[3] = {0.0, 0.0, 0.0};
    for (int32_t p = P.aptr[row]; p < P.aptr[row + 1]; ++p) {
      const int32_t j = P.acol[p];
      for (int c = 0; c < D; ++c) kc[c] = fma(Kall[p], un[c * np2 + j], kc[c]);
    }
    for (int32_t p = P.bptr[row]; p < P.bptr[row + 1]; ++p) {
      const double pv = pn[P.bcol[p]];
      for (int c = 0; c < D; ++c) kc[c] = fma(Bc[c][p], pv, kc[c]);
    }
    for (int t = 0; t < P.s; ++t)
      for (int c = 0; c < D; ++c) {
        double mc = 0.0;
        const double* fc = f + ((int64_t)t * D + c) * np2;
        for (int32_t p = P.aptr[row]; p < P.aptr[row + 1]; ++p) mc = fma(P.Mall[p], fc[P.acol[p]], mc);
        F[t * P.m + c * nf + row] = mc - kc[c];
      }
  } else if (row < nf + P.nv) {
    const int64_t v = row - nf;
    double a = 0.0;
    for (int32_t p = btaptr[v]; p < btaptr[v + 1]; ++p) {
      const int32_t j = btacol[p];
      for (int c = 0; c < D; ++c) a = fma(BTA[c][p], un[c * np2 + j], a);
    }
    for (int t = 0; t < P.s; ++t) F[t * P.m + D * nf + v] = -a;
  }
}

cudaError_t launch_stage_rhs_full(Ctx& C, const double* un_all, const double* pn, const double* f,
                                  double* F) {
  Level& L = C.L.back();
  RhsParams P;
  P.s = C.s;
  P.dim = L.dim;
  P.Bz = L.b.v[2];
  P.BTz = L.bt.v[2];
  P.nf = L.nf;
  P.nv = L.nv;
  P.np2 = L.np2;
  P.m = L.m;
  P.aptr = L.mall.ptr;
  P.acol = L.mall.col;
  P.Mall = L.mall.v[0];
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.K = L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.btptr = L.bt.ptr;
  P.btcol = L.bt.col;
  P.BTx = L.bt.v[0];
  P.BTy = L.bt.v[1];
  const int64_t rows = L.nf + L.nv;
  P.dim = L.dim;
  P.Bz = L.b.v[2];
  k_stage_rhs_full<<<(unsigned)((rows + 255) / 256), 256, 0, C.stream>>>(
      P, L.btall.ptr, L.btall.col, L.btall.v[0], L.btall.v[1], L.btall.v[2], L.mall.v[1], un_all,
      pn, f, F);
  return cudaGetLastError();
}

__global__ void k_advance(int s, int64_t nu_, int64_t np_, int64_t m, double b0, double b1,
                          double b2, const double* __restrict__ k, double* __restrict__ un,
                          double* __restrict__ pn) {
  const double bw[3] = {b0, b1, b2};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu_ + np_;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int t = 0; t < s; ++t) acc = fma(bw[t], k[t * m + i], acc);
    if (i < nu_)
      un[i] += acc;
    else
      pn[i - nu_] += acc;
  }
}

cudaError_t launch_advance(Ctx& C, const double* k, double* un, double* pn) {
  Level& L = C.L.back();
  double bw[3] = {0, 0, 0};
  for (int t = 0; t < C.s; ++t) bw[t] = C.dt * C.b[t];
  k_advance<<<grid_for(L.m), 256, 0, C.stream>>>(C.s, L.dim * L.nf, L.nv, L.m, bw[0], bw[1], bw[2],
                                                 k, un, pn);
  return cudaGetLastError();
}

}  // namespace irkmg

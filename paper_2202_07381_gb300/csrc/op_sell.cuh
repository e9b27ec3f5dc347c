// The stage operator row by row on SELL-32 copies of the operators (Section
// 3.1: J = I_s ⊗ [[M,0],[0,0]] + dt A ⊗ [[K,B],[Bᵀ,0]]), shared by the
// per-level operator kernel (k_linalg.cu) and the batched persistent smoother
// (k_batch.cu).
#pragma once

#include <cstdint>

namespace irkmg {

struct OpParams {
  int64_t nf, nv, m;
  const double* Bz;                          // third component (3D)
  int64_t nf_pad;  // velocity rows rounded up to a whole slice (SELL kernel)
  double mix[9];  // dt * A (or dt * Aᵀ), row-major 3x3
  const int32_t *vptr, *vcol;
  const double *M, *K;
  const int32_t *bptr, *bcol;
  const double *Bx, *By;
  const int32_t *btptr, *btcol;
  const double *BTx, *BTy;
  // SELL-32 copies
  const int64_t *svp, *sbp, *sbtp;
  const int32_t *svc, *sbc, *sbtc;
  const double *sM, *sK, *sBx, *sBy, *sBTx, *sBTy, *sBz, *sBTz;
  // Navier-Stokes Newton blocks (2D): SELL copies of W_i,dc per stage i, added
  // as y_i,d += sum_c W_i,dc z_i,c with z_i = sum_t mix[i][t] x_t (null: off)
  const double* sW[3][4];
  int ns_on;
};

// One row of the stage operator on SELL-32 storage: row indices tidg in
// [0, nf_pad) are velocity rows, [nf_pad, nf_pad + nv) pressure rows, so
// every warp maps onto one slice and all matrix reads are coalesced.  S
// stages, D velocity components (a stage block is [u_1 .. u_D on the free
// nodes; p]).  r = F - J x, or r = J x when F is null.  XL2: x is read
// through L2 only (ld.global.cg), for an x written earlier by other CTAs of
// the same launch.
template <int S, int D, bool XL2 = false>
__device__ __forceinline__ void residual_sell_row(const OpParams& P, int64_t tidg,
                                                  const double* __restrict__ F,
                                                  const double* __restrict__ x,
                                                  double* __restrict__ r) {
  const int64_t nf = P.nf, m = P.m;
  const double* sB[3] = {P.sBx, P.sBy, P.sBz};
  const double* sBT[3] = {P.sBTx, P.sBTy, P.sBTz};
  if (tidg < P.nf_pad) {
    const int64_t row = tidg;
    if (row >= nf) return;
    double am[S][D], ak[S][D];
#pragma unroll
    for (int t = 0; t < S; ++t)
#pragma unroll
      for (int c = 0; c < D; ++c) am[t][c] = ak[t][c] = 0.0;
    const int64_t sl = row >> 5, lane = row & 31;
    const int64_t b0 = P.svp[sl], b1 = P.svp[sl + 1];
    double an[S][D];
#pragma unroll
    for (int t = 0; t < S; ++t)
#pragma unroll
      for (int c = 0; c < D; ++c) an[t][c] = 0.0;
    for (int64_t e = b0 + lane; e < b1; e += 32) {
      const int32_t j = P.svc[e];
      const double mv = P.sM[e], kv = P.sK[e];
      double xv[S][D];
#pragma unroll
      for (int t = 0; t < S; ++t)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          xv[t][c] = XL2 ? __ldcg(x + t * m + c * nf + j) : x[t * m + c * nf + j];
          am[t][c] = fma(mv, xv[t][c], am[t][c]);
          ak[t][c] = fma(kv, xv[t][c], ak[t][c]);
        }
      if (D == 2 && P.ns_on) {
#pragma unroll
        for (int i = 0; i < S; ++i) {
          double z[D];
#pragma unroll
          for (int c = 0; c < D; ++c) {
            z[c] = 0.0;
#pragma unroll
            for (int t = 0; t < S; ++t) z[c] = fma(P.mix[i * 3 + t], xv[t][c], z[c]);
          }
#pragma unroll
          for (int d = 0; d < D; ++d)
#pragma unroll
            for (int c = 0; c < D; ++c) an[i][d] = fma(P.sW[i][2 * d + c][e], z[c], an[i][d]);
        }
      }
    }
    const int64_t c0 = P.sbp[sl], c1 = P.sbp[sl + 1];
    for (int64_t e = c0 + lane; e < c1; e += 32) {
      const int32_t vtx = P.sbc[e];
      double bv[D];
#pragma unroll
      for (int c = 0; c < D; ++c) bv[c] = sB[c][e];
#pragma unroll
      for (int t = 0; t < S; ++t) {
        const double pv = XL2 ? __ldcg(x + t * m + D * nf + vtx) : x[t * m + D * nf + vtx];
#pragma unroll
        for (int c = 0; c < D; ++c) ak[t][c] = fma(bv[c], pv, ak[t][c]);
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double y = am[i][c] + an[i][c];
#pragma unroll
        for (int t = 0; t < S; ++t) y = fma(P.mix[i * 3 + t], ak[t][c], y);
        const int64_t g = i * m + c * nf + row;
        r[g] = F ? F[g] - y : y;
      }
  } else {
    const int64_t v = tidg - P.nf_pad;
    if (v >= P.nv) return;
    double ap[S];
#pragma unroll
    for (int t = 0; t < S; ++t) ap[t] = 0.0;
    const int64_t sl = v >> 5, lane = v & 31;
    const int64_t b0 = P.sbtp[sl], b1 = P.sbtp[sl + 1];
    for (int64_t e = b0 + lane; e < b1; e += 32) {
      const int32_t j = P.sbtc[e];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double bv = sBT[c][e];
#pragma unroll
        for (int t = 0; t < S; ++t)
          ap[t] = fma(bv, XL2 ? __ldcg(x + t * m + c * nf + j) : x[t * m + c * nf + j], ap[t]);
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double y = 0.0;
#pragma unroll
      for (int t = 0; t < S; ++t) y = fma(P.mix[i * 3 + t], ap[t], y);
      const int64_t g = i * m + D * nf + v;
      r[g] = F ? F[g] - y : y;
    }
  }
}


struct Ctx;
struct Level;
// The operator of level L (transpose: Jᵀ) as OpParams (k_linalg.cu).
OpParams op_params(Ctx& C, Level& L, int transpose);

}  // namespace irkmg

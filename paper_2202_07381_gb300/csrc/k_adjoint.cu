// Kernels of the forward IRK step with a P0 forcing control and of its
// discrete adjoint (Section 3.1 stage equations, differentiated step by step):
//   forward:  F_i += C th (every stage), with C[a, c] = int_c phi_a;
//   adjoint:  kb_j = dt b_j [ub; pb];  after J^T lam = kb:
//             ub -= sum_i (K^T lam_i,u + B lam_i,p),  pb -= sum_i B^T lam_i,u,
//             thb += C^T sum_i lam_i,u,
//             dnu += -(1/nu) sum_i lam_i,u . K (u^n + dt sum_j a_ij k_j,u);
//   objective: 1/2 e^T M2 e and its gradient M2 e, e = u - u_target.
// Reductions are two-pass with kMultidotBlocks blocks in a fixed order.
#include "irkmg_internal.h"

namespace irkmg {

__global__ void k_cell_load(int64_t nf, int64_t nc, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ w,
                            const double* __restrict__ th, double* __restrict__ g) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nf) return;
  double gx = 0.0, gy = 0.0;
  for (int32_t p = ptr[a]; p < ptr[a + 1]; ++p) {
    gx = fma(w[p], th[col[p]], gx);
    gy = fma(w[p], th[nc + col[p]], gy);
  }
  g[a] = gx;
  g[nf + a] = gy;
}

cudaError_t launch_cell_load(Ctx& C, const double* theta, double* g) {
  Level& L = C.L.back();
  k_cell_load<<<(unsigned)((L.nf + 255) / 256), 256, 0, C.stream>>>(
      L.nf, L.mesh.nc, C.cload.ptr, C.cload.col, C.cload.v[0], theta, g);
  return cudaGetLastError();
}

__global__ void k_add_to_stages(int s, int64_t m, int64_t nu_, const double* __restrict__ g,
                                double* __restrict__ F) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu_;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double gi = g[i];
    for (int t = 0; t < s; ++t) F[t * m + i] += gi;
  }
}

cudaError_t launch_add_to_stages(Ctx& C, const double* g, double* F) {
  Level& L = C.L.back();
  k_add_to_stages<<<(unsigned)((2 * L.nf + 255) / 256), 256, 0, C.stream>>>(C.s, L.m, 2 * L.nf,
                                                                             g, F);
  return cudaGetLastError();
}

__global__ void k_kbar(int s, int64_t m, int64_t nu_, double b0, double b1, double b2,
                       const double* __restrict__ ub, const double* __restrict__ pb,
                       double* __restrict__ kb) {
  const double bw[3] = {b0, b1, b2};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = i < nu_ ? ub[i] : pb[i - nu_];
    for (int t = 0; t < s; ++t) kb[t * m + i] = bw[t] * v;
  }
}

cudaError_t launch_kbar(Ctx& C, const double* ub, const double* pb, double* kb) {
  Level& L = C.L.back();
  double bw[3] = {0, 0, 0};
  for (int t = 0; t < C.s; ++t) bw[t] = C.dt * C.b[t];
  k_kbar<<<(unsigned)((L.m + 255) / 256), 256, 0, C.stream>>>(C.s, L.m, 2 * L.nf, bw[0], bw[1],
                                                              bw[2], ub, pb, kb);
  return cudaGetLastError();
}

struct AdjParams {
  int s;
  int64_t nf, nv, m;
  const int32_t *vptr, *vcol;
  const double* KT;
  const int32_t *bptr, *bcol;
  const double *Bx, *By;
  const int32_t *btptr, *btcol;
  const double *BTx, *BTy;
};

__global__ void k_adjoint_update(AdjParams P, const double* __restrict__ lam, double* __restrict__ ub,
                                 double* __restrict__ pb) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nf = P.nf, m = P.m;
  if (row < nf) {
    double ax = 0.0, ay = 0.0;
    for (int t = 0; t < P.s; ++t) {
      const double* l = lam + t * m;
      for (int32_t p = P.vptr[row]; p < P.vptr[row + 1]; ++p) {
        const int32_t j = P.vcol[p];
        ax = fma(P.KT[p], l[j], ax);
        ay = fma(P.KT[p], l[nf + j], ay);
      }
      for (int32_t p = P.bptr[row]; p < P.bptr[row + 1]; ++p) {
        const double lp = l[2 * nf + P.bcol[p]];
        ax = fma(P.Bx[p], lp, ax);
        ay = fma(P.By[p], lp, ay);
      }
    }
    ub[row] -= ax;
    ub[nf + row] -= ay;
  } else if (row < nf + P.nv) {
    const int64_t v = row - nf;
    double a = 0.0;
    for (int t = 0; t < P.s; ++t) {
      const double* l = lam + t * m;
      for (int32_t p = P.btptr[v]; p < P.btptr[v + 1]; ++p) {
        const int32_t j = P.btcol[p];
        a = fma(P.BTx[p], l[j], fma(P.BTy[p], l[nf + j], a));
      }
    }
    pb[v] -= a;
  }
}

cudaError_t launch_adjoint_update(Ctx& C, const double* lam, double* ub, double* pb) {
  Level& L = C.L.back();
  AdjParams P;
  P.s = C.s;
  P.nf = L.nf;
  P.nv = L.nv;
  P.m = L.m;
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.KT = L.vel.v[2];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.btptr = L.bt.ptr;
  P.btcol = L.bt.col;
  P.BTx = L.bt.v[0];
  P.BTy = L.bt.v[1];
  k_adjoint_update<<<(unsigned)((L.nf + L.nv + 255) / 256), 256, 0, C.stream>>>(P, lam, ub, pb);
  return cudaGetLastError();
}

__global__ void k_theta_bar(int s, int64_t nf, int64_t nc, int64_t m, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ w,
                            const double* __restrict__ lam, double* __restrict__ thb) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double ax = 0.0, ay = 0.0;
  for (int t = 0; t < s; ++t)
    for (int32_t p = ptr[c]; p < ptr[c + 1]; ++p) {
      ax = fma(w[p], lam[t * m + col[p]], ax);
      ay = fma(w[p], lam[t * m + nf + col[p]], ay);
    }
  thb[c] += ax;
  thb[nc + c] += ay;
}

cudaError_t launch_theta_bar(Ctx& C, const double* lam, double* thb) {
  Level& L = C.L.back();
  k_theta_bar<<<(unsigned)((L.mesh.nc + 255) / 256), 256, 0, C.stream>>>(
      C.s, L.nf, L.mesh.nc, L.m, C.cloadt.ptr, C.cloadt.col, C.cloadt.v[0], lam, thb);
  return cudaGetLastError();
}

// Block partial sums of per-row terms, then one block adds them in order.
__device__ void block_partial(double v, double* part) {
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double scale, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += part[b];
    out[0] = scale * s;
  }
}

struct DnuParams {
  int s;
  int64_t nf, m;
  double mix[9];  // dt * A
  const int32_t *vptr, *vcol;
  const double* K;
};

// sum over velocity rows a, stages i and components d of
//   lam_i,d[a] * (K (u^n_d + sum_j dt a_ij k_j,d))[a]
__global__ void __launch_bounds__(256) k_dnu_part(DnuParams P, const double* __restrict__ lam,
                                                  const double* __restrict__ k,
                                                  const double* __restrict__ un,
                                                  double* __restrict__ part) {
  double acc = 0.0;
  const int64_t n = P.nf;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  for (int64_t a = r0 + threadIdx.x; a < r1; a += blockDim.x) {
    for (int d = 0; d < 2; ++d) {
      double ku[3] = {0, 0, 0}, kk[3] = {0, 0, 0};  // (K u^n)[a], (K k_j)[a]
      for (int32_t p = P.vptr[a]; p < P.vptr[a + 1]; ++p) {
        const int32_t j = P.vcol[p];
        const double kv = P.K[p];
        ku[0] = fma(kv, un[d * n + j], ku[0]);
        for (int t = 0; t < P.s; ++t) kk[t] = fma(kv, k[t * P.m + d * n + j], kk[t]);
      }
      for (int i = 0; i < P.s; ++i) {
        double y = ku[0];
        for (int t = 0; t < P.s; ++t) y = fma(P.mix[i * 3 + t], kk[t], y);
        acc = fma(lam[i * P.m + d * n + a], y, acc);
      }
    }
  }
  block_partial(acc, part);
}

cudaError_t launch_dnu(Ctx& C, const double* lam, const double* k, const double* un, double* part,
                       double* out) {
  Level& L = C.L.back();
  DnuParams P;
  P.s = C.s;
  P.nf = L.nf;
  P.m = L.m;
  for (int i = 0; i < 9; ++i) P.mix[i] = 0.0;
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j) P.mix[i * 3 + j] = C.dt * C.A[i * C.s + j];
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.K = L.vel.v[1];
  k_dnu_part<<<kMultidotBlocks, 256, 0, C.stream>>>(P, lam, k, un, part);
  k_sum_parts<<<1, 32, 0, C.stream>>>(part, kMultidotBlocks, -1.0 / C.nu, out);
  return cudaGetLastError();
}

// grad = M2 (u - ut) on the free velocity DoFs; out = 1/2 e . grad
__global__ void __launch_bounds__(256) k_tracking_part(int64_t nf, const int32_t* __restrict__ vptr,
                                                       const int32_t* __restrict__ vcol,
                                                       const double* __restrict__ M,
                                                       const double* __restrict__ u,
                                                       const double* __restrict__ ut,
                                                       double* __restrict__ grad,
                                                       double* __restrict__ part) {
  double acc = 0.0;
  const int64_t n = 2 * nf;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const int64_t d = i / nf, a = i - d * nf;
    double g = 0.0;
    for (int32_t p = vptr[a]; p < vptr[a + 1]; ++p) {
      const int64_t j = d * nf + vcol[p];
      g = fma(M[p], u[j] - ut[j], g);
    }
    if (grad) grad[i] = g;
    acc = fma(0.5 * (u[i] - ut[i]), g, acc);
  }
  block_partial(acc, part);
}

cudaError_t launch_tracking(Ctx& C, const double* u, const double* ut, double* grad, double* part,
                            double* out) {
  Level& L = C.L.back();
  k_tracking_part<<<kMultidotBlocks, 256, 0, C.stream>>>(L.nf, L.vel.ptr, L.vel.col, L.vel.v[0], u,
                                                         ut, grad, part);
  k_sum_parts<<<1, 32, 0, C.stream>>>(part, kMultidotBlocks, 1.0, out);
  return cudaGetLastError();
}

}  // namespace irkmg

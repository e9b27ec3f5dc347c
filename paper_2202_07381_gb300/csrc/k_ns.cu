// Navier–Stokes Newton blocks on the GPU (Section 3.2), 2D Taylor–Hood:
//
//   k_ns_stage_velocity: U_t = u^n + dt Σ_j a_tj k_j at every P2 node (the
//     stages are zero on Dirichlet nodes, which keep u^n);
//   k_ns_assemble: for every free row a of the velocity pattern,
//     W_t,dc[a, b] = δ_dc C(U_t)[a, b] + R_dc(U_t)[a, b],
//     C(U)[a, b] = ∫ (U·∇φ_b) φ_a,   R_dc(U)[a, b] = ∫ φ_a φ_b ∂U_d/∂x_c,
//     and g[d][a] = Σ_b C(U)[a, b] U_d[b] over every column b, summed over the
//     cells around node a in ascending cell order by the row's own thread, so
//     the result is deterministic and needs no atomics.  The integrands have
//     degree 5: the 7-point rule of Radon integrates them exactly;
//   k_ns_sell_scatter: the CSR-ordered blocks into the SELL-32 slots the
//     stage operator reads.
#include "irkmg_internal.h"

namespace irkmg {

struct NsMix {
  double a[9];  // Butcher matrix, row stride 3
};

struct NsAsm {
  int64_t nf, nv, stride;  // stride: length of one U component (finest P2 nodes)
  const double* xy;        // vertex coordinates, nv x 2
  const int32_t *cells, *cell_edges;
  const int32_t *nc_ptr, *nc_idx;  // P2 node -> cells (ascending)
  const int32_t *p2_to_free, *free_to_p2;
  const int32_t *vptr, *vcol;
  const double* U;  // this stage: U[d * stride + node]
  double* W[4];     // CSR-ordered outputs on the velocity pattern
  double* g;        // 2 x nf, or null
};

__device__ __forceinline__ int ns_find(const int32_t* __restrict__ col, int32_t b, int32_t e, int32_t key) {
  while (b < e) {
    const int32_t mid = (b + e) >> 1;
    if (col[mid] < key)
      b = mid + 1;
    else
      e = mid;
  }
  return b;
}

__global__ void k_ns_assemble(NsAsm P) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= P.nf) return;
  // Radon's 7-point rule: centroid, and two orbits (α, α, 1 − 2α)
  const double r15 = sqrt(15.0);
  const double al[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
  const double wt[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
  const int32_t p0 = P.vptr[a], p1 = P.vptr[a + 1];
  for (int k = 0; k < 4; ++k)
    for (int32_t p = p0; p < p1; ++p) P.W[k][p] = 0.0;
  const int32_t na = P.free_to_p2[a];
  double gx = 0.0, gy = 0.0;
  for (int32_t q = P.nc_ptr[na]; q < P.nc_ptr[na + 1]; ++q) {
    const int32_t c = P.nc_idx[q];
    int32_t node[6];
    for (int i = 0; i < 3; ++i) {
      node[i] = P.cells[3 * c + i];
      node[3 + i] = (int32_t)(P.nv + P.cell_edges[3 * c + i]);
    }
    int la = 0;
    for (int i = 0; i < 6; ++i)
      if (node[i] == na) la = i;
    // barycentric gradients: [∇λ1; ∇λ2] = J⁻¹ with J = [x1 − x0, x2 − x0] (columns)
    const double x0 = P.xy[2 * node[0]], y0 = P.xy[2 * node[0] + 1];
    const double j00 = P.xy[2 * node[1]] - x0, j10 = P.xy[2 * node[1] + 1] - y0;
    const double j01 = P.xy[2 * node[2]] - x0, j11 = P.xy[2 * node[2] + 1] - y0;
    const double det = j00 * j11 - j01 * j10;
    const double area = 0.5 * fabs(det);
    double gl[3][2];
    gl[1][0] = j11 / det;
    gl[1][1] = -j01 / det;
    gl[2][0] = -j10 / det;
    gl[2][1] = j00 / det;
    gl[0][0] = -gl[1][0] - gl[2][0];
    gl[0][1] = -gl[1][1] - gl[2][1];
    double Ul[2][6];
    for (int d = 0; d < 2; ++d)
      for (int i = 0; i < 6; ++i) Ul[d][i] = P.U[d * P.stride + node[i]];
    double Ce[6], Re[2][2][6];
    for (int b = 0; b < 6; ++b) {
      Ce[b] = 0.0;
      Re[0][0][b] = Re[0][1][b] = Re[1][0][b] = Re[1][1][b] = 0.0;
    }
    for (int iq = 0; iq < 7; ++iq) {
      double lam[3], w;
      if (iq == 0) {
        lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
        w = 9.0 / 40.0;
      } else {
        const int gi = (iq - 1) / 3, r = (iq - 1) % 3;
        lam[0] = lam[1] = lam[2] = al[gi];
        lam[r] = 1.0 - 2.0 * al[gi];
        w = wt[gi];
      }
      w *= area;
      // P2 basis: vertex i -> λ_i (2 λ_i − 1); edges (0,1), (1,2), (0,2) -> 4 λ_i λ_j
      const int ea[3] = {0, 1, 0}, eb[3] = {1, 2, 2};
      double phi[6], gp[6][2];
      for (int i = 0; i < 3; ++i) {
        phi[i] = lam[i] * (2.0 * lam[i] - 1.0);
        for (int k = 0; k < 2; ++k) gp[i][k] = (4.0 * lam[i] - 1.0) * gl[i][k];
      }
      for (int e = 0; e < 3; ++e) {
        const int i = ea[e], j = eb[e];
        phi[3 + e] = 4.0 * lam[i] * lam[j];
        for (int k = 0; k < 2; ++k) gp[3 + e][k] = 4.0 * (lam[i] * gl[j][k] + lam[j] * gl[i][k]);
      }
      double u[2] = {0.0, 0.0}, du[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      for (int i = 0; i < 6; ++i)
        for (int d = 0; d < 2; ++d) {
          u[d] += Ul[d][i] * phi[i];
          for (int k = 0; k < 2; ++k) du[d][k] += Ul[d][i] * gp[i][k];
        }
      const double wa = w * phi[la];
      for (int b = 0; b < 6; ++b) {
        Ce[b] += wa * (u[0] * gp[b][0] + u[1] * gp[b][1]);
        const double pp = wa * phi[b];
        for (int d = 0; d < 2; ++d)
          for (int k = 0; k < 2; ++k) Re[d][k][b] += pp * du[d][k];
      }
    }
    for (int b = 0; b < 6; ++b) {
      gx += Ce[b] * Ul[0][b];
      gy += Ce[b] * Ul[1][b];
      const int32_t fb = P.p2_to_free[node[b]];
      if (fb < 0) continue;
      const int32_t sl = ns_find(P.vcol, p0, p1, fb);
      for (int d = 0; d < 2; ++d)
        for (int k = 0; k < 2; ++k) P.W[2 * d + k][sl] += (d == k ? Ce[b] : 0.0) + Re[d][k][b];
    }
  }
  if (P.g) {
    P.g[a] = gx;
    P.g[P.nf + a] = gy;
  }
}

// U[t][d][node] for every finest P2 node.
__global__ void k_ns_stage_velocity(int s, double dt, NsMix A, int64_t np2, int64_t nf, int64_t m,
                                    const int32_t* __restrict__ p2_to_free,
                                    const double* __restrict__ un_all, const double* __restrict__ k,
                                    double* __restrict__ U) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)s * 2 * np2) return;
  const int64_t t = id / (2 * np2), rem = id - t * 2 * np2, d = rem / np2, node = rem - d * np2;
  double u = un_all[d * np2 + node];
  const int32_t f = p2_to_free[node];
  if (f >= 0)
    for (int j = 0; j < s; ++j) u += dt * A.a[t * 3 + j] * k[j * m + d * nf + f];
  U[id] = u;
}

__global__ void k_ns_sell_scatter(int64_t nnz, const int64_t* __restrict__ perm,
                                  const double* __restrict__ csr, double* __restrict__ sell) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) sell[perm[p]] = csr[p];
}

cudaError_t launch_ns_stage_velocity(Ctx& C, const double* un_all, const double* k, double* U) {
  Level& L = C.L.back();
  NsMix A{};
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j) A.a[i * 3 + j] = C.A[i * C.s + j];
  const int64_t n = (int64_t)C.s * 2 * L.np2;
  k_ns_stage_velocity<<<(unsigned)((n + 255) / 256), 256, 0, C.stream>>>(
      C.s, C.dt, A, L.np2, L.nf, L.m, L.d_p2_to_free, un_all, k, U);
  return cudaGetLastError();
}

cudaError_t launch_ns_assemble(Ctx& C, Level& L, int t, const double* U, int64_t stride, double* g) {
  NsAsm P{};
  P.nf = L.nf;
  P.nv = L.nv;
  P.stride = stride;
  P.xy = L.d_xy;
  P.cells = L.d_cells;
  P.cell_edges = L.d_cell_edges;
  P.nc_ptr = L.d_nc_ptr;
  P.nc_idx = L.d_nc_idx;
  P.p2_to_free = L.d_p2_to_free;
  P.free_to_p2 = L.d_free_to_p2;
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.U = U;
  for (int k = 0; k < 4; ++k) P.W[k] = L.d_ns_csr[t][k];
  P.g = g;
  k_ns_assemble<<<(unsigned)((L.nf + 127) / 128), 128, 0, C.stream>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nnz = L.vel.nnz;
  for (int k = 0; k < 4; ++k)
    k_ns_sell_scatter<<<(unsigned)((nnz + 255) / 256), 256, 0, C.stream>>>(
        nnz, L.d_sell_perm, L.d_ns_csr[t][k], L.d_ns_sell[t][k]);
  return cudaGetLastError();
}

}  // namespace irkmg

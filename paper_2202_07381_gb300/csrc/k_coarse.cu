// Coarsest-grid direct solve (Section 4.1: the coarsest systems are solved
// directly).  The stage operator of the coarsest level has one constant
// pressure mode per stage in its kernel, so it is bordered:
//     [[J, N], [Nᵀ, 0]],  N[:, t] = indicator of stage t's pressure block,
// which is nonsingular; its solution has zero pressure sum in every stage.
// The bordered matrix is assembled densely on the device and inverted once by
// Gauss–Jordan elimination with partial pivoting (one pivot/scale kernel and
// one rank-1 update kernel per column); every solve is then a dense mat-vec
// that reads the inverse from L2-resident memory.
#include <cfloat>

#include "irkmg_internal.h"

namespace irkmg {

struct CoarseBuild {
  int s, dim;
  int64_t nf, nv, m, n;  // n = bordered size
  double mix[9];
  const int32_t *vptr, *vcol;
  const double *M, *K;
  const int32_t *bptr, *bcol;
  const double *Bx, *By;
  const int32_t *btptr, *btcol;
  const double *BTx, *BTy;
  const double *Bz, *BTz;
  const double* W[3][4];  // Navier-Stokes Newton blocks per stage (CSR), 2D
  int ns_on;
};

// One thread per (stage t, row of the single-stage operator).
__global__ void k_coarse_build(CoarseBuild P, double* __restrict__ D) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows1 = P.nf + P.nv;
  if (id >= P.s * rows1) return;
  const int t = (int)(id / rows1);
  const int64_t row = id - t * rows1;
  const double* Bc[3] = {P.Bx, P.By, P.Bz};
  const double* BTc[3] = {P.BTx, P.BTy, P.BTz};
  const int64_t poff = P.dim * P.nf;
  if (row < P.nf) {
    for (int d = 0; d < P.dim; ++d) {
      double* Drow = D + (t * P.m + d * P.nf + row) * P.n;
      for (int32_t p = P.vptr[row]; p < P.vptr[row + 1]; ++p) {
        const int32_t j = P.vcol[p];
        for (int u = 0; u < P.s; ++u) {
          Drow[u * P.m + d * P.nf + j] += (t == u ? P.M[p] : 0.0) + P.mix[t * 3 + u] * P.K[p];
          if (P.ns_on)
            for (int c = 0; c < 2; ++c)
              Drow[u * P.m + c * P.nf + j] += P.mix[t * 3 + u] * P.W[t][2 * d + c][p];
        }
      }
      for (int32_t p = P.bptr[row]; p < P.bptr[row + 1]; ++p) {
        const int32_t vtx = P.bcol[p];
        const double bv = Bc[d][p];
        for (int u = 0; u < P.s; ++u) Drow[u * P.m + poff + vtx] = P.mix[t * 3 + u] * bv;
      }
    }
  } else {
    const int64_t v = row - P.nf;
    double* Drow = D + (t * P.m + poff + v) * P.n;
    for (int32_t p = P.btptr[v]; p < P.btptr[v + 1]; ++p) {
      const int32_t j = P.btcol[p];
      for (int u = 0; u < P.s; ++u)
        for (int d = 0; d < P.dim; ++d) Drow[u * P.m + d * P.nf + j] = P.mix[t * 3 + u] * BTc[d][p];
    }
    const int64_t N = P.s * P.m;
    Drow[N + t] = 1.0;                          // border column
    D[(N + t) * P.n + t * P.m + poff + v] = 1.0;  // border row
  }
}

cudaError_t launch_coarse_build(Ctx& C, double* dense) {
  Level& L = C.L[0];
  CoarseBuild P{};
  P.s = C.s;
  P.dim = L.dim;
  P.Bz = L.b.v[2];
  P.BTz = L.bt.v[2];
  P.nf = L.nf;
  P.nv = L.nv;
  P.m = L.m;
  P.n = C.nb;
  for (int i = 0; i < 9; ++i) P.mix[i] = 0.0;
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j) P.mix[i * 3 + j] = C.dt * C.A[i * C.s + j];
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.M = L.vel.v[0];
  P.K = L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.btptr = L.bt.ptr;
  P.btcol = L.bt.col;
  P.BTx = L.bt.v[0];
  P.BTy = L.bt.v[1];
  P.ns_on = C.ns ? 1 : 0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) P.W[i][k] = L.d_ns_csr[i][k];
  cudaError_t e = cudaMemsetAsync(dense, 0, sizeof(double) * C.nb * C.nb, C.stream);
  if (e != cudaSuccess) return e;
  const int64_t thr = C.s * (L.nf + L.nv);
  k_coarse_build<<<(unsigned)((thr + 127) / 128), 128, 0, C.stream>>>(P, dense);
  return cudaGetLastError();
}

// max |D| over all entries (non-negative doubles order like their bit patterns)
__global__ void k_maxabs(const double* __restrict__ D, int64_t n2, unsigned long long* out) {
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(D[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// Step k, part 1 (one block): pivot search in column k, row swap, save
// column k, scale the pivot row.
__global__ void __launch_bounds__(1024) k_gj_pivot(double* D, int64_t n, int64_t k, double* colk,
                                                   int32_t* perm, const unsigned long long* maxabs,
                                                   int* err) {
  __shared__ double rv[1024];
  __shared__ int64_t ri[1024];
  double best = -1.0;
  int64_t bi = k;
  for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(D[i * n + k]);
    if (a > best) {
      best = a;
      bi = i;
    }
  }
  rv[threadIdx.x] = best;
  ri[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) {
      const double a = rv[threadIdx.x + o];
      const int64_t ia = ri[threadIdx.x + o];
      if (a > rv[threadIdx.x] || (a == rv[threadIdx.x] && ia < ri[threadIdx.x])) {
        rv[threadIdx.x] = a;
        ri[threadIdx.x] = ia;
      }
    }
    __syncthreads();
  }
  const int64_t p = ri[0];
  const double pabs = rv[0];
  if (threadIdx.x == 0) {
    perm[k] = (int32_t)p;
    const double thr = 1e3 * DBL_EPSILON * __longlong_as_double((long long)*maxabs);
    if (!(pabs > thr) && atomicCAS(&err[0], 0, IRKMG_ESINGULAR) == 0) err[1] = (int)k;
  }
  if (p != k)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double x = D[k * n + j];
      D[k * n + j] = D[p * n + j];
      D[p * n + j] = x;
    }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) colk[i] = D[i * n + k];
  __syncthreads();
  const double pinv = pabs > 0.0 ? 1.0 / colk[k] : 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
    D[k * n + j] = (j == k ? 1.0 : D[k * n + j]) * pinv;
}

// Step k, part 2: D[i][j] = (j == k ? 0 : D[i][j]) - colk[i] * D[k][j], i != k.
__global__ void k_gj_update(double* __restrict__ D, int64_t n, int64_t k,
                            const double* __restrict__ colk) {
  const int64_t i = blockIdx.y;
  if (i == k) return;
  const double f = colk[i];
  if (f == 0.0) return;
  const double* Dk = D + k * n;
  double* Di = D + i * n;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    Di[j] = (j == k ? 0.0 : Di[j]) - f * Dk[j];
}

// Undo the row interchanges as column interchanges in reverse order.
__global__ void k_gj_unpermute(double* D, int64_t n, const int32_t* __restrict__ perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* Di = D + i * n;
  for (int64_t k = n - 1; k >= 0; --k) {
    const int32_t p = perm[k];
    if (p != k) {
      const double x = Di[k];
      Di[k] = Di[p];
      Di[p] = x;
    }
  }
}

cudaError_t coarse_invert(Ctx& C, double* D, int64_t n) {
  double* colk = nullptr;
  unsigned long long* mx = nullptr;
  cudaError_t e = cudaMallocAsync(&colk, sizeof(double) * n + 64, C.stream);
  if (e != cudaSuccess) return e;
  mx = (unsigned long long*)(colk + n);
  if ((e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), C.stream)) != cudaSuccess) return e;
  k_maxabs<<<152 * 4, 256, 0, C.stream>>>(D, n * n, mx);
  const unsigned gx = (unsigned)((n + 255) / 256);
  for (int64_t k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 1024, 0, C.stream>>>(D, n, k, colk, C.d_coarse_perm, mx, C.d_err);
    k_gj_update<<<dim3(gx, (unsigned)n), 256, 0, C.stream>>>(D, n, k, colk);
  }
  k_gj_unpermute<<<(unsigned)((n + 127) / 128), 128, 0, C.stream>>>(D, n, C.d_coarse_perm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaFreeAsync(colk, C.stream);
}

// x = X[0:N, 0:N] r (the border rows/columns only carry the multipliers).
// Warp per row of the row-major inverse; transpose = 1 uses the columns.
__global__ void k_coarse_apply(const double* __restrict__ X, int64_t n, int64_t N,
                               const double* __restrict__ r, double* __restrict__ x) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  const double* Xr = X + row * n;
  double acc = 0.0;
  for (int64_t j = lane; j < N; j += 32) acc = fma(Xr[j], r[j], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[row] = acc;
}

__global__ void k_coarse_apply_t(const double* __restrict__ X, int64_t n, int64_t N,
                                 const double* __restrict__ r, double* __restrict__ x) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= N) return;
  double acc = 0.0;
  for (int64_t i = 0; i < N; ++i) acc = fma(X[i * n + col], r[i], acc);
  x[col] = acc;
}

cudaError_t launch_coarse_apply(Ctx& C, const double* r, double* x, int transpose) {
  const int64_t N = C.L[0].N;
  if (transpose)
    k_coarse_apply_t<<<(unsigned)((N + 127) / 128), 128, 0, C.stream>>>(C.d_coarse_inv, C.nb, N,
                                                                         r, x);
  else
    k_coarse_apply<<<(unsigned)((N * 32 + 255) / 256), 256, 0, C.stream>>>(C.d_coarse_inv, C.nb,
                                                                           N, r, x);
  return cudaGetLastError();
}

}  // namespace irkmg

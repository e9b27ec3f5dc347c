// Vertex-star Vanka patches on the GPU (Section 4.2, Fig. 1 left):
//   * patch maps: for every vertex v, the free P2 nodes in the closure of the
//     cells around v (ascending);  the patch S_v is, per stage, the u_x and
//     u_y DoFs of those nodes and the single pressure DoF of v;
//   * distance-2 colouring (patches of one colour share no DoF), computed by
//     Jones–Plassmann rounds with priority = -vertex id, which reproduces the
//     sequential greedy colouring in vertex order exactly;
//   * gather of A_v = R_v J R_vᵀ from the assembled level operators and its
//     explicit inverse by Gauss–Jordan elimination with partial pivoting;
//   * the additive correction  out += scale · R_vᵀ A_v⁻¹ R_v r, one launch per
//     colour, so the scatter needs no atomics and is deterministic.
#include <algorithm>
#include <cfloat>
#include <cstdio>

#include "irkmg_internal.h"
#include "tma.cuh"

namespace irkmg {

constexpr int kMaxStar = 24;        // cells around a vertex handled by the map kernel
constexpr int kMaxPatchNodes = 96;  // free P2 nodes per patch (interior: 19 in 2D, 65 in 3D)

// ---------------------------------------------------------------------------
// Patch maps
// ---------------------------------------------------------------------------
__global__ void k_patch_maps(int32_t nv, int kv, int ke, const int32_t* __restrict__ cells,
                             const int32_t* __restrict__ cell_edges,
                             const int32_t* __restrict__ vc_ptr, const int32_t* __restrict__ vc_idx,
                             const int32_t* __restrict__ p2_to_free, int32_t maxnodes,
                             int32_t* __restrict__ tmp, int32_t* __restrict__ cnt) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  int32_t buf[10 * kMaxStar];
  int n = 0;
  const int32_t b0 = vc_ptr[v], b1 = vc_ptr[v + 1];
  if (b1 - b0 > kMaxStar) {
    cnt[v] = -1;
    return;
  }
  for (int32_t p = b0; p < b1; ++p) {
    const int32_t c = vc_idx[p];
    for (int a = 0; a < kv; ++a) {
      int32_t f = p2_to_free[cells[kv * c + a]];
      if (f >= 0) buf[n++] = f;
    }
    for (int a = 0; a < ke; ++a) {
      int32_t f = p2_to_free[nv + cell_edges[ke * c + a]];
      if (f >= 0) buf[n++] = f;
    }
  }
  // insertion sort + unique (free numbering preserves P2 order)
  for (int i = 1; i < n; ++i) {
    int32_t x = buf[i];
    int j = i - 1;
    while (j >= 0 && buf[j] > x) {
      buf[j + 1] = buf[j];
      --j;
    }
    buf[j + 1] = x;
  }
  int u = 0;
  for (int i = 0; i < n; ++i)
    if (u == 0 || buf[i] != buf[u - 1]) buf[u++] = buf[i];
  if (u > maxnodes) {
    cnt[v] = -1;
    return;
  }
  for (int i = 0; i < u; ++i) tmp[(int64_t)v * maxnodes + i] = buf[i];
  cnt[v] = u;
}

__global__ void k_compact_patches(int32_t nv, int32_t maxnodes, const int32_t* __restrict__ tmp,
                                  const int32_t* __restrict__ ptr, int32_t* __restrict__ nodes) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int32_t b = ptr[v], e = ptr[v + 1];
  for (int32_t i = 0; i < e - b; ++i) nodes[b + i] = tmp[(int64_t)v * maxnodes + i];
}

// Exclusive scan of n counts into n+1 offsets (single block; set-up only).
__global__ void k_scan(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  __shared__ int32_t s[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    int32_t x = (i < n) ? in[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int32_t y = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < n) out[i] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

cudaError_t launch_patch_maps(Level& L, cudaStream_t st, int maxnodes, int32_t* d_tmp,
                              int32_t* d_cnt) {
  int32_t nv = (int32_t)L.nv;
  k_patch_maps<<<(nv + 127) / 128, 128, 0, st>>>(nv, L.mesh.nvc(), L.mesh.nle(), L.d_cells,
                                                  L.d_cell_edges, L.d_vc_ptr, L.d_vc_idx,
                                                  L.d_p2_to_free, maxnodes, d_tmp, d_cnt);
  return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_compact_patches(Level& L, cudaStream_t st, int maxnodes, const int32_t* d_tmp,
                                   const int32_t* d_cnt) {
  (void)d_cnt;
  int32_t nv = (int32_t)L.nv;
  k_compact_patches<<<(nv + 127) / 128, 128, 0, st>>>(nv, maxnodes, d_tmp, L.d_patch_ptr,
                                                       L.d_patch_nodes);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Distance-2 colouring, one Jones–Plassmann round.  A vertex is coloured once
// every lower-id vertex within graph distance 2 is coloured; it takes the
// smallest colour none of them uses.  Colours are written once, so reading a
// neighbour coloured in the same round is harmless.
// ---------------------------------------------------------------------------
constexpr int kMaxColours = 256;

__global__ void k_colour_round(int32_t nv, const int32_t* __restrict__ vv_ptr,
                               const int32_t* __restrict__ vv_idx, int32_t* colour,
                               int* remaining, int* overflow) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  volatile int32_t* col = colour;
  if (col[v] >= 0) return;
  uint64_t mask[kMaxColours / 64] = {0, 0, 0, 0};
  bool ready = true;
  for (int32_t p = vv_ptr[v]; p < vv_ptr[v + 1] && ready; ++p) {
    const int32_t x = vv_idx[p];
    if (x < v) {
      int32_t cx = col[x];
      if (cx < 0) {
        ready = false;
        break;
      }
      mask[cx >> 6] |= 1ull << (cx & 63);
    }
    for (int32_t q = vv_ptr[x]; q < vv_ptr[x + 1]; ++q) {
      const int32_t y = vv_idx[q];
      if (y >= v) continue;
      int32_t cy = col[y];
      if (cy < 0) {
        ready = false;
        break;
      }
      mask[cy >> 6] |= 1ull << (cy & 63);
    }
  }
  if (!ready) {
    atomicAdd(remaining, 1);
    return;
  }
  int c = 0;
  while (c < kMaxColours && (mask[c >> 6] >> (c & 63)) & 1ull) ++c;
  if (c >= kMaxColours) {
    atomicExch(overflow, 1);
    c = kMaxColours - 1;
  }
  col[v] = c;
}

cudaError_t launch_colour_round(Level& L, cudaStream_t st, int* d_remaining, int* d_overflow) {
  int32_t nv = (int32_t)L.nv;
  k_colour_round<<<(nv + 127) / 128, 128, 0, st>>>(nv, L.d_vv_ptr, L.d_vv_idx, L.d_colour,
                                                    d_remaining, d_overflow);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Patch gather + explicit inverse (one CTA per patch, FP64 in shared memory).
// Local order of S_v inside a stage: u_x of the L nodes, u_y of the L nodes,
// p_v; stages consecutive.  Block entries (Section 3.1 Kronecker form):
//   velocity-velocity  delta_tu M_ab + dt a_tu K_ab   (same component)
//   velocity-pressure  dt a_tu B^d_{a v}
//   pressure-velocity  dt a_tu B^d_{b v}              (row of Bᵀ)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int csr_find(const int32_t* __restrict__ col, int32_t b, int32_t e,
                                        int32_t key) {
  while (b < e) {
    int32_t mid = (b + e) >> 1;
    int32_t c = col[mid];
    if (c < key)
      b = mid + 1;
    else
      e = mid;
  }
  return b;  // caller checks col[b] == key
}

struct InvParams {
  int s, dim;
  double A[9];
  double dt;
  int64_t nf;
  const int32_t *patch_ptr, *patch_nodes, *order;
  const int64_t* fac_off;
  const int32_t *vptr, *vcol;
  const double *M, *K;
  const int32_t *bptr, *bcol;
  const double *Bx, *By, *Bz;
  int* err;  // [0] status, [1] patch id
  // Navier-Stokes Newton blocks (2D): CSR copies of W_t,dc per stage t; the
  // velocity block (t, u) gains dt a_tu W_t,dd' (null / ns_on = 0: off)
  const double* W[3][4];
  int ns_on;
};

// Shared-memory scratch of one patch inversion.
struct InvScratch {
  int32_t nodes[kMaxPatchNodes];
  int32_t perm[3 * (2 * kMaxPatchNodes + 1)];
  double colk[3 * (2 * kMaxPatchNodes + 1)];
  double red_v[256];
  int red_i[256];
  double maxabs;
};

// Builds I_s ⊗ M̃ + dt A ⊗ K̃ of patch v (s = P.s, A = P.A, nodes already in
// W.nodes, L of them) row-major in A_ (np = s (D L + 1)), and overwrites it
// with its inverse (Gauss–Jordan, partial pivoting).  All threads of the block
// take part; a pivot below 1e3 eps max|A| records IRKMG_ESINGULAR for v.
__device__ void patch_build_invert(const InvParams& P, int32_t v, int L, double* A, InvScratch& W) {
  const int D = P.dim;
  const int q = D * L + 1, np = P.s * q;
  int32_t* nodes = W.nodes;
  int32_t* s_perm = W.perm;
  double* colk = W.colk;
  double* red_v = W.red_v;
  int* red_i = W.red_i;
  for (int i = threadIdx.x; i < np * np; i += blockDim.x) A[i] = 0.0;
  __syncthreads();
  // velocity-velocity blocks
  for (int idx = threadIdx.x; idx < L * L; idx += blockDim.x) {
    const int a = idx / L, b = idx % L;
    const int32_t ra = nodes[a], cb = nodes[b];
    const int32_t p0 = P.vptr[ra], p1 = P.vptr[ra + 1];
    const int32_t pos = csr_find(P.vcol, p0, p1, cb);
    double mab = 0.0, kab = 0.0;
    if (pos < p1 && P.vcol[pos] == cb) {
      mab = P.M[pos];
      kab = P.K[pos];
    }
    for (int t = 0; t < P.s; ++t)
      for (int u = 0; u < P.s; ++u) {
        const double val = (t == u ? mab : 0.0) + P.dt * P.A[t * 3 + u] * kab;
        for (int d = 0; d < D; ++d) A[(t * q + d * L + a) * np + (u * q + d * L + b)] = val;
        if (P.ns_on && D == 2 && pos < p1 && P.vcol[pos] == cb) {
          const double f = P.dt * P.A[t * 3 + u];
          for (int d = 0; d < 2; ++d)
            for (int c = 0; c < 2; ++c)
              A[(t * q + d * L + a) * np + (u * q + c * L + b)] += f * P.W[t][2 * d + c][pos];
        }
      }
  }
  // velocity-pressure and pressure-velocity blocks
  for (int a = threadIdx.x; a < L; a += blockDim.x) {
    const int32_t ra = nodes[a];
    const int32_t p0 = P.bptr[ra], p1 = P.bptr[ra + 1];
    const int32_t pos = csr_find(P.bcol, p0, p1, v);
    double bv[3] = {0.0, 0.0, 0.0};
    const double* Bc[3] = {P.Bx, P.By, P.Bz};
    if (pos < p1 && P.bcol[pos] == v)
      for (int d = 0; d < D; ++d) bv[d] = Bc[d][pos];
    for (int t = 0; t < P.s; ++t)
      for (int u = 0; u < P.s; ++u) {
        const double f = P.dt * P.A[t * 3 + u];
        for (int d = 0; d < D; ++d) {
          A[(t * q + d * L + a) * np + (u * q + D * L)] = f * bv[d];
          A[(t * q + D * L) * np + (u * q + d * L + a)] = f * bv[d];
        }
      }
  }
  __syncthreads();
  // max |A| for the singularity threshold
  double mx = 0.0;
  for (int i = threadIdx.x; i < np * np; i += blockDim.x) mx = fmax(mx, fabs(A[i]));
  red_v[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) red_v[threadIdx.x] = fmax(red_v[threadIdx.x], red_v[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) W.maxabs = red_v[0];
  __syncthreads();
  const double thresh = 1e3 * DBL_EPSILON * W.maxabs;
  // Gauss–Jordan with partial pivoting (first largest |.|), in place
  for (int k = 0; k < np; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < np; i += blockDim.x) {
      double a = fabs(A[i * np + k]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
    red_v[threadIdx.x] = best;
    red_i[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < (unsigned)o) {
        double a = red_v[threadIdx.x + o];
        int ia = red_i[threadIdx.x + o];
        if (a > red_v[threadIdx.x] || (a == red_v[threadIdx.x] && ia < red_i[threadIdx.x])) {
          red_v[threadIdx.x] = a;
          red_i[threadIdx.x] = ia;
        }
      }
      __syncthreads();
    }
    const int p = red_i[0];
    const double pabs = red_v[0];
    if (threadIdx.x == 0) s_perm[k] = p;
    if (p != k)
      for (int j = threadIdx.x; j < np; j += blockDim.x) {
        double x = A[k * np + j];
        A[k * np + j] = A[p * np + j];
        A[p * np + j] = x;
      }
    __syncthreads();
    if (!(pabs > thresh)) {
      if (threadIdx.x == 0 && atomicCAS(&P.err[0], 0, IRKMG_ESINGULAR) == 0) P.err[1] = v;
    }
    for (int i = threadIdx.x; i < np; i += blockDim.x) colk[i] = A[i * np + k];
    __syncthreads();
    const double pinv = (pabs > 0.0) ? 1.0 / colk[k] : 0.0;
    for (int j = threadIdx.x; j < np; j += blockDim.x)
      A[k * np + j] = (j == k ? 1.0 : A[k * np + j]) * pinv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
      const int i = idx / np, j = idx - i * np;
      if (i == k) continue;
      A[idx] = (j == k ? 0.0 : A[idx]) - colk[i] * A[k * np + j];
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int k = np - 1; k >= 0; --k) {
    const int p = s_perm[k];
    if (p != k)
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        double x = A[i * np + k];
        A[i * np + k] = A[i * np + p];
        A[i * np + p] = x;
      }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_patch_invert(InvParams P, int64_t npatch, T* fac) {
  extern __shared__ double smem[];
  __shared__ InvScratch W;
  const int64_t pi = blockIdx.x;
  if (pi >= npatch) return;
  const int32_t v = P.order[pi];
  const int32_t nb = P.patch_ptr[v], L = P.patch_ptr[v + 1] - nb;
  const int np = P.s * (P.dim * L + 1);
  double* A = smem;  // row-major np x np
  for (int i = threadIdx.x; i < L; i += blockDim.x) W.nodes[i] = P.patch_nodes[nb + i];
  patch_build_invert(P, v, L, A, W);
  // store column-major: X[j*np + i] = Ainv[i][j]
  T* X = fac + P.fac_off[pi];
  for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
    const int j = idx / np, i = idx - j * np;
    X[idx] = (T)A[i * np + j];
  }
}

// Kronecker-decoupled patch factors: for every block of the real block
// diagonalisation A = T D T⁻¹ (one real eigenvalue λ, or one pair α ± iβ as
// [[α, β], [−β, α]]) the patch matrix I ⊗ M̃ + dt D_b ⊗ K̃ of that block is
// built and inverted, and its n×n pieces are stored column-major one after
// the other: kind 0 (real): the inverse; kind 1 (pair): X, Y from the first
// block column [X; Y] of the inverse; kind 2 (pair): X + Y, X, Y.  The n
// spatial DoF indices follow the matrices (see k_patch_gidx_kron).
template <typename T>
__global__ void __launch_bounds__(256) k_patch_invert_kron(InvParams P, KronPlan K, int64_t npatch,
                                                           T* fac) {
  extern __shared__ double smem[];
  __shared__ InvScratch W;
  const int64_t pi = blockIdx.x;
  if (pi >= npatch) return;
  const int32_t v = P.order[pi];
  const int32_t nb = P.patch_ptr[v], L = P.patch_ptr[v + 1] - nb;
  const int n = P.dim * L + 1;
  const int64_t nn = (int64_t)n * n;
  double* A = smem;
  for (int i = threadIdx.x; i < L; i += blockDim.x) W.nodes[i] = P.patch_nodes[nb + i];
  T* base = fac + P.fac_off[pi];
  for (int b = 0; b < K.nblk; ++b) {
    InvParams Q = P;
    const int q = K.blk_size[b];
    Q.s = q;
    for (int i = 0; i < 9; ++i) Q.A[i] = 0.0;
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) Q.A[i * 3 + j] = K.blk[b][i * q + j];
    patch_build_invert(Q, v, L, A, W);
    const int np = q * n;  // row-major np x np inverse in A
    T* X = base + (int64_t)K.blk_mat[b] * nn;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int j = idx / n, i = idx - j * n;  // column-major (i, j)
      const double x = A[i * np + j];
      if (K.blk_kind[b] == 0) {
        X[idx] = (T)x;
      } else {
        const double y = A[(n + i) * np + j];
        if (K.blk_kind[b] == 1) {
          X[idx] = (T)x;
          X[nn + idx] = (T)y;
        } else {
          X[idx] = (T)(x + y);
          X[nn + idx] = (T)x;
          X[2 * nn + idx] = (T)y;
        }
      }
    }
    __syncthreads();  // A is rebuilt by the next block
  }
}

cudaError_t launch_patch_invert(Ctx& C, Level& L, int precision) {
  InvParams P{};
  P.s = C.s;
  P.dim = L.dim;
  P.Bz = L.b.v[2];
  for (int i = 0; i < 9; ++i) P.A[i] = 0.0;
  for (int i = 0; i < C.s; ++i)
    for (int j = 0; j < C.s; ++j) P.A[i * 3 + j] = C.A[i * C.s + j];
  P.dt = C.dt;
  P.nf = L.nf;
  P.patch_ptr = L.d_patch_ptr;
  P.patch_nodes = L.d_patch_nodes;
  P.order = L.d_order;
  P.fac_off = L.d_fac_off;
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.M = L.vel.v[0];
  P.K = L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.err = C.d_err;
  P.ns_on = C.ns ? 1 : 0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) P.W[i][k] = L.d_ns_csr[i][k];
  const size_t smem = (size_t)L.max_np * L.max_np * sizeof(double);
  if (precision == 64) {
    cudaFuncSetAttribute(k_patch_invert<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_invert<double><<<(unsigned)L.nv, 256, smem, C.stream>>>(P, L.nv, (double*)L.d_fac);
  } else {
    cudaFuncSetAttribute(k_patch_invert<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_invert<float><<<(unsigned)L.nv, 256, smem, C.stream>>>(P, L.nv, (float*)L.d_fac);
  }
  return cudaGetLastError();
}

cudaError_t launch_patch_invert_kron(Ctx& C, Level& L) {
  InvParams P{};
  P.s = C.s;
  P.dim = L.dim;
  P.Bz = L.b.v[2];
  for (int i = 0; i < 9; ++i) P.A[i] = 0.0;
  P.dt = C.dt;
  P.nf = L.nf;
  P.patch_ptr = L.d_patch_ptr;
  P.patch_nodes = L.d_patch_nodes;
  P.order = L.d_order;
  P.fac_off = L.d_fac_off;
  P.vptr = L.vel.ptr;
  P.vcol = L.vel.col;
  P.M = L.vel.v[0];
  P.K = L.vel.v[1];
  P.bptr = L.b.ptr;
  P.bcol = L.b.col;
  P.Bx = L.b.v[0];
  P.By = L.b.v[1];
  P.err = C.d_err;
  int q = 1;
  for (int b = 0; b < C.kplan.nblk; ++b) q = std::max(q, C.kplan.blk_size[b]);
  const size_t smem = (size_t)(q * L.kron_nmax) * (q * L.kron_nmax) * sizeof(double);
  if (C.opt.patch_precision == 64) {
    cudaFuncSetAttribute(k_patch_invert_kron<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_invert_kron<double><<<(unsigned)L.nv, 256, smem, C.stream>>>(P, C.kplan, L.nv,
                                                                        (double*)L.d_fac);
  } else {
    cudaFuncSetAttribute(k_patch_invert_kron<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_patch_invert_kron<float><<<(unsigned)L.nv, 256, smem, C.stream>>>(P, C.kplan, L.nv,
                                                                       (float*)L.d_fac);
  }
  return cudaGetLastError();
}

// Spatial DoF indices of every ordered patch of a decoupled level (n of them,
// velocity components then the pressure vertex), stored after its nm
// matrices; stage t adds t·m.
template <typename T>
__global__ void k_patch_gidx_kron(int D, int nm, int64_t nf, int64_t npatch,
                                  const int32_t* __restrict__ patch_ptr,
                                  const int32_t* __restrict__ patch_nodes,
                                  const int32_t* __restrict__ order,
                                  const int64_t* __restrict__ fac_off, T* fac) {
  const int64_t pi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pi >= npatch) return;
  const int32_t v = order[pi];
  const int32_t nb = patch_ptr[v], L = patch_ptr[v + 1] - nb;
  const int n = D * L + 1;
  const int64_t xbytes = ((int64_t)nm * n * n * (int64_t)sizeof(T) + 15) & ~(int64_t)15;
  int32_t* g = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(fac + fac_off[pi]) + xbytes);
  for (int k = lane; k < n; k += 32) {
    int64_t gi;
    if (k < D * L) {
      const int c = k / L;
      gi = c * nf + patch_nodes[nb + k - c * L];
    } else {
      gi = D * nf + v;
    }
    g[k] = (int32_t)gi;
  }
}

cudaError_t launch_patch_gidx_kron(Ctx& C, Level& L) {
  const unsigned grid = (unsigned)((L.nv * 32 + 255) / 256);
  if (C.opt.patch_precision == 64)
    k_patch_gidx_kron<double><<<grid, 256, 0, C.stream>>>(L.dim, C.kplan.nm, L.nf, L.nv,
                                                          L.d_patch_ptr, L.d_patch_nodes,
                                                          L.d_order, L.d_fac_off, (double*)L.d_fac);
  else
    k_patch_gidx_kron<float><<<grid, 256, 0, C.stream>>>(L.dim, C.kplan.nm, L.nf, L.nv,
                                                         L.d_patch_ptr, L.d_patch_nodes, L.d_order,
                                                         L.d_fac_off, (float*)L.d_fac);
  return cudaGetLastError();
}

// Global DoF index list of every ordered patch, stored after its inverse.
template <typename T>
__global__ void k_patch_gidx(int s, int D, int64_t nf, int64_t m, int64_t npatch,
                             const int32_t* __restrict__ patch_ptr,
                             const int32_t* __restrict__ patch_nodes,
                             const int32_t* __restrict__ order, const int64_t* __restrict__ fac_off,
                             T* fac) {
  const int64_t pi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pi >= npatch) return;
  const int32_t v = order[pi];
  const int32_t nb = patch_ptr[v], L = patch_ptr[v + 1] - nb;
  const int q = D * L + 1, np = s * q;
  const int64_t xbytes = ((int64_t)np * np * (int64_t)sizeof(T) + 15) & ~(int64_t)15;
  int32_t* g = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(fac + fac_off[pi]) + xbytes);
  for (int i = lane; i < np; i += 32) {
    const int t = i / q, k = i - t * q;
    int64_t gi;
    if (k < D * L) {
      const int c = k / L;
      gi = t * m + c * nf + patch_nodes[nb + k - c * L];
    } else {
      gi = t * m + D * nf + v;
    }
    g[i] = (int32_t)gi;
  }
}

cudaError_t launch_patch_gidx(Ctx& C, Level& L) {
  const unsigned grid = (unsigned)((L.nv * 32 + 255) / 256);
  if (C.opt.patch_precision == 64)
    k_patch_gidx<double><<<grid, 256, 0, C.stream>>>(C.s, L.dim, L.nf, L.m, L.nv, L.d_patch_ptr,
                                                     L.d_patch_nodes, L.d_order, L.d_fac_off,
                                                     (double*)L.d_fac);
  else
    k_patch_gidx<float><<<grid, 256, 0, C.stream>>>(C.s, L.dim, L.nf, L.m, L.nv, L.d_patch_ptr,
                                                    L.d_patch_nodes, L.d_order, L.d_fac_off,
                                                    (float*)L.d_fac);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Vanka apply for one colour: warp per patch.  y = A_v⁻¹ r|_{S_v} as a dense
// column-major mat-vec (lanes over rows, one column per step, fully coalesced
// loads of the stored inverse), then out[S_v] += scale · y.  Patches of one
// colour share no DoF, so the read-modify-write needs no atomics.
// transpose = 1 applies (A_v⁻¹)ᵀ = (A_vᵀ)⁻¹, the patch inverse of Jᵀ.
// ---------------------------------------------------------------------------
constexpr int kApplyWarps = 8;
constexpr int kMaxNp = 160;

struct ApplyParams {
  int s, dim;
  int64_t nf, m;
  const int32_t *patch_ptr, *patch_nodes, *order, *np;
  const int64_t* fac_off;
  const double* r;
  double* out;
  double scale;
  int64_t first, count;  // ordered-patch range of this colour
};

template <typename T, int R>
__global__ void __launch_bounds__(kApplyWarps * 32) k_vanka_apply(ApplyParams P, const T* __restrict__ fac) {
  __shared__ T s_r[kApplyWarps][kMaxNp];
  __shared__ int32_t s_g[kApplyWarps][kMaxNp];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kApplyWarps + warp;
  if (w >= P.count) return;
  const int64_t pi = P.first + w;
  const int32_t v = P.order[pi];
  const int32_t nb = P.patch_ptr[v], L = P.patch_ptr[v + 1] - nb;
  const int q = P.dim * L + 1, np = P.s * q;
  for (int i = lane; i < np; i += 32) {
    const int t = i / q, k = i - t * q;
    int64_t g;
    if (k < P.dim * L) {
      const int c = k / L;
      g = t * P.m + c * P.nf + P.patch_nodes[nb + k - c * L];
    } else {
      g = t * P.m + P.dim * P.nf + v;
    }
    s_g[warp][i] = (int32_t)g;
    s_r[warp][i] = (T)P.r[g];
  }
  __syncwarp();
  const T* X = fac + P.fac_off[pi];
  T y[R];
#pragma unroll
  for (int k = 0; k < R; ++k) y[k] = (T)0;
#pragma unroll 4
  for (int j = 0; j < np; ++j) {
    const T rj = s_r[warp][j];
    const T* col = X + (int64_t)j * np;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = lane + 32 * k;
      if (i < np) y[k] = fma(__ldcs(col + i), rj, y[k]);  // read once: evict-first
    }
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = lane + 32 * k;
    if (i < np) {
      const int32_t g = s_g[warp][i];
      P.out[g] += P.scale * (double)y[k];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kApplyWarps * 32) k_vanka_apply_t(ApplyParams P, const T* __restrict__ fac) {
  __shared__ T s_r[kApplyWarps][kMaxNp];
  __shared__ int32_t s_g[kApplyWarps][kMaxNp];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kApplyWarps + warp;
  if (w >= P.count) return;
  const int64_t pi = P.first + w;
  const int32_t v = P.order[pi];
  const int32_t nb = P.patch_ptr[v], L = P.patch_ptr[v + 1] - nb;
  const int q = P.dim * L + 1, np = P.s * q;
  for (int i = lane; i < np; i += 32) {
    const int t = i / q, k = i - t * q;
    int64_t g;
    if (k < P.dim * L) {
      const int c = k / L;
      g = t * P.m + c * P.nf + P.patch_nodes[nb + k - c * L];
    } else {
      g = t * P.m + P.dim * P.nf + v;
    }
    s_g[warp][i] = (int32_t)g;
    s_r[warp][i] = (T)P.r[g];
  }
  __syncwarp();
  const T* X = fac + P.fac_off[pi];
  // (Xᵀ r)_i = sum_j X[i*np + j] r_j : column i of the column-major X is contiguous
  for (int i = 0; i < np; ++i) {
    T acc = (T)0;
    for (int j = lane; j < np; j += 32) acc = fma(X[(int64_t)i * np + j], s_r[warp][j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == (i & 31)) P.out[s_g[warp][i]] += P.scale * (double)acc;
  }
}


// ---------------------------------------------------------------------------
// TMA-staged Vanka apply (persistent over the patches of one colour).
// One CTA of kStagedThreads threads works on one patch at a time (thread i owns
// row i, and row i + kStagedThreads when n_p > kStagedThreads).  Each patch
// inverse is one contiguous 16-byte-aligned block, streamed into a ring of
// shared-memory stages by the TMA unit (cp.async.bulk, completion on an
// mbarrier); while the CTA computes patch k from shared memory the copies of
// the next stages are in flight, and their residual entries are gathered by
// plain loads.  Every mbarrier wait is bounded: on expiry the CTA records
// IRKMG_ETIMEOUT, waits (bounded) for its own copies still in flight, and
// returns.
// ---------------------------------------------------------------------------
constexpr int kStagedThreads = 256;
constexpr int kMaxStages = 4;


struct StagedParams {
  ApplyParams a;
  int stages;
  uint32_t stage_bytes;  // bytes per stage (largest patch block, rounded to 128)
  uint32_t rpart_off;    // offset of the gathered residual / partial sums in dynamic smem
  int64_t spins;
  int* err;
};

// One CTA works on one patch at a time.  Thread t owns row (t mod 128) [and
// that row + 128 when n_p > 128] over column half (t / 128); the halves are
// added through shared memory.  The patch block (inverse + index list) arrives
// by one bulk copy; the residual entries are gathered through the index list.
template <typename T>
__global__ void __launch_bounds__(kStagedThreads) k_vanka_apply_staged(StagedParams S, const T* __restrict__ fac) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar[kMaxStages];
  __shared__ int s_abort;
  const ApplyParams& P = S.a;
  T* s_r = reinterpret_cast<T*>(dyn + S.rpart_off);
  T* s_part = s_r + kMaxNp;  // [2][128]
  const int tid = threadIdx.x;
  const int row = tid & 127, half = tid >> 7;
  const int64_t nmine = (P.count > blockIdx.x) ? (P.count - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int st = 0; st < S.stages; ++st) mbar_init(&bar[st], 1);
    s_abort = 0;
  }
  fence_proxy_async();
  __syncthreads();

  auto block_bytes = [](int np) -> uint32_t {
    return (uint32_t)((((int64_t)np * np * (int64_t)sizeof(T) + 15) & ~(int64_t)15) +
                      (((int64_t)np * 4 + 15) & ~(int64_t)15));
  };
  const uint64_t pol = l2_evict_first_policy();
  // thread 0: start the bulk copy of this CTA's k-th patch block into stage st
  auto issue = [&](int64_t k, int st) {
    const int64_t pi = P.first + blockIdx.x + k * gridDim.x;
    const uint32_t bytes = block_bytes(P.np[pi]);
    mbar_expect_tx(&bar[st], bytes);
    bulk_g2s(dyn + (size_t)st * S.stage_bytes, fac + P.fac_off[pi], bytes, &bar[st], pol);
  };
  if (tid == 0) {
    const int64_t pre = nmine < S.stages ? nmine : S.stages;
    for (int64_t k = 0; k < pre; ++k) issue(k, (int)k);
  }

  for (int64_t k = 0; k < nmine; ++k) {
    const int st = (int)(k % S.stages);
    const uint32_t parity = (uint32_t)((k / S.stages) & 1);
    const int64_t pi = P.first + blockIdx.x + k * gridDim.x;
    const int np = P.np[pi];
    if (!mbar_wait_bounded(&bar[st], parity, S.spins)) {
      s_abort = 1;
      atomicCAS(&S.err[0], 0, IRKMG_ETIMEOUT);
    }
    __syncthreads();
    if (s_abort) {
      // wait (bounded) for every copy this CTA still has in flight (patches
      // k .. k + stages - 1 are issued), then leave
      for (int64_t j = k; j < nmine && j < k + S.stages; ++j)
        mbar_drain(&bar[j % S.stages], (uint32_t)((j / S.stages) & 1));
      return;
    }
    const unsigned char* stage = dyn + (size_t)st * S.stage_bytes;
    const T* X = reinterpret_cast<const T*>(stage);
    const int32_t* G = reinterpret_cast<const int32_t*>(
        stage + (((int64_t)np * np * (int64_t)sizeof(T) + 15) & ~(int64_t)15));
    for (int i = tid; i < np; i += kStagedThreads) s_r[i] = (T)P.r[G[i]];
    __syncthreads();
    const int jb = half ? (np >> 1) : 0, je = half ? np : (np >> 1);
    const int r1 = row + 128;
    T a0 = (T)0, b0 = (T)0, a1 = (T)0, b1 = (T)0;
    if (r1 < np) {
      int j = jb;
      for (; j + 1 < je; j += 2) {
        const T x0 = s_r[j], x1 = s_r[j + 1];
        a0 = fma(X[j * np + row], x0, a0);
        b0 = fma(X[(j + 1) * np + row], x1, b0);
        a1 = fma(X[j * np + r1], x0, a1);
        b1 = fma(X[(j + 1) * np + r1], x1, b1);
      }
      if (j < je) {
        a0 = fma(X[j * np + row], s_r[j], a0);
        a1 = fma(X[j * np + r1], s_r[j], a1);
      }
    } else if (row < np) {
      int j = jb;
#pragma unroll 4
      for (; j + 1 < je; j += 2) {
        a0 = fma(X[j * np + row], s_r[j], a0);
        b0 = fma(X[(j + 1) * np + row], s_r[j + 1], b0);
      }
      if (j < je) a0 = fma(X[j * np + row], s_r[j], a0);
    }
    if (half) {
      s_part[row] = a0 + b0;
      if (r1 < np) s_part[128 + row] = a1 + b1;
    }
    __syncthreads();
    if (!half) {
      if (row < np) P.out[G[row]] += P.scale * (double)(a0 + b0 + s_part[row]);
      if (r1 < np) P.out[G[r1]] += P.scale * (double)(a1 + b1 + s_part[128 + row]);
    }
    fence_proxy_async();
    __syncthreads();  // stage st, s_r and s_part fully consumed
    if (tid == 0 && k + S.stages < nmine) issue(k + S.stages, st);
  }
}

// Launch shape of the staged apply for a level: two CTAs per SM when one
// stage each fits, else one CTA with two or more stages; false when neither
// fits (the warp-per-patch kernel is used then).
struct StagedShape {
  int stages, ctas_per_sm;
  uint32_t stage_bytes, rpart_off, dyn_bytes;
};
bool staged_config(int max_np, int prec, StagedShape* out) {
  if (max_np > kMaxNp) return false;
  const size_t w = prec == 64 ? 8 : 4;
  const size_t blk = ((((size_t)max_np * max_np * w + 15) & ~(size_t)15) +
                      (((size_t)max_np * 4 + 15) & ~(size_t)15));
  const size_t sb = (blk + 127) & ~(size_t)127;
  const size_t extra = (kMaxNp + 256) * w;  // gathered residual + partial sums
  const size_t static_b = 128;  // barriers + abort flag (ptxas: 128 bytes)
  const size_t per_sm = 233472, reserved = 1024, per_block = 232448;
  for (int ctas = 2; ctas >= 1; --ctas) {
    const size_t budget = std::min(per_sm / ctas - reserved, per_block) - static_b - extra;
    int st = (int)(budget / sb);
    if (st > kMaxStages) st = kMaxStages;
    if (st >= (ctas == 2 ? 1 : 2)) {
      out->stages = st;
      out->ctas_per_sm = ctas;
      out->stage_bytes = (uint32_t)sb;
      out->rpart_off = (uint32_t)(st * sb);
      out->dyn_bytes = (uint32_t)(st * sb + extra);
      return true;
    }
  }
  return false;
}

bool vanka_staged_fits(Ctx& C, Level& L) {
  StagedShape shp;
  return staged_config(L.max_np, C.opt.patch_precision, &shp);
}

cudaError_t launch_vanka(Ctx& C, Level& L, int colour, const double* r, double* out, double scale,
                         int transpose) {
  ApplyParams P{};
  P.s = C.s;
  P.dim = L.dim;
  P.nf = L.nf;
  P.m = L.m;
  P.patch_ptr = L.d_patch_ptr;
  P.patch_nodes = L.d_patch_nodes;
  P.order = L.d_order;
  P.np = L.d_np;
  P.fac_off = L.d_fac_off;
  P.r = r;
  P.out = out;
  P.scale = scale;
  P.first = L.colour_start[colour];
  P.count = L.colour_start[colour + 1] - P.first;
  if (P.count <= 0) return cudaSuccess;
  const int prec = C.opt.patch_precision;
  StagedShape shp;
  if (!transpose && L.apply_kernel == 1 && staged_config(L.max_np, prec, &shp)) {
    StagedParams S{};
    S.a = P;
    S.stages = shp.stages;
    S.stage_bytes = shp.stage_bytes;
    S.rpart_off = shp.rpart_off;
    S.spins = C.opt.timeout_spins > 0 ? C.opt.timeout_spins : (int64_t)1 << 26;
    S.err = C.d_err;
    const int64_t cap = 152 * shp.ctas_per_sm;
    const int64_t ctas = P.count < cap ? P.count : cap;
    const size_t smem = shp.dyn_bytes;
    if (prec == 64) {
      cudaFuncSetAttribute(k_vanka_apply_staged<double>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_vanka_apply_staged<double><<<(unsigned)ctas, kStagedThreads, smem, C.stream>>>(
          S, (const double*)L.d_fac);
    } else {
      cudaFuncSetAttribute(k_vanka_apply_staged<float>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_vanka_apply_staged<float><<<(unsigned)ctas, kStagedThreads, smem, C.stream>>>(
          S, (const float*)L.d_fac);
    }
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((P.count + kApplyWarps - 1) / kApplyWarps);
  if (transpose) {
    if (prec == 64)
      k_vanka_apply_t<double><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, (const double*)L.d_fac);
    else
      k_vanka_apply_t<float><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, (const float*)L.d_fac);
    return cudaGetLastError();
  }
  const int R = (L.max_np + 31) / 32;
  if (prec == 64) {
    const double* f = (const double*)L.d_fac;
    switch (R) {
      case 1: k_vanka_apply<double, 1><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      case 2: k_vanka_apply<double, 2><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      case 3: k_vanka_apply<double, 3><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      case 4: k_vanka_apply<double, 4><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      default: k_vanka_apply<double, 5><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
    }
  } else {
    const float* f = (const float*)L.d_fac;
    switch (R) {
      case 1: k_vanka_apply<float, 1><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      case 2: k_vanka_apply<float, 2><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      case 3: k_vanka_apply<float, 3><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      case 4: k_vanka_apply<float, 4><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
      default: k_vanka_apply<float, 5><<<grid, kApplyWarps * 32, 0, C.stream>>>(P, f); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace irkmg

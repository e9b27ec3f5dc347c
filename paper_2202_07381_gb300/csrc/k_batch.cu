// Batched relaxation of many independent stage systems in one persistent
// launch: the Chebyshev-accelerated additive Vanka steps (Sections 4.2 and
// 5.1) on the finest level of every system of a batch, each step in three
// phases over the union of the systems' work,
//   A  residual      t = F - J x        (a thread per operator row; on a
//                                        first step from x = 0, t = F),
//   B  patch solves  Y = A_v⁻¹ R_v t     (a warp per patch, fixed point),
//   C  sum + update  c = Σ_v R_vᵀ Y_v, d = ρ'ρ d + (2ρ'/δ) c, x += d
//                                        (a thread per DoF),
// separated by grid-wide barriers.  The launch is cooperative (every CTA
// resident); the CTAs take the work units of a phase in a grid-stride loop,
// and a unit's system is found by a search of the phase's prefix sums.
//
// The phases run the same device functions as the per-system kernels
// (residual_sell_row, fx_patch, the per-DoF sum in contribution order) and
// the rounding steps of the per-system Chebyshev update, so a batch relaxes
// each system bit for bit as the system's own one-launch relaxation does.
//
// Data written during the launch by other CTAs (the iterate, the residual,
// the patch results) is read through L2 only (ld.global.cg).
//
// Every barrier wait is bounded (timeout_spins polls, the first one at once,
// and 2 s of wall time).  A CTA whose wait expires records IRKMG_ETIMEOUT and
// leaves the kernel; the others then expire at that barrier or the next one.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fx_patch.cuh"
#include "irkmg_internal.h"
#include "op_sell.cuh"
#include "tma.cuh"

namespace irkmg {

namespace {

constexpr int kBatchThreads = 32 * kFxWarps;  // one patch per warp in phase B
constexpr int kBatchMaxSys = 128;
constexpr int kBatchMaxSteps = 8;

// One system's finest level (device copy, built per solve).
struct BatchSys {
  OpParams op;       // stage operator J
  FxApply fx;        // patch apply of every patch from t into ybuf
  const int2* fac;   // fixed-point patch blocks
  const int32_t *cptr, *cidx;  // per-DoF contribution lists into ybuf
  const double* ybuf;
  int64_t Q, m, rows, npatch;
  double *t, *d;     // residual, Chebyshev direction
  double c_old[kBatchMaxSteps], c_new[kBatchMaxSteps];  // ρ'ρ and 2ρ'/δ per step (ρ: 1/θ at 0)
};

// One launch: the active systems, their right-hand sides and iterates, and
// the prefix sums of the work units of each phase.
struct BatchLaunch {
  int n;                             // active systems
  int nsteps, zero_init;
  int sys[kBatchMaxSys];             // index into the BatchSys array
  const double* b[kBatchMaxSys];
  double* x[kBatchMaxSys];
  int64_t op_pref[kBatchMaxSys + 1];     // 256 operator rows per unit
  int64_t patch_pref[kBatchMaxSys + 1];  // kFxWarps patches per unit
  int64_t dof_pref[kBatchMaxSys + 1];    // 256 DoFs per unit
  unsigned* bar;
  int64_t spins;
  int* err;
  uint32_t warp_bytes;
  int pair;  // every system in the complex layout's pair structure: paired rows
};

__device__ __forceinline__ int find_unit(const int64_t* pref, int n, int64_t u) {
  int lo = 0, hi = n;  // pref[lo] <= u < pref[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pref[mid] <= u)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Grid-wide barrier on bar[0] (arrivals) and bar[1] (generation), both zero
// before the launch.  False, with IRKMG_ETIMEOUT recorded, if the wait expired.
__device__ bool grid_sync(unsigned* bar, int64_t spins, int* err, int* s_fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();  // this CTA's writes before its arrival
    bool ok = true;
    if (atomicAdd(bar, 1u) + 1 == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      ok = false;
      const uint64_t t0 = global_ns();
      for (int64_t k = 0; k < spins; ++k) {
        if (*gen != g) {
          ok = true;
          break;
        }
        __nanosleep(64);
        if ((k & 255) == 255 && global_ns() - t0 > 2000000000ull) break;
      }
      if (!ok) atomicCAS(err, 0, IRKMG_ETIMEOUT);
    }
    __threadfence();  // the other CTAs' writes before this CTA's reads
    *s_fail = ok ? 0 : 1;
  }
  __syncthreads();
  return *s_fail == 0;
}

// Copies the parameter block of system k into shared memory (all threads of
// the CTA, 8-byte words), so that the work of a unit reads it from there.
template <typename T>
__device__ __forceinline__ void stage_params(T* dst, const T* src, int* s_have, int k) {
  static_assert(sizeof(T) % 8 == 0, "8-byte words");
  if (*s_have == k) return;  // the CTA's previous unit was of the same system
  __syncthreads();           // the previous unit's readers are done
  const uint64_t* s8 = reinterpret_cast<const uint64_t*>(src);
  uint64_t* d8 = reinterpret_cast<uint64_t*>(dst);
  for (int w = threadIdx.x; w < (int)(sizeof(T) / 8); w += blockDim.x) d8[w] = s8[w];
  __syncthreads();
  if (threadIdx.x == 0) *s_have = k;  // read by the next call only after a barrier
}

// Patches outside the paired path (boundary stars; other layouts), out of
// line so that their registers do not count against the paired path's.
__device__ __noinline__ void batch_patch_generic(const FxApply& P, const int2* __restrict__ fac,
                                                 unsigned char* base, int lane, int64_t pi, int np) {
  if (np == kFxN2)
    fx_patch<kFxN2, 1, 4, false, true>(P, fac, base, lane, pi, np);
  else
    fx_patch<0, 1, 4, false, true>(P, fac, base, lane, pi, np);
}

template <int S>
__global__ void __launch_bounds__(kBatchThreads, 3) k_batch_smooth(BatchLaunch R,
                                                                  const BatchSys* __restrict__ sys) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ int s_fail;
  __shared__ __align__(16) OpParams s_op;
  __shared__ __align__(16) FxApply s_fx;
  __shared__ int s_have_op, s_have_fx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = R.n;
  unsigned char* base = dyn + (size_t)warp * R.warp_bytes;
  if (tid == 0) s_have_op = s_have_fx = -1;
  __syncthreads();
  for (int step = 0; step < R.nsteps; ++step) {
    const bool from_zero = step == 0 && R.zero_init;
    // A: t = b - J x (256 operator rows per unit); from x = 0, t = b (256
    // DoFs per unit)
    if (!from_zero) {
      for (int64_t u = blockIdx.x; u < R.op_pref[n]; u += gridDim.x) {
        const int i = find_unit(R.op_pref, n, u);
        const BatchSys& B = sys[R.sys[i]];
        stage_params(&s_op, &B.op, &s_have_op, R.sys[i]);
        const int64_t row = (u - R.op_pref[i]) * kBatchThreads + tid;
        if (row < B.rows) residual_sell_row<S, 2, true>(s_op, row, R.b[i], R.x[i], B.t);
      }
    } else {
      for (int64_t u = blockIdx.x; u < R.dof_pref[n]; u += gridDim.x) {
        const int i = find_unit(R.dof_pref, n, u);
        const BatchSys& B = sys[R.sys[i]];
        const int64_t id = (u - R.dof_pref[i]) * kBatchThreads + tid;
        if (id < (int64_t)S * B.m) B.t[id] = R.b[i][id];
      }
    }
    if (!grid_sync(R.bar, R.spins, R.err, &s_fail)) return;
    // B: every patch from t into the system's result buffer
    for (int64_t u = blockIdx.x; u < R.patch_pref[n]; u += gridDim.x) {
      const int i = find_unit(R.patch_pref, n, u);
      const BatchSys& B = sys[R.sys[i]];
      stage_params(&s_fx, &B.fx, &s_have_fx, R.sys[i]);
      const int64_t k = (u - R.patch_pref[i]) * kFxWarps + warp;
      if (k < B.npatch) {
        const int64_t pi = fx_pi(s_fx, k);  // vertex order, as the one-launch apply
        const int np = s_fx.np[pi];
        if (S >= 2 && R.pair && np == kFxN2)  // complex layout: paired rows
          fx_patch_pair<8, S == 3, true>(s_fx, B.fac, base, lane, pi);
        else
          batch_patch_generic(s_fx, B.fac, base, lane, pi, np);
      }
    }
    if (!grid_sync(R.bar, R.spins, R.err, &s_fail)) return;
    // C: per-DoF sum of the patch results in contribution order, then the
    // Chebyshev update with the per-system rounding steps: d scaled (one
    // product), the sum added by one fma, x += d by one fma
    for (int64_t u = blockIdx.x; u < R.dof_pref[n]; u += gridDim.x) {
      const int i = find_unit(R.dof_pref, n, u);
      const BatchSys& B = sys[R.sys[i]];
      const int64_t id = (u - R.dof_pref[i]) * kBatchThreads + tid;
      if (id < (int64_t)S * B.m) {
        const int64_t t = id / B.m, dd = id - t * B.m;
        const double* yt = B.ybuf + t * B.Q;
        double a = 0.0;
        for (int32_t e = B.cptr[dd]; e < B.cptr[dd + 1]; ++e) a += __ldcg(yt + B.cidx[e]);
        const double d0 = step == 0 ? 0.0 : __dmul_rn(B.c_old[step], __ldcg(B.d + id));
        const double d1 = __fma_rn(B.c_new[step], a, d0);
        B.d[id] = d1;
        double* x = R.x[i];
        x[id] = from_zero ? d1 : __fma_rn(1.0, d1, __dmul_rn(1.0, __ldcg(x + id)));
      }
    }
    if (step + 1 < R.nsteps && !grid_sync(R.bar, R.spins, R.err, &s_fail)) return;
  }
}

template <int S>
cudaError_t launch_t(const BatchLaunch& R, const BatchSys* sys, int ctas, size_t dyn,
                     cudaStream_t st) {
  auto kern = k_batch_smooth<S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  BatchLaunch r = R;
  const BatchSys* p = sys;
  void* args[] = {&r, &p};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)ctas), dim3(kBatchThreads),
                                     args, dyn, st);
}

template <int S>
int max_ctas(size_t dyn, int* out) {
  auto kern = k_batch_smooth<S>;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, dyn);
  if (e != cudaSuccess) return -1;
  *out = nsm * per_sm;
  return 0;
}

}  // namespace

struct BatchPlan {
  std::vector<Ctx*> sys;
  int s = 0;
  BatchSys* d_sys = nullptr;  // device array, one per system
  unsigned* d_bar = nullptr;
  size_t dyn = 0;
  uint32_t warp_bytes = 0;
  int ctas = 0;
  int pair = 0;
};

// Why a batch cannot relax in one persistent launch ("" when it can): every
// system 2D, the same stage count, Chebyshev smoothing with at most
// kBatchMaxSteps steps, a fixed-point decoupled finest level, and at most
// kBatchMaxSys systems.
std::string batch_plan_unsupported(const std::vector<Ctx*>& sys) {
  if (sys.empty() || (int)sys.size() > kBatchMaxSys) return "batch size";
  for (Ctx* C : sys) {
    const Level& L = C->L.back();
    if (C->dim != 2 || C->s != sys[0]->s) return "2D systems of one stage count";
    if (C->opt.smoother != 1 || C->opt.nu_pre < 1 || C->opt.nu_post < 1 ||
        C->opt.nu_pre > kBatchMaxSteps || C->opt.nu_post > kBatchMaxSteps)
      return "Chebyshev smoothing with 1..8 steps";
    if (!L.fixed || (int)C->L.size() < 2) return "fixed-point decoupled finest levels";
    if (C->ns && C->ns_active) return "no Newton blocks";
  }
  return "";
}

int batch_plan_create(const std::vector<Ctx*>& sys, BatchPlan** out) {
  *out = nullptr;
  if (!batch_plan_unsupported(sys).empty()) return IRKMG_ENOTIMPL;
  BatchPlan* P = new (std::nothrow) BatchPlan();
  if (!P) return IRKMG_ENOMEM;
  P->sys = sys;
  P->s = sys[0]->s;
  size_t wb = 0;
  P->pair = 1;
  for (Ctx* C : sys) {
    const Level& L = C->L.back();
    wb = std::max(wb, fx_warp_bytes(C->s, std::max(C->kplan.ns, C->kplan.nt), C->kplan.nt,
                                    L.kron_nmax));
    bool real = false;
    if (!fx_pair_plan(C->kplan, &real) || real != (P->s == 3)) P->pair = 0;
  }
  if (P->pair) wb = std::max(wb, sizeof(FxPairSmem));
  P->warp_bytes = (uint32_t)wb;
  P->dyn = (size_t)kFxWarps * wb;
  int rc = P->s == 3 ? max_ctas<3>(P->dyn, &P->ctas)
                     : P->s == 2 ? max_ctas<2>(P->dyn, &P->ctas) : max_ctas<1>(P->dyn, &P->ctas);
  if (rc != 0 || P->ctas < 1 ||
      cudaMalloc(&P->d_sys, sizeof(BatchSys) * sys.size()) != cudaSuccess ||
      cudaMalloc(&P->d_bar, sizeof(unsigned) * 2) != cudaSuccess) {
    batch_plan_destroy(P);
    return IRKMG_ECUDA;
  }
  *out = P;
  return IRKMG_OK;
}

void batch_plan_destroy(BatchPlan* P) {
  if (!P) return;
  if (P->d_sys) cudaFree(P->d_sys);
  if (P->d_bar) cudaFree(P->d_bar);
  delete P;
}

// Upload the systems' finest-level data and Chebyshev coefficients (they
// follow irkmg_update, irkmg_set_wind and the Chebyshev interval).
int batch_plan_refresh(BatchPlan* P, cudaStream_t st) {
  std::vector<BatchSys> h(P->sys.size());
  for (size_t i = 0; i < P->sys.size(); ++i) {
    Ctx& C = *P->sys[i];
    Level& L = C.L.back();
    BatchSys& B = h[i];
    B.op = op_params(C, L, 0);
    B.fx = fx_params(C, L, -1, L.t, nullptr, 1.0, 0);
    B.fac = (const int2*)L.d_fac;
    B.cptr = L.d_cptr;
    B.cidx = L.d_cidx;
    B.ybuf = C.d_Y;
    B.Q = L.Q;
    B.m = L.m;
    B.rows = (L.nf + 31) / 32 * 32 + L.nv;
    B.npatch = L.nv;
    B.t = L.t;
    B.d = L.d;
    // the per-system smoother's coefficients: step 0 scales by 1/θ, step k by
    // 2ρ_k/δ after d *= ρ_k ρ_{k-1}, ρ_0 = δ/θ, ρ_k = 1/(2θ/δ - ρ_{k-1})
    const double theta = 0.5 * (L.cheb_hi + L.cheb_lo);
    const double delta = 0.5 * (L.cheb_hi - L.cheb_lo);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    B.c_old[0] = 0.0;
    B.c_new[0] = 1.0 / theta;
    for (int k = 1; k < kBatchMaxSteps; ++k) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      B.c_old[k] = rho_new * rho;
      B.c_new[k] = 2.0 * rho_new / delta;
      rho = rho_new;
    }
  }
  cudaError_t e = cudaMemcpyAsync(P->d_sys, h.data(), sizeof(BatchSys) * h.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // h goes out of scope
  return e == cudaSuccess ? IRKMG_OK : IRKMG_ECUDA;
}

// nsteps relaxation steps on J_i x_i = b_i for the active systems, in one
// cooperative launch on st.
cudaError_t batch_plan_smooth(BatchPlan* P, const std::vector<int>& active,
                              const std::vector<const double*>& b, const std::vector<double*>& x,
                              int nsteps, bool zero_init, int64_t spins, int* err,
                              cudaStream_t st) {
  if (active.empty() || nsteps <= 0) return cudaSuccess;
  BatchLaunch R{};
  R.n = (int)active.size();
  R.nsteps = nsteps;
  R.zero_init = zero_init ? 1 : 0;
  R.op_pref[0] = R.patch_pref[0] = R.dof_pref[0] = 0;
  for (int k = 0; k < R.n; ++k) {
    const int i = active[k];
    const Ctx& C = *P->sys[i];
    const Level& L = C.L.back();
    R.sys[k] = i;
    R.b[k] = b[k];
    R.x[k] = x[k];
    const int64_t rows = (L.nf + 31) / 32 * 32 + L.nv;
    R.op_pref[k + 1] = R.op_pref[k] + (rows + kBatchThreads - 1) / kBatchThreads;
    R.patch_pref[k + 1] = R.patch_pref[k] + (L.nv + kFxWarps - 1) / kFxWarps;
    R.dof_pref[k + 1] = R.dof_pref[k] + ((int64_t)C.s * L.m + kBatchThreads - 1) / kBatchThreads;
  }
  R.bar = P->d_bar;
  R.spins = spins > 0 ? spins : (int64_t)1 << 26;
  R.err = err;
  R.warp_bytes = P->warp_bytes;
  R.pair = P->pair;
  cudaError_t e = cudaMemsetAsync(P->d_bar, 0, sizeof(unsigned) * 2, st);
  if (e != cudaSuccess) return e;
  const int64_t most = std::max(R.patch_pref[R.n], std::max(R.op_pref[R.n], R.dof_pref[R.n]));
  const int ctas = (int)std::min<int64_t>(P->ctas, most);
  return P->s == 3 ? launch_t<3>(R, P->d_sys, ctas, P->dyn, st)
                   : P->s == 2 ? launch_t<2>(R, P->d_sys, ctas, P->dyn, st)
                               : launch_t<1>(R, P->d_sys, ctas, P->dyn, st);
}

}  // namespace irkmg

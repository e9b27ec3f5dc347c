// Internal declarations of the irkmg library (host set-up structures, device
// level data and kernel launchers).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/irkmg.h"

namespace irkmg {

// ---------------------------------------------------------------------------
// Host-side mesh level (Section 4.1: uniform refinements of a coarsest mesh;
// Section 3.1: Taylor–Hood P2–P1 numbering).
// ---------------------------------------------------------------------------
struct HostMesh {
  int dim = 2;                      // 2: triangles, 3: tetrahedra
  int64_t nv = 0, nc = 0, ne = 0, np2 = 0, nf = 0;
  std::vector<double> xy;           // nv*dim
  std::vector<int32_t> cells;       // nc*(dim+1)
  std::vector<uint8_t> bnd;         // nv, Dirichlet vertex flags
  std::vector<int32_t> edges;       // ne*2, sorted pairs, lexicographic
  std::vector<int32_t> cell_edges;  // nc*nle: local edges (0,1),(1,2),(0,2)[,(0,3),(1,3),(2,3)]
  int nvc() const { return dim + 1; }             // vertices per cell
  int nle() const { return dim == 2 ? 3 : 6; }    // edges per cell
  int nn() const { return nvc() + nle(); }        // P2 nodes per cell
  std::vector<uint8_t> edge_dir;    // ne, Dirichlet edge flags
  std::vector<int32_t> p2_to_free;  // np2, -1 on Dirichlet nodes
  std::vector<int32_t> free_to_p2;  // nf
  std::vector<int32_t> vc_ptr, vc_idx;  // vertex -> cells (ascending)
  std::vector<int32_t> vv_ptr, vv_idx;  // vertex -> vertices through edges (ascending)
};

// Returns an empty string on success, else the reason.
std::string build_mesh(const double* xy, const int64_t* cells, const uint8_t* bnd, int64_t nv,
                       int64_t nc, int dim, HostMesh& out);
extern const int kLocalEdges[6][2];
void refine_mesh(const HostMesh& c, HostMesh& f);
// Edge id of the sorted pair (a, b), or -1.
int64_t find_edge(const HostMesh& m, int32_t a, int32_t b);

struct HostCSR {
  int64_t nrows = 0, ncols = 0;
  std::vector<int32_t> ptr, col;
  std::vector<double> v[3];
  int64_t nnz() const { return (int64_t)col.size(); }
};

// Transfer between coarse level c and its red refinement f (Section 4.1:
// canonical P2 / P1 interpolation, free nodes only).
void build_prolongation(const HostMesh& c, const HostMesh& f, HostCSR& Pu, HostCSR& Pp);
HostCSR transpose_csr(const HostCSR& A, int nvals);
// Host threads for the set-up loops: IRKMG_HOST_THREADS if set (1..64), else
// the hardware concurrency (at most 64).  No result depends on the count.
unsigned host_threads();

// Assembled free-DoF operators of one level (Section 3.1).  Values per
// velocity component d are in v[d] of the B structures (d < dim).
struct HostOps {
  HostCSR vel;   // nf x nf: v[0] = M, v[1] = nu K (+ C), v[2] = transpose of v[1]
  HostCSR mall;  // nf x np2: v[0] = M, v[1] = nu K (+ C), with every column (for M f, K u)
  HostCSR btall; // nv x np2: v[d] = B_d^T with every velocity column
  HostCSR b;     // nf x nv : v[d] = B_d   (B = -int psi_q d phi_a / dx_d)
  HostCSR bt;    // nv x nf : v[d] = B_d^T
};
// wind: np2*2 nodal values or nullptr
void assemble_level(const HostMesh& m, double nu, const double* wind, HostOps& ops);

void assemble_cell_load(const HostMesh& m, HostCSR& C);

// Radau IIA closed forms.
int radau_iia(int s, double* A, double* b, double* c);
int gauss_tableau(int s, double* A, double* b, double* c);
int lobatto_iiic_tableau(int s, double* A, double* b, double* c);

// Real block diagonalisation A = T D T⁻¹ of the Butcher matrix (s ≤ 3): D has
// 1×1 blocks (real eigenvalues) and 2×2 blocks [[α, β], [−β, α]] (pairs α ± iβ);
// block b covers columns col0[b] .. col0[b] + blk_size[b] − 1 of T.
constexpr int kKronMaxTasks = 6;
constexpr int kKronMaxSrc = 6;
struct KronSplit {
  int s, nblk;
  int blk_size[3], col0[3];
  double blk[3][4];  // row-major blk_size x blk_size
  double T[9], Tinv[9];
};
// Apply plan of the decoupled patch solve (host_kron.cpp): ns source vectors
// src_c = Σ_t G[c][t] r_t, nt tasks acc_τ = M_{task_mat[τ]} src_{task_src[τ]},
// and x_t = Σ_τ H[t][τ] acc_τ; nm stored n×n matrices per patch.
struct KronPlan {
  int s, layout, nblk, ns, nt, nm;
  int blk_size[3], blk_kind[3], blk_mat[3];  // kind 0 real, 1 (X, Y), 2 (X + Y, X, Y)
  double blk[3][4];
  double G[kKronMaxSrc * 3];
  double H[3 * kKronMaxTasks];
  int task_mat[kKronMaxTasks], task_src[kKronMaxTasks];
};
int kron_split(int s, const double* A, KronSplit* out);
// Eigenvalues of the n x n upper Hessenberg H (row-major), wr + i wi.
int hessenberg_eigvals(int n, const double* H, double* wr, double* wi);
int kron_plan(const KronSplit& K, int layout, KronPlan* out);
// Whether the plan is the complex layout in the order the paired applies are
// written for (the pair first: X, Y = 0, 1, tasks X·w1, X·w2, Y·w1, Y·w2 on
// sources 0, 1; then, for s = 3, the real block 2 with task 4 on source 2);
// *real = 1 with the real block.  k_patch_fixed.cu.
bool fx_pair_plan(const KronPlan& K, bool* real);

// ---------------------------------------------------------------------------
// Device data.
// ---------------------------------------------------------------------------
struct DevCSR {
  int32_t nrows = 0;
  int64_t nnz = 0;
  int32_t* ptr = nullptr;
  int32_t* col = nullptr;
  double* v[3] = {nullptr, nullptr, nullptr};
};

// Sliced ELLPACK with slices of 32 rows: entry k of row r sits at
// ptr[r/32] + 32 k + r%32 (column-major inside a slice), padded with zero
// values on the row's own last column, so a warp reads every entry coalesced.
struct DevSELL {
  int32_t nrows = 0;
  int64_t* ptr = nullptr;  // nslices + 1 offsets
  int32_t* col = nullptr;
  double* v[3] = {nullptr, nullptr, nullptr};
  int64_t stored = 0;
};

// Fixed-point copies of a level's SELL operator for the exact stage operator
// (k_op_fixed.cu): 57-bit rows as (low, high) int32 limbs with one row
// exponent per matrix (Bᵀ: both components under one), and the work arrays
// of one application (x as 58-bit limbs; the block maxima of x).
struct FxOpLevel {
  int2 *qM = nullptr, *qK = nullptr, *qB[2] = {nullptr, nullptr}, *qT[2] = {nullptr, nullptr};
  int16_t *eM = nullptr, *eK = nullptr, *eB[2] = {nullptr, nullptr}, *eT = nullptr;
  int2* xl = nullptr;
  unsigned long long* bmax = nullptr;
};

struct Level {
  HostMesh mesh;
  int dim = 2;
  int64_t nf = 0, nv = 0, np2 = 0, m = 0, N = 0;
  HostOps hops;
  DevCSR vel, b, bt, mall, btall;
  DevSELL svel, sb, sbt;  // SELL copies of vel, b and bt for the stage operator
  bool fxop_on = false;   // the exact fixed-point stage operator (op_fixed)
  FxOpLevel fxop;
  // transfer from level-1 into this level (l > 0), SELL-32 with col −1 after
  // the end of a row
  DevSELL pu, put, pp, ppt;
  // topology for patch construction
  int32_t *d_cells = nullptr, *d_cell_edges = nullptr, *d_vc_ptr = nullptr, *d_vc_idx = nullptr;
  int32_t *d_vv_ptr = nullptr, *d_vv_idx = nullptr, *d_p2_to_free = nullptr;
  // patches (Section 4.2)
  int32_t *d_patch_ptr = nullptr, *d_patch_nodes = nullptr;
  std::vector<int32_t> h_patch_ptr, h_patch_nodes, h_colour;
  int32_t* d_colour = nullptr;
  int ncolours = 0;
  std::vector<int64_t> colour_start;   // into the colour-ordered patch list
  int32_t* d_order = nullptr;          // patches sorted by (colour, id)
  int64_t* d_fac_off = nullptr;        // element offset of each ordered patch's block
  int32_t* d_np = nullptr;             // n_p of each ordered patch
  void* d_fac = nullptr;
  int64_t fac_elems = 0;
  int max_np = 0;
  bool big = false;                    // patches above kMaxSmallNp: blocked LU + LU apply
  bool kron = false;                   // Kronecker-decoupled patch factors (KronPlan)
  bool kron_big = false;               // ... factored by the blocked LU (blocks above 160 DoFs)
  int kron_nmax = 0;                   // largest spatial patch size n on a decoupled level
  bool fixed = false;                  // decoupled FP64 blocks stored as per-row fixed point
  int16_t* d_fexp = nullptr;           // ... their row exponents [ordered patch][matrix][nmax]
  int apply_kernel = 1;                // 1 staged, 2 warp-per-patch, 3 big-patch mat-vec,
                                       // 4 decoupled warp-per-patch, 5 decoupled staged,
                                       // 6 decoupled CTA-per-patch (large patches),
                                       // 7 decoupled warp-specialised TMA pipeline,
                                       // 8 decoupled fixed point, warp per patch,
                                       // 9 decoupled fixed point, TMA-staged
  float apply_ms[3] = {0, 0, 0};       // autotuner timings of one sweep per kernel
  int kron_shape = 0;                  // launch shape of the staged decoupled apply (0, 1)
  double cheb_lo = 2.0, cheb_hi = 8.0; // Chebyshev interval of this level's smoother
  // one-launch relaxation of a decoupled level: patch results to Ctx::d_Y at
  // t·Q + qoff[p] + i·ystride, then the per-DoF sum over the contribution
  // lists.  Warp-per-patch levels: row-major over (local row i, patch vertex
  // v), qoff[p] = v and ystride = the vertex count rounded up to 32, so that
  // consecutive vertices' results for one local row are adjacent, and the
  // launch takes the patches in vertex order (d_perm: ordered index of
  // vertex v's patch).  Large-patch (3D) levels: each patch's results
  // contiguous (qoff[p] = Σ n over the patches before it, ystride 1), the
  // patches in colour order (d_perm null).
  bool single = false;
  int64_t Q = 0;                       // stage stride of d_Y: n_max · ystride
  int64_t Qent = 0;                    // Σ n over the patches
  int64_t ystride = 1;
  int64_t* d_qoff = nullptr;           // per ordered patch: its vertex (large patches: Σ n before it)
  int32_t* d_perm = nullptr;           // per vertex: ordered index of its patch
  int32_t *d_cptr = nullptr, *d_cidx = nullptr;  // spatial DoF -> entries qoff[p] + i·ystride
  double reduce_bytes = 0.0;           // algorithmic bytes of one reduction launch
  double factor_flops = 0.0;           // explicit inverses of the patch blocks: 2 m³ per block
  int kron_cap[2][2] = {{0, 0}, {0, 0}};  // its resident CTAs per [shape][transpose] (0 unset)
  int ws_cap[2] = {0, 0};              // resident CTAs of the warp-specialised apply
  int fx_cap[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // ... of the staged fixed-point apply per shape
  // work vectors (length N)
  double *r = nullptr, *z = nullptr, *t = nullptr, *d = nullptr;
  // Navier-Stokes Newton blocks W_t,dc per stage (2D): CSR-ordered on the
  // velocity pattern (gathers, coarse build) and SELL-ordered (stage operator)
  double* d_ns_csr[3][4] = {{nullptr}};
  double* d_ns_sell[3][4] = {{nullptr}};
  // topology for the GPU assembly of the Newton blocks
  double* d_xy = nullptr;                        // vertex coordinates
  int32_t *d_nc_ptr = nullptr, *d_nc_idx = nullptr;  // P2 node -> cells
  int32_t* d_free_to_p2 = nullptr;
  int64_t* d_sell_perm = nullptr;                // SELL slot of every velocity CSR entry
  // algorithmic bytes for tracing
  std::vector<double> colour_bytes, colour_flops;
  double op_bytes = 0.0, op_flops = 0.0;
};

struct Ctx {
  int s = 0;
  int dim = 2;
  double A[9] = {0}, AT[9] = {0}, b[3] = {0}, c[3] = {0};
  double dt = 0, nu = 1;
  irkmg_options opt{};
  KronPlan kplan{};
  bool kron = false;          // decoupled patch solves requested and the tableau splits
  double* d_Y = nullptr;      // s · max Q patch results of the one-launch relaxation
  bool ns = false;            // Navier-Stokes Newton blocks set (irkmg_ns_set_state)
  bool ns_active = true;      // ... and included in the stage operator (off: Stokes part)
  double* d_ns_g = nullptr;   // s x 2 nf: C(U_i) U_i on the finest free rows
  double* d_ns_U = nullptr;   // s x 2 x np2: stage velocities at every finest P2 node
  cudaStream_t stream = nullptr;
  std::vector<double> wind;  // finest-level nodal wind (empty for Stokes)
  std::vector<Level> L;
  std::vector<void*> allocs;
  // coarse bordered inverse, row-major n_b x n_b
  double* d_coarse_inv = nullptr;
  int64_t nb = 0;
  int32_t* d_coarse_perm = nullptr;
  // FGMRES storage (finest level)
  double *d_V = nullptr, *d_Z = nullptr, *d_w = nullptr, *d_part = nullptr, *d_h = nullptr;
  double* h_h = nullptr;  // pinned
  int restart_alloc = 0;
  int* d_err = nullptr;   // device error word: [0] status, [1] index
  int64_t dev_bytes = 0;
  int* h_err = nullptr;    // pinned mirror of d_err
  // time stepping and adjoint (finest level)
  DevCSR cload, cloadt;    // P0 cell load C (nf x nc) and its transpose
  double *d_F = nullptr, *d_kb = nullptr, *d_lam = nullptr, *d_scalar = nullptr;
  // tracing
  int64_t launches = 0;
  bool trace_on = false;
  // CUDA graph of one V-cycle from d_gin to d_gout (batched solves)
  cudaGraphExec_t vgraph = nullptr;
  // CUDA graphs of the coarse part of the V-cycle (levels 0 .. nl-2, from
  // L[nl-2].r to L[nl-2].z; [0] J, [1] Jᵀ), launched on gstream between events
  cudaGraphExec_t cgraph[2] = {nullptr, nullptr};
  int64_t cgraph_launches[2] = {0, 0};
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  bool capturing = false;
  double *d_gin = nullptr, *d_gout = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_class;       // 0 vanka, 1 operator (one per event pair)
  std::vector<double> ev_bytes, ev_flops;
  size_t ev_used = 0;
};

// Launchers (all on ctx stream).  Each returns cudaGetLastError().
cudaError_t launch_patch_maps(Level& L, cudaStream_t st, int maxnodes, int32_t* d_tmp,
                              int32_t* d_cnt);
cudaError_t launch_compact_patches(Level& L, cudaStream_t st, int maxnodes, const int32_t* d_tmp,
                                   const int32_t* d_cnt);
cudaError_t launch_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
cudaError_t launch_colour_round(Level& L, cudaStream_t st, int* d_remaining, int* d_overflow);
cudaError_t launch_patch_invert(Ctx& C, Level& L, int precision);
cudaError_t launch_patch_gidx(Ctx& C, Level& L);
cudaError_t launch_patch_invert_kron(Ctx& C, Level& L);
cudaError_t launch_patch_gidx_kron(Ctx& C, Level& L);
cudaError_t launch_vanka_kron(Ctx& C, Level& L, int colour, const double* r, double* out,
                              double scale, int transpose);  // colour -1: all patches to d_Y
// A Chebyshev step fused into the per-DoF sum (one-launch relaxation): with
// c the summed patch corrections, d ← (dzero ? 0 : c1·d) + scale·c and then
// x ← d (xadd false) or x ← x + d, each operation rounded as the separate
// axpby / sum / axpby launches round it.
struct ChebFuse {
  double c1;
  bool dzero, xadd;
  double* x;
};
cudaError_t launch_vanka_reduce(Ctx& C, Level& L, double* out, double scale,
                                const ChebFuse* f = nullptr);
int kron_max_slots();
bool fixed_fits(Ctx& C, Level& L);
int fixed_shapes();  // launch shapes of the fixed-point apply (Level::kron_shape):
                     // 0..3 warp per patch, 4.. TMA-staged
int fixed_shape_kernel(int shape);  // 8: warp per patch, 9: TMA-staged
bool fixed_shape_fits(Ctx& C, Level& L, int shape);
cudaError_t launch_patch_to_fixed(Ctx& C, Level& L);
cudaError_t launch_vanka_kron_fx(Ctx& C, Level& L, int colour, const double* r, double* out,
                                 double scale, int transpose);
bool kron_staged_fits(Ctx& C, Level& L, int shape);
bool kron_ws_fits(Ctx& C, Level& L);
cudaError_t launch_vanka(Ctx& C, Level& L, int colour, const double* r, double* out, double scale,
                         int transpose);
bool vanka_staged_fits(Ctx& C, Level& L);
cudaError_t launch_residual(Ctx& C, Level& L, const double* F, const double* x, double* r,
                            int transpose);
bool op_fixed_fits(Ctx& C, Level& L);
cudaError_t launch_op_fixed_convert(Ctx& C, Level& L);
cudaError_t launch_residual_fx(Ctx& C, Level& L, const double* F, const double* x, double* r);
cudaError_t launch_restrict(Ctx& C, Level& Lf, const double* fine, double* coarse);
cudaError_t launch_prolong(Ctx& C, Level& Lf, const double* coarse, double* fine, int add);
cudaError_t launch_axpby(double* y, const double* x, double a, double b, int64_t n,
                         cudaStream_t st);  // y = a*x + b*y
cudaError_t launch_fill(double* y, double v, int64_t n, cudaStream_t st);
cudaError_t launch_fill_sin(double* y, int64_t n, cudaStream_t st);  // y_i = sin(i + 1)
cudaError_t launch_multidot(const double* V, int64_t ldv, int k, const double* w, int64_t n,
                            double* part, double* out, cudaStream_t st);
cudaError_t launch_multiaxpy(double* w, const double* V, int64_t ldv, int k, const double* h,
                             double sign, int64_t n, cudaStream_t st);
// w += sign·V h fused with the next reduction (Vᵀ w into out[0..k), or
// ‖w‖² into out[0] when norm): bitwise launch_multiaxpy then launch_multidot.
cudaError_t launch_multiaxpy_dot(double* w, const double* V, int64_t ldv, int k, const double* h,
                                 double sign, int64_t n, double* part, double* out, bool norm,
                                 cudaStream_t st);  // w += sign * V h
cudaError_t launch_pressure_mean_remove(Ctx& C, Level& L, double* x);
cudaError_t launch_stage_rhs(Ctx& C, const double* un, const double* pn, const double* f,
                             double* F);
cudaError_t launch_advance(Ctx& C, const double* k, double* un, double* pn);
cudaError_t launch_stage_rhs_full(Ctx& C, const double* un_all, const double* pn, const double* f,
                                  double* F);
cudaError_t launch_coarse_build(Ctx& C, double* dense);
cudaError_t coarse_invert(Ctx& C, double* dense, int64_t n);
cudaError_t launch_coarse_apply(Ctx& C, const double* r, double* x, int transpose);

cudaError_t launch_cell_load(Ctx& C, const double* theta, double* g);
cudaError_t launch_ns_stage_velocity(Ctx& C, const double* un_all, const double* k, double* U);
cudaError_t launch_ns_assemble(Ctx& C, Level& L, int t, const double* U, int64_t stride, double* g);
cudaError_t launch_add_to_stages(Ctx& C, const double* g, double* F);
cudaError_t launch_kbar(Ctx& C, const double* ub, const double* pb, double* kb);
cudaError_t launch_adjoint_update(Ctx& C, const double* lam, double* ub, double* pb);
cudaError_t launch_theta_bar(Ctx& C, const double* lam, double* thb);
cudaError_t launch_dnu(Ctx& C, const double* lam, const double* k, const double* un, double* part,
                       double* out);
cudaError_t launch_tracking(Ctx& C, const double* u, const double* ut, double* grad, double* part,
                            double* out);

cudaError_t launch_patch_lu_big(Ctx& C, Level& L);
cudaError_t launch_patch_inv_from_lu(Ctx& C, Level& L, void* work, int64_t ws, int ctas);
cudaError_t launch_vanka_big(Ctx& C, Level& L, int colour, const double* r, double* out,
                             double scale);
cudaError_t launch_patch_factor_kron_big(Ctx& C, Level& L, void* work, int64_t ws, int ctas);
int64_t kron_big_workspace(int pmax, int nmax, int prec);
int kron_big_max_n();

// Batched relaxation of the finest levels of many systems in one persistent
// launch (k_batch.cu).  batch_plan_unsupported gives why a set of systems
// cannot use it ("" when it can).
struct BatchPlan;
std::string batch_plan_unsupported(const std::vector<Ctx*>& sys);
int batch_plan_create(const std::vector<Ctx*>& sys, BatchPlan** out);
void batch_plan_destroy(BatchPlan* P);
int batch_plan_refresh(BatchPlan* P, cudaStream_t st);
cudaError_t batch_plan_smooth(BatchPlan* P, const std::vector<int>& active,
                              const std::vector<const double*>& b, const std::vector<double*>& x,
                              int nsteps, bool zero_init, int64_t spins, int* err,
                              cudaStream_t st);

constexpr int kMultidotBlocks = 304;
constexpr int kMaxSmallNp = 160;  // patches up to this size: explicit inverse in shared memory
constexpr int kMaxBigNp = 512;    // patches up to this size: blocked LU in the patch block  // 2 x 152 SMs; fixed for a deterministic sum order

}  // namespace irkmg

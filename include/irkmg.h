/*
 * irkmg — monolithic multigrid for fully implicit Runge–Kutta stage systems of
 * incompressible (Stokes / Oseen) flow on one NVIDIA GB300 GPU (sm_103a).
 *
 * The method is that of Abu-Labdeh, MacLachlan & Farrell, "Monolithic multigrid
 * for implicit Runge–Kutta discretizations of incompressible fluid flow"
 * (arXiv:2202.07381):
 *   - the stage system (Section 3.1, Kronecker form)
 *       ( I_s ⊗ [[M,0],[0,0]] + dt·A ⊗ [[K,B],[Bᵀ,0]] ) k = F,
 *     Taylor–Hood P2–P1 on triangles, K = nu·(P2 stiffness) [+ Oseen convection],
 *     B the weak gradient from −<p, div v>;
 *   - FGMRES as the outer Krylov method (Section 4);
 *   - a geometric V-cycle with rediscretised coarse operators, I_s⊗P transfers,
 *     restriction Pᵀ and a direct coarsest solve (Section 4.1);
 *   - additive vertex-star Vanka relaxation with all s stages in every patch
 *     (Section 4.2), damped or Chebyshev-accelerated (Section 5.1).
 *
 * Vector layout (every d_* vector of a level): stage-major, length
 * N = s·(d·nf + nv); inside a stage the u_x block over the nf free
 * (non-Dirichlet) P2 nodes, then the u_y block (then u_z in 3D), then the
 * pressure block over all nv vertices.  This is the ordering of Section 3.1 (stages consecutive,
 * each (k_u, k_p) pair kept together).
 *
 * Numbering: mesh edges are the sorted vertex pairs in lexicographic order;
 * P2 nodes are the vertices followed by the edge midpoints; free P2 nodes keep
 * that order.  Refinement keeps coarse vertex ids and appends one vertex per
 * coarse edge, so the P2 nodes of level l are the vertices of level l+1.
 *
 * Ownership: host arrays passed to a call are read during the call only.  All
 * d_* pointers are caller-owned device pointers (e.g. the data pointer of a
 * contiguous float64 CUDA tensor), read and written on the context's stream
 * (irkmg_options.cuda_stream).  The context owns every device buffer it
 * allocates (matrices, patch inverses, Krylov basis) and frees them in
 * irkmg_destroy.
 *
 * Errors: every int-returning call returns one of the IRKMG_* codes below;
 * nothing aborts, traps or throws across this interface.  irkmg_last_error()
 * gives a one-line description of the most recent failure on the calling
 * thread.
 */
#ifndef IRKMG_H
#define IRKMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define IRKMG_OK 0
#define IRKMG_EINVAL 1     /* bad sizes/arguments, inconsistent tableau, bad mesh  */
#define IRKMG_ENOMEM 2     /* device or host allocation failed                      */
#define IRKMG_ECUDA 3      /* a CUDA runtime call or kernel launch failed          */
#define IRKMG_ESINGULAR 4  /* a patch or coarse pivot fell below 1e3·eps·max|A|    */
#define IRKMG_ENOCONV 5    /* FGMRES hit maxit; the best iterate is written        */
#define IRKMG_ETIMEOUT 6   /* a bounded device wait expired                        */
#define IRKMG_ENOTIMPL 7   /* the requested form is not built                      */

typedef struct irkmg_ctx irkmg_ctx;

/* Coarsest mesh (Section 4.1: the hierarchy is its uniform refinements).
 * dim = 2: triangles (red refinement); dim = 3: tetrahedra (Bey refinement).
 * coords: nverts·dim doubles; cells: ncells·(dim+1) vertex ids; bnd_vertex: 1
 * on Dirichlet (no-slip) vertices.  An edge is Dirichlet iff it lies on a
 * boundary facet and both ends are flagged.  In 3D, vectors hold u_x, u_y and
 * u_z blocks before the pressure block; patches above 160 DoFs are inverted
 * through a blocked LU on the GPU (their transposed solves, the Oseen wind and
 * the adjoint entry points return IRKMG_ENOTIMPL in 3D). */
typedef struct {
  int dim;
  int64_t nverts, ncells;
  const double *coords;
  const int64_t *cells;
  const uint8_t *bnd_vertex;
} irkmg_mesh;

/* Butcher tableau (Section 2): A row-major s×s, b and c of length s.
 * irkmg_setup checks sum_j b_j = 1 and sum_j a_ij = c_i to 1e-12. */
typedef struct {
  int s;
  const double *A, *b, *c;
} irkmg_tableau;

/* Solver options; irkmg_default_options fills the paper's 2D Stokes choices
 * (Section 5.1): V(2,2), Chebyshev on [2, 8], FGMRES restart 30. */
typedef struct {
  int nlevels;             /* levels including the coarsest (>= 2)                  */
  int nu_pre, nu_post;     /* relaxation steps before / after the coarse correction */
  int smoother;            /* 0: damped additive Vanka (omega); 1: Chebyshev        */
  double omega;            /* damping of smoother 0                                 */
  double cheb_lo, cheb_hi; /* Chebyshev interval of smoother 1                      */
  double rtol, atol;       /* stop when ||F - J k|| <= max(rtol ||F||, atol)        */
  int restart, maxit;      /* FGMRES(restart), at most maxit iterations in total    */
  int patch_precision;     /* 64: FP64 patch inverses; 32: FP32 inverses + applies  */
  const double *wind;      /* host, finest-level Oseen wind at every P2 node,
                              np2·2 doubles (x, y per node), or NULL for Stokes     */
  void *cuda_stream;       /* cudaStream_t to run on; NULL = legacy default stream  */
  int64_t timeout_spins;   /* bound on polls of one device-side wait (0 = 2^26; the
                              first poll returns at once, later ones may suspend
                              the thread briefly; each wait also gives up after
                              2 s); an expired wait makes FGMRES return
                              IRKMG_ETIMEOUT                                        */
  int apply_variant;       /* Vanka apply kernel per level (dense or decoupled form
                              alike): 0 = autotuned at set-up (every candidate
                              timed once per level, the fastest kept); 1 = TMA-
                              staged (patch blocks streamed to shared memory by
                              cp.async.bulk) wherever it fits; 2 = warp-per-patch
                              mat-vec everywhere; 3, 4 = as 1, 2 and, on decoupled
                              levels, one launch over all patches whose results
                              are summed per DoF by a second, deterministic
                              launch (instead of one launch per colour); 5, 6 =
                              on decoupled levels the warp-specialised TMA
                              pipeline (one producer warp, seven consumer warps
                              each working on whole patches), per colour / one
                              launch; elsewhere as 1                               */
  int patch_form;          /* 0 = one dense s·n patch system per vertex (Section 4.2);
                              1..3 = Kronecker-decoupled patch solves: with the
                              Butcher matrix A = T D T⁻¹ (D real block diagonal,
                              2×2 blocks for complex eigenvalue pairs) every patch
                              system I⊗M̃ + Δt A⊗K̃ splits into one n×n system per
                              real eigenvalue and one complex n×n system per pair
                              (the Kronecker form of Section 3), stored as s n×n
                              matrices (2: complex form X, Y) or s + pairs of them
                              (3: X + Y, X, Y, three real mat-vecs per pair);
                              1 picks 2 for FP32 patches and for 2D FP64 patches
                              with patch_fixed = 1 (their applies are bound by
                              memory traffic), 3 otherwise (fewest FP64
                              multiply-adds).  Exact in
                              exact arithmetic.  Blocks up to 160 DoFs are
                              inverted in shared memory, larger ones (3D, up to
                              512) by the blocked LU; with decoupling, 3D works
                              for s = 3 too (dense: 588 DoFs, above the limit).
                              IRKMG_ENOTIMPL if A has a repeated eigenvalue.       */
  int cheb_auto;           /* 1: per level, the Chebyshev interval [λ/4, λ] with λ the
                              largest real Ritz value of 20 Arnoldi steps on the
                              Vanka-preconditioned operator of that level, found at
                              set-up and on every update (Section 5.1's estimate);
                              0: [cheb_lo, cheb_hi] on every level                 */
  int patch_lu_tc;         /* FP32 patches above 160 DoFs (3D): 1 = trailing updates
                              of the blocked patch LU on the tensor cores
                              (tcgen05.mma kind::tf32, operands split hi + lo for
                              FP32-level products), 0 = on the CUDA cores          */
  int patch_fixed;         /* decoupled FP64 patches (patch_form != 0, blocks of at
                              most 63 DoFs: the 2D levels): 1 = every stored
                              inverse row kept as 57-bit fixed point with its own
                              power of two, applied by exact integer dot products
                              (32×32→64-bit multiply-adds) against the patch's
                              sources scaled to 58-bit integers, rounded once to
                              FP64; 0 = FP64 entries and FP64 FMAs.  Levels that do
                              not qualify keep FP64 entries                        */
  int op_fixed;            /* 2D levels, s ≤ 3: 1 = the stage operator J x (and
                              the residual F − J x) from 57-bit fixed-point copies
                              of its rows (one power of two per row) and the
                              iterate as 58-bit integers with one power of two per
                              velocity / pressure group, the stage mixing dt·A
                              applied exactly to the iterate (rounded once to 58
                              bits), every product sum exact and rounded once to
                              FP64, at most three sums added in FP64 per output;
                              0 = FP64 FMAs.  The transposed operator and the
                              Newton blocks of Navier–Stokes stay FP64            */
} irkmg_options;

typedef struct {
  int iters;               /* FGMRES iterations taken                               */
  int status;              /* IRKMG_* of the solve                                  */
  double r0, rfinal;       /* ||F - J k0||, final true residual norm                */
  double t_setup, t_solve; /* seconds (host clock around synchronised work)         */
  int64_t bad_index;       /* patch id (or coarse row) for IRKMG_ESINGULAR, else -1 */
} irkmg_stats;

typedef struct {
  int64_t nv, ne, nc;      /* vertices, edges, cells of the level                   */
  int64_t np2, nf;         /* P2 nodes, free P2 nodes                               */
  int64_t m, N;            /* per-stage length 2 nf + nv, full length s·m           */
  int64_t npatch, ncolours;/* Vanka patches (one per vertex), colours               */
  int64_t max_patch_dofs;  /* largest patch size s·(2·nodes + 1)                    */
  int64_t factor_bytes;    /* bytes of stored patch blocks (inverses + index list)  */
  int64_t apply_kernel;    /* Vanka apply kernel in use: 1 TMA-staged, 2 warp-per-patch,
                              3 CTA-per-patch mat-vec (patches above 160 DoFs, whose
                              inverses come from a blocked LU; 3D); decoupled form
                              (patch_form != 0): 4 warp-per-patch, 5 TMA-staged,
                              6 CTA-per-patch (blocks above 160 DoFs, factored by
                              the blocked LU; 3D), 7 warp-specialised TMA
                              pipeline; patch_fixed: 8 warp-per-patch, 9 TMA-
                              staged exact fixed-point mat-vecs, 10 warp-per-
                              patch with X and Y rows paired (complex layout)     */
  double apply_ms[2];      /* autotuner: one sweep with the fastest staged (or, for
                              decoupled levels, CTA-per-patch) candidate / the
                              fastest warp-per-patch candidate (0 if untimed)      */
  int64_t dim;             /* 2 or 3                                                */
  int64_t single_launch;   /* 1: the level relaxes by one launch over all patches
                              plus a deterministic per-DoF sum (decoupled form);
                              0: one launch per colour                             */
  double cheb[2];          /* Chebyshev interval used on the level                  */
  int64_t apply_shape;     /* launch shape of the apply kernel: 0..1 for kernel 5
                              (staged, three- or two-stage ring); 0..3 for kernel 8
                              (columns per load batch × resident CTAs per SM:
                              8×3, 4×4, 6×3, 8×4), 4..6 for kernel 9 (stages ×
                              CTAs per SM: 4×1, 3×1, 2×2), 7..8 for kernel 10
                              (columns per load batch 8, 2; 4 CTAs per SM; the
                              transposed apply of such a level runs kernel 8
                              with shape 3); 0 otherwise                           */
} irkmg_level_info;

/* ---- set-up -------------------------------------------------------------- */

/* Defaults described above.  Never fails. */
void irkmg_default_options(irkmg_options *opt);

/* Radau IIA(s) tableau into host arrays A[s*s], b[s], c[s] (Section 5: the
 * standard RadauIIA family).  s in 1..3 from closed forms.  EINVAL otherwise. */
int irkmg_radau_iia(int s, double *A, double *b, double *c);

/* Gauss(s) (order 2s, A-stable) and LobattoIIIC(s) (order 2s - 2, L-stable)
 * tableaux, s = 2, 3, from closed forms; the paper runs both families beside
 * RadauIIA (Section 5, Tables 1 and 2).  Same output layout as above. */
int irkmg_gauss(int s, double *A, double *b, double *c);
int irkmg_lobatto_iiic(int s, double *A, double *b, double *c);

/* The real block diagonalisation A = T D T⁻¹ (s ≤ 3, row-major s×s outputs)
 * behind the decoupled patch solves (patch_form != 0): D holds the real
 * eigenvalues of A as 1×1 blocks and each complex pair α ± iβ (β > 0) as the
 * 2×2 block [[α, β], [−β, α]], real blocks first; T holds unit eigenvectors
 * for real eigenvalues and, for a pair, Re v and Im v of a unit eigenvector v
 * whose phase makes them orthogonal.  It rests on the Kronecker form
 * of the stage system (Section 3).  IRKMG_ENOTIMPL when two eigenvalues
 * coincide.  Host only; no device work. */
int irkmg_kron_split(int s, const double *A, double *T, double *Tinv, double *D);

/* Eigenvalues wr + i·wi of the n×n upper Hessenberg H (row-major, n <= 512):
 * the Ritz values of an Arnoldi process (shifted QR in complex arithmetic).
 * Host only. */
int irkmg_hessenberg_eigvals(int n, const double *H, double *wr, double *wi);

/* Section 5.1's estimate of the largest eigenvalue of the Vanka-preconditioned
 * operator D⁻¹J of a level (D⁻¹ = Σ_v R_vᵀ A_v⁻¹ R_v): nsteps (2 .. restart)
 * Arnoldi steps from d_x0 (device, N of the level) or, if NULL, from
 * x_i = sin(i + 1); *lambda = the largest real part of the Ritz values, which
 * ritz_re / ritz_im (host, nsteps each, may be NULL) receive. */
int irkmg_estimate_lambda(irkmg_ctx *ctx, int level, int nsteps, const double *d_x0,
                          double *ritz_re, double *ritz_im, double *lambda);

/* Build the hierarchy, assemble every level, build patch maps and colourings,
 * factor (invert) every patch and the bordered coarsest system.  Host inputs
 * are copied.  On failure *out is NULL.  The host part of the assembly runs on
 * the hardware-concurrency threads (environment variable IRKMG_HOST_THREADS,
 * 1..64, overrides); every entry is summed in one fixed order, so nothing
 * depends on the thread count. */
int irkmg_setup(const irkmg_mesh *mesh, const irkmg_tableau *tab, double dt, double nu,
                const irkmg_options *opt, irkmg_ctx **out);

/* Re-assemble and re-factor for a new dt and nu (same mesh, tableau, wind). */
int irkmg_update(irkmg_ctx *ctx, double dt, double nu);

/* Replace the Oseen wind (host array, finest-level P2 nodes, np2·2 doubles,
 * x and y per node; NULL returns to Stokes) and re-assemble and re-factor every
 * level, as irkmg_update does; coarse levels take the wind at their own P2
 * nodes (which are finest-level nodes).  This is the frozen-wind update of a
 * Picard linearisation of Navier–Stokes (Section 3.2). */
int irkmg_set_wind(irkmg_ctx *ctx, const double *wind);

/* Sizes of level l (0 = coarsest, nlevels-1 = finest). */
int irkmg_level_info_get(const irkmg_ctx *ctx, int level, irkmg_level_info *info);
/* Pin the launch shape (see irkmg_level_info.apply_shape) and, on decoupled
 * levels, the relaxation mode (single_launch 1: one launch over all patches and
 * the per-DoF sum; 0: one launch per colour) of level >= 1, overriding the
 * set-up autotuner.  IRKMG_EINVAL for a shape the level's kernel does not have
 * (or whose shared memory does not fit) and for single_launch = 1 on a level
 * with dense patches. */
int irkmg_level_set_apply(irkmg_ctx *ctx, int level, int shape, int single_launch);

/* Replace the bound on the polls of one device-side wait (irkmg_options.
 * timeout_spins; 0 = 2^26, and each wait also gives up after 2 s) for the
 * calls that follow.  A wait that expires records IRKMG_ETIMEOUT, its CTA
 * waits (with its own bound) for the copies it still has in flight and
 * leaves; FGMRES returns IRKMG_ETIMEOUT after the Arnoldi step that saw it and
 * the context stays usable.  Failure detection of the staged kernels
 * (Section 4.2's patch solves streamed by bulk copies); IRKMG_EINVAL if
 * timeout_spins < 0. */
int irkmg_set_timeout(irkmg_ctx *ctx, int64_t timeout_spins);

/* Host copies of set-up data of level l, for inspection and tests.
 * irkmg_p2_coords: np2·2 doubles.  irkmg_free_nodes: nf int64 P2-node ids.
 * irkmg_patch_map: ptr[npatch+1] and nodes[ptr[npatch]] (free-node ids,
 * ascending per patch: the velocity nodes of the closure of the star of each
 * vertex, Section 4.2).  irkmg_colouring: colour per vertex (greedy distance-2
 * colouring in vertex-id order).  Pass NULL to query sizes through
 * irkmg_level_info_get first. */
int irkmg_p2_coords(const irkmg_ctx *ctx, int level, double *xy);
int irkmg_free_nodes(const irkmg_ctx *ctx, int level, int64_t *ids);
int irkmg_patch_map(const irkmg_ctx *ctx, int level, int64_t *ptr, int32_t *nodes);
int irkmg_colouring(const irkmg_ctx *ctx, int level, int32_t *colour);

/* ---- operators on level l (device vectors of length N_l) ---------------- */

/* y = J x (transpose = 0) or y = Jᵀ x (transpose = 1), Section 3.1. */
int irkmg_apply(irkmg_ctx *ctx, int level, const double *d_x, double *d_y, int transpose);

/* c = sum_v R_vᵀ (R_v J R_vᵀ)^{-1} R_v r  (one additive Vanka correction,
 * Section 4.2), with the stored patch inverses; transpose = 1 uses Jᵀ. */
int irkmg_vanka_correction(irkmg_ctx *ctx, int level, const double *d_r, double *d_c,
                           int transpose);

/* nsteps relaxation steps on J x = F from the x given (in/out), with the
 * smoother of the options (Sections 4.2, 5.1). */
int irkmg_smooth(irkmg_ctx *ctx, int level, const double *d_F, double *d_x, int nsteps,
                 int transpose);

/* The same relaxation as irkmg_smooth, with no device allocation anywhere on
 * its path.  The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc when they relax a vector — for example code whose
 * device memory is entirely reserved by another framework's caching
 * allocator, or a time loop that must not pay the device-wide synchronisation
 * an allocation can imply.  Its two work vectors (residual and Chebyshev
 * direction) live in one file-scope static device array of
 * 2 × 524,288 doubles (8 MB, held by every GPU that loads the library until
 * the process exits), so the level must have N <= 524,288 (e.g. 128×128 with
 * s = 3); larger levels are rejected with IRKMG_EINVAL and no work is done.
 * Each call made outside stream capture looks up the array's device address
 * with the calling device current (so a device context that was torn down and
 * re-created is followed); a call made during capture reuses the address the
 * last uncaptured call on that device found, so make the first call on a
 * device before any stream capture (otherwise IRKMG_EINVAL).  Every call shares the array: calls that overlap on the GPU (other
 * streams, other contexts, other threads) race and must be serialised by the
 * caller.  The array keeps the last call's contents; every value a call reads
 * from it is written (or cleared) first by that same call. */
int irkmg_smooth_noalloc(irkmg_ctx *ctx, int level, const double *d_F, double *d_x, int nsteps,
                         int transpose);

/* Transfers between level l (fine) and l-1: d_coarse = (I_s ⊗ P)ᵀ d_fine, and
 * d_fine = (I_s ⊗ P) d_coarse (overwrites), Section 4.1. */
int irkmg_restrict(irkmg_ctx *ctx, int level, const double *d_fine, double *d_coarse);
int irkmg_prolong(irkmg_ctx *ctx, int level, const double *d_coarse, double *d_fine);

/* Coarsest-level direct solve of the bordered system [[J, N], [Nᵀ, 0]] (N:
 * one constant-pressure column per stage); the result has zero pressure sum
 * in every stage. */
int irkmg_coarse_solve(irkmg_ctx *ctx, const double *d_r, double *d_x, int transpose);

/* ---- the solver ---------------------------------------------------------- */

/* One V(nu_pre, nu_post) cycle on the finest level with zero initial guess. */
int irkmg_vcycle(irkmg_ctx *ctx, const double *d_r, double *d_z, int transpose);

/* FGMRES(restart) right-preconditioned by the V-cycle: J k = F on the finest
 * level.  d_k holds the initial guess on entry and the solution on return.
 * Each preconditioned vector has its per-stage pressure mean removed.
 * stats may be NULL.  Returns ENOCONV (with the best iterate) at maxit. */
int irkmg_solve(irkmg_ctx *ctx, const double *d_F, double *d_k, irkmg_stats *stats);

/* The same for the transposed stage operator: Jᵀ lam = G (discrete adjoint;
 * transposed Vanka patches, A -> Aᵀ). */
int irkmg_adjoint_solve(irkmg_ctx *ctx, const double *d_G, double *d_lam, irkmg_stats *stats);

/* ---- time stepping (Section 3.1) ----------------------------------------- */

/* F_i = [ M f_i - K u^n - B p^n ; -Bᵀ u^n ] on the finest level.
 * d_un: 2·nf (u_x then u_y on free nodes), d_pn: nv, d_f: s·2·np2 (stage,
 * component, every P2 node: the interpolant of the forcing at t + c_i dt). */
int irkmg_stage_rhs(irkmg_ctx *ctx, const double *d_un, const double *d_pn, const double *d_f,
                    double *d_F);

/* u^{n+1} = u^n + dt sum_j b_j k_j^u and likewise p (in place). */
int irkmg_advance(irkmg_ctx *ctx, const double *d_k, double *d_un, double *d_pn);

/* The stage right-hand side with u^n given at every P2 node (2·np2: u_x then
 * u_y), so that boundary values of u^n enter (a moving lid, Section 3.1 with
 * inhomogeneous Dirichlet data carried by u^n):
 * F_i = [ M f_i - K u^n - B p^n ; -Bᵀ u^n ] with K (including any Oseen
 * convection) and Bᵀ over every velocity column.  The stages themselves stay
 * homogeneous on the boundary (the boundary data is steady). */
int irkmg_stage_rhs_full(irkmg_ctx *ctx, const double *d_un_all, const double *d_pn,
                         const double *d_f, double *d_F);

/* ---- batched solves of independent stage systems --------------------------
 * A batch groups contexts of any sizes, tableaux, dt, nu and winds.  Creating
 * it gives every context its own non-blocking stream (restored by
 * irkmg_batch_destroy; contexts stay owned by the caller and must outlive the
 * batch).  irkmg_batch_solve runs FGMRES on all systems in lock step: each
 * Arnoldi step of every unconverged system is issued on its stream, then all
 * are synchronised once and the small Hessenberg updates run on the host.
 *
 * When every system is 2D with the same stage count, Chebyshev smoothing of
 * 1..8 steps and fixed-point decoupled patches on its finest level
 * (patch_form != 0, patch_fixed = 1), and there are at most 128 systems, the
 * finest-level relaxation of all unconverged systems runs as ONE persistent
 * cooperative launch per smoothing stage (operator rows, patch solves and
 * per-DoF sums of every system, separated by bounded grid-wide barriers that
 * report IRKMG_ETIMEOUT through the solve, with the bound of the first
 * system's timeout_spins); the coarse corrections run on the systems' own
 * streams.  The batch then relaxes those finest levels by one launch over all
 * patches plus the per-DoF sum, also in irkmg_solve on those contexts until
 * irkmg_batch_destroy restores their mode.  Otherwise each system's V-cycle
 * is one CUDA graph on its stream, captured on first use.  Either way the
 * results equal those of irkmg_solve on each system (bit for bit in the same
 * relaxation mode).  d_F[i], d_k[i] live on the device of system i's context;
 * stats (may be NULL) has nsys entries. */
typedef struct irkmg_batch irkmg_batch;
int irkmg_batch_create(int nsys, irkmg_ctx *const *ctxs, irkmg_batch **out);
int irkmg_batch_solve(irkmg_batch *batch, const double *const *d_F, double *const *d_k,
                      irkmg_stats *stats);
/* 1 if the batch relaxes its finest levels in one persistent launch, else 0. */
int irkmg_batch_persistent(const irkmg_batch *batch);
/* Switch a qualifying batch between the persistent launch (on = 1, the
 * default) and one V-cycle graph per system (on = 0); the finest levels stay
 * in the one-launch relaxation mode either way, so the results do not change.
 * IRKMG_ENOTIMPL for on = 1 on a batch that does not qualify. */
int irkmg_batch_set_persistent(irkmg_batch *batch, int on);
void irkmg_batch_destroy(irkmg_batch *batch);

/* ---- Navier–Stokes: Newton on the stage equations (Section 3.2) ---------
 * With U_t = u^n + dt Σ_j a_tj k_j and P_t = p^n + dt Σ_j a_tj k_j^p the stage
 * residual is F_t = [ M k_t + N(U_t) + K U_t + B P_t − M f_t ; Bᵀ U_t ], N(U) =
 * C(U) U the discrete <u·∇u, v>.  Its Jacobian has the velocity blocks
 * δ_tu M + dt a_tu (K + C(U_t) + R(U_t)), R(w)_dc = ∫ φ_a φ_b ∂w_d/∂x_c, which
 * depend on the row stage and couple the components: dense patches only
 * (patch_form 0), 2D, no frozen wind. */
typedef struct {
  int newton_iters;        /* Newton steps taken                                    */
  int linear_iters;        /* FGMRES iterations over all Newton steps               */
  int status;
  double f0, ffinal;       /* ||F(k0)||, ||F(k)|| at the end                         */
  double t_solve;          /* seconds                                               */
} irkmg_ns_stats;

/* Set the Newton blocks for the stage velocities U (host, s x 2 x np2: stage,
 * component, finest P2 node, Dirichlet values included) on every level
 * (injected to coarse levels), refactor the patches and the coarsest solve. */
int irkmg_ns_set_state(irkmg_ctx *ctx, const double *U);
/* F(k) on the finest level for the state last set (that of k): u^n at every
 * P2 node (2·np2), p^n, f (s·2·np2 nodal forcing), k and F (N each). */
int irkmg_ns_residual(irkmg_ctx *ctx, const double *d_un_all, const double *d_pn,
                      const double *d_f, const double *d_k, double *d_F);
/* Inexact Newton from the guess in d_k (e.g. the previous step's stages,
 * Section 3.2) until ||F|| <= atol or maxit steps: each step sets the state,
 * forms F and solves J δ = −F by the preconditioned FGMRES to the relative
 * tolerance of Eisenstat and Walker's choice 2 (γ = 0.9, α = 2, safeguard,
 * η ≤ 0.9, η_0 = 0.5).  IRKMG_ENOCONV if maxit is reached. */
int irkmg_ns_newton(irkmg_ctx *ctx, const double *d_un_all, const double *d_pn,
                    const double *d_f, double *d_k, double atol, int maxit,
                    irkmg_ns_stats *stats);

/* ---- forcing control and the discrete adjoint (differentiation of the
 * Section 3.1 time stepping; the paper does not differentiate) ------------- */

/* Velocity load of a per-cell constant forcing th: g = C th with
 * C[a, c] = ∫_c φ_a on the finest level.  d_theta: 2·nc (x block, then y
 * block, cell ids of the finest mesh); d_g: 2·nf (u_x block, then u_y). */
int irkmg_forcing_load(irkmg_ctx *ctx, const double *d_theta, double *d_g);

/* One implicit RK time step on the finest level (Section 3.1):
 * F = irkmg_stage_rhs(u^n, p^n, f) plus d_g in every stage (d_g may be NULL),
 * J k = F by FGMRES from a zero guess (stages written to d_k, length N), then
 * u^n, p^n advanced in place to u^{n+1}, p^{n+1}.  Status as irkmg_solve. */
int irkmg_step(irkmg_ctx *ctx, double *d_un, double *d_pn, const double *d_f, const double *d_g,
               double *d_k, irkmg_stats *stats);

/* Reverse of irkmg_step for the adjoint state (ub, pb) = dObj/d(u^{n+1}, p^{n+1})
 * (in) -> dObj/d(u^n, p^n) (out, in place), given that step's stages d_k and
 * start state d_un:  kb_j = dt b_j [ub; pb],  Jᵀ lam = kb (FGMRES with the
 * transposed V-cycle),  ub -= sum_i (Kᵀ lam_i,u + B lam_i,p),
 * pb -= sum_i Bᵀ lam_i,u.  It also accumulates the forcing gradient
 * d_theta_bar += Cᵀ sum_i lam_i,u (2·nc, may be NULL) and, through K = nu·K1
 * in both J and F, *d_nu += -(1/nu) sum_i lam_i,u · K (u^n + dt sum_j a_ij k_j,u)
 * (host double, may be NULL). */
int irkmg_adjoint_step(irkmg_ctx *ctx, double *d_ubar, double *d_pbar, const double *d_k,
                       const double *d_un, double *d_theta_bar, double *d_nu, irkmg_stats *stats);

/* Tracking objective on the finest level: *value = 1/2 eᵀ M2 e with
 * e = u - u_target (free velocity DoFs, M2 = diag(M, M)); d_grad = M2 e
 * (2·nf, may be NULL).  *value is a host double. */
int irkmg_tracking(irkmg_ctx *ctx, const double *d_u, const double *d_utarget, double *d_grad,
                   double *value);

/* ---- tracing ---------------------------------------------------------------- */

/* Kernel accounting since the last irkmg_trace_enable.  `launches` counts every
 * kernel the library issued (with tracing on or off).  With tracing on, each
 * finest-level Vanka colour launch, each finest-level stage-operator launch,
 * each finest-level transfer and each Gram–Schmidt step of FGMRES is bracketed
 * by CUDA events on the context stream; *_ms is their summed device time and *_bytes their
 * algorithmic bytes: per Vanka sweep, sum over patches of n_p^2·w + 4·n_p plus
 * 24·N for reading r and updating the target (split over the colour launches
 * in proportion to their inverse bytes); per operator application,
 * nnz(vel)·20 + (nnz(B) + nnz(Bᵀ))·20 + 24·N bytes. */
typedef struct {
  int64_t launches;
  int64_t vanka_launches;
  double vanka_ms, vanka_bytes;
  int64_t op_launches;
  double op_ms, op_bytes;
  double vanka_flops;      /* 2·n_p^2 per patch applied in the timed Vanka launches
                              (decoupled form: 2·(nt·n² + (ns + nt)·s·n), see
                              patch_form)                                           */
  double op_flops;         /* 2·(4s·nnz(vel) + 2s·(nnz(B) + nnz(Bᵀ)) + 2s²·n_f + s²·n_v)
                              per timed operator launch                              */
  int64_t reduce_launches; /* timed per-DoF sums of the one-launch relaxation      */
  double reduce_ms, reduce_bytes;
  int64_t xfer_launches;   /* timed finest-level transfers (Section 4.1): restriction
                              to the next level (8·(N_f + N_c) bytes: the fine vector
                              read, the coarse one written) and prolongation added
                              into the fine vector (8·(N_c + 2 N_f) bytes); the
                              interpolation weights are closed-form per refinement
                              pattern and not counted                              */
  double xfer_ms, xfer_bytes;
  int64_t arnoldi_steps;   /* timed classical Gram–Schmidt steps (twice) of FGMRES
                              (Section 4) after the j-th preconditioned product:
                              per pass the j + 1 basis vectors and w are read by
                              the dot products and again by the update, which
                              also writes w, then ||w||²:
                              8N·(2(j + 2) + 2(j + 3) + 1) bytes                    */
  double arnoldi_ms, arnoldi_bytes;
  int64_t factor_launches;  /* timed finest-level patch factorisations (set-up work of
                               Section 4.2, redone by irkmg_update): every patch
                               block inverted explicitly, 2 m³ flops for an m × m
                               block (LU 2/3 m³ plus the inverse from it 4/3 m³)    */
  double factor_ms, factor_flops;
} irkmg_trace;

/* Reset the counters; on = 1 also starts event timing.  Never fails on a valid ctx. */
int irkmg_trace_enable(irkmg_ctx *ctx, int on);
/* Synchronise the context stream and return the totals (resets the event pool). */
int irkmg_trace_read(irkmg_ctx *ctx, irkmg_trace *out);

/* ---- teardown, diagnostics ------------------------------------------------ */
void irkmg_destroy(irkmg_ctx *ctx);
const char *irkmg_strerror(int status);
const char *irkmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IRKMG_H */

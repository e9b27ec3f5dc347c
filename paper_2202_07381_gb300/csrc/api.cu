// irkmg C ABI: set-up of the hierarchy, the V-cycle, the smoothers and FGMRES.
//
// Section 4: FGMRES right-preconditioned by a monolithic V-cycle whose
// relaxation is the IRK-extended additive Vanka step (Section 4.2), damped or
// Chebyshev-accelerated (Section 5.1), with I_s ⊗ P transfers, restriction Pᵀ
// and a direct coarsest solve (Section 4.1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "irkmg_internal.h"

using namespace irkmg;

struct irkmg_ctx : public Ctx {};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(IRKMG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

template <typename T>
int dalloc(Ctx& C, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(IRKMG_ENOMEM, "cudaMalloc of " + std::to_string(sizeof(T) * count) +
                                  " bytes failed: " + cudaGetErrorString(e));
  }
  C.allocs.push_back((void*)*p);
  C.dev_bytes += (int64_t)(sizeof(T) * count);
  return IRKMG_OK;
}

template <typename T>
int upload(Ctx& C, T** p, const std::vector<T>& h) {
  int rc = dalloc(C, p, h.size());
  if (rc) return rc;
  if (!h.empty()) CK(cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return IRKMG_OK;
}

int upload_csr(Ctx& C, DevCSR& d, const HostCSR& h, int nvals) {
  d.nrows = (int32_t)h.nrows;
  d.nnz = h.nnz();
  int rc;
  if ((rc = upload(C, &d.ptr, h.ptr))) return rc;
  if ((rc = upload(C, &d.col, h.col))) return rc;
  for (int k = 0; k < nvals; ++k)
    if ((rc = upload(C, &d.v[k], h.v[k]))) return rc;
  return IRKMG_OK;
}

// SELL-32 copy of a host CSR (see DevSELL).
struct HostSELL {
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> v[3];
};

// skip_pad: padded entries get column −1 (the transfers stop there) instead
// of the row's last column with a zero value.
HostSELL to_sell(const HostCSR& A, int nvals, bool skip_pad = false) {
  HostSELL S;
  const int64_t n = A.nrows, ns = (n + 31) / 32;
  S.ptr.assign(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) {
    int32_t w = 0;
    for (int64_t r = sl * 32; r < std::min(n, sl * 32 + 32); ++r)
      w = std::max(w, A.ptr[r + 1] - A.ptr[r]);
    S.ptr[sl + 1] = S.ptr[sl] + 32 * (int64_t)w;
  }
  S.col.assign(S.ptr[ns], 0);
  for (int k = 0; k < nvals; ++k) S.v[k].assign(S.ptr[ns], 0.0);
  for (int64_t r = 0; r < n; ++r) {
    const int64_t base = S.ptr[r / 32] + r % 32;
    const int64_t w = (S.ptr[r / 32 + 1] - S.ptr[r / 32]) / 32;
    const int32_t len = A.ptr[r + 1] - A.ptr[r];
    const int32_t pad = len > 0 ? A.col[A.ptr[r + 1] - 1] : 0;
    for (int64_t k = 0; k < w; ++k) {
      const int64_t dst = base + 32 * k;
      if (k < len) {
        S.col[dst] = A.col[A.ptr[r] + k];
        for (int q = 0; q < nvals; ++q) S.v[q][dst] = A.v[q][A.ptr[r] + k];
      } else {
        S.col[dst] = skip_pad ? -1 : pad;
      }
    }
  }
  return S;
}

int upload_sell(Ctx& C, DevSELL& d, const HostCSR& h, int nvals, bool skip_pad = false) {
  HostSELL S = to_sell(h, nvals, skip_pad);
  d.nrows = (int32_t)h.nrows;
  d.stored = (int64_t)S.col.size();
  int rc;
  if ((rc = upload(C, &d.ptr, S.ptr))) return rc;
  if ((rc = upload(C, &d.col, S.col))) return rc;
  for (int k = 0; k < nvals; ++k)
    if ((rc = upload(C, &d.v[k], S.v[k]))) return rc;
  return IRKMG_OK;
}

int refresh_sell_values(Ctx& C, DevSELL& d, const HostCSR& h, int nvals) {
  (void)C;
  HostSELL S = to_sell(h, nvals);
  for (int k = 0; k < nvals; ++k)
    CK(cudaMemcpy(d.v[k], S.v[k].data(), sizeof(double) * S.v[k].size(), cudaMemcpyHostToDevice));
  return IRKMG_OK;
}

int refresh_csr_values(Ctx& C, DevCSR& d, const HostCSR& h, int nvals) {
  (void)C;
  for (int k = 0; k < nvals; ++k)
    CK(cudaMemcpy(d.v[k], h.v[k].data(), sizeof(double) * h.v[k].size(), cudaMemcpyHostToDevice));
  return IRKMG_OK;
}

int check_err(Ctx& C, const char* what, irkmg_stats* st = nullptr) {
  int h[2] = {0, 0};
  CK(cudaMemcpy(h, C.d_err, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[0] != 0) {
    CK(cudaMemset(C.d_err, 0, sizeof(int) * 2));
    if (st) st->bad_index = h[1];
    return fail(h[0], std::string(what) + ": singular pivot at index " + std::to_string(h[1]));
  }
  return IRKMG_OK;
}

// --- tracing -----------------------------------------------------------------
// Returns the start/stop event pair to record around one traced launch.
int trace_pair(Ctx& C, int cls, double bytes, cudaEvent_t* a, cudaEvent_t* b,
               double flops = 0.0) {
  if (C.ev_used + 2 > C.ev.size()) {
    for (int k = 0; k < 256; ++k) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      C.ev.push_back(e);
    }
  }
  *a = C.ev[C.ev_used];
  *b = C.ev[C.ev_used + 1];
  C.ev_used += 2;
  C.ev_class.push_back(cls);
  C.ev_bytes.push_back(bytes);
  C.ev_flops.push_back(flops);
  return IRKMG_OK;
}

// Stage operator (r = F - J x, or y = J x when F is null), counted and traced.
int op(Ctx& C, Level& L, const double* F, const double* x, double* r, int tr) {
  if (tr && C.ns && C.ns_active)
    return fail(IRKMG_ENOTIMPL, "transposed Navier-Stokes Newton operator");
  const bool timed = C.trace_on && &L == &C.L.back();
  cudaEvent_t a = nullptr, b = nullptr;
  if (timed) {
    int rc = trace_pair(C, 1, L.op_bytes - (F ? 0.0 : 8.0 * L.N), &a, &b, L.op_flops);
    if (rc) return rc;
    CK(cudaEventRecord(a, C.stream));
  }
  CK(launch_residual(C, L, F, x, r, tr));
  C.launches++;
  if (timed) CK(cudaEventRecord(b, C.stream));
  return IRKMG_OK;
}

void level_trace_bytes(Ctx& C, Level& L) {
  const double w = C.opt.patch_precision == 64 ? 8.0 : 4.0;
  L.colour_bytes.assign(L.ncolours, 0.0);
  L.colour_flops.assign(L.ncolours, 0.0);
  double total = 0.0;
  std::vector<double> inv(L.ncolours, 0.0);
  const double s = (double)C.s;
  for (int64_t v = 0; v < L.nv; ++v) {
    const double n = (double)(L.dim * (L.h_patch_ptr[v + 1] - L.h_patch_ptr[v]) + 1);
    double fb, fl;
    if (L.kron) {
      // nm stored n x n matrices, n indices; nt mat-vecs plus the source and
      // output transforms (ns·s and s·nt multiply-adds per spatial DoF)
      const KronPlan& K = C.kplan;
      fb = K.nm * n * n * w + 4.0 * n;
      fl = 2.0 * (K.nt * n * n + (double)K.ns * s * n + s * K.nt * n);
    } else {
      const double np = s * n;
      fb = np * np * w + 4.0 * np;
      fl = 2.0 * np * np;
    }
    inv[L.h_colour[v]] += fb;
    L.colour_flops[L.h_colour[v]] += fl;
    total += fb;
  }
  double invsum = 0.0;
  for (double x : inv) invsum += x;
  const double sweep = total + 24.0 * (double)L.N;
  for (int c = 0; c < L.ncolours; ++c) L.colour_bytes[c] = sweep * inv[c] / invsum;
}

// --- patches: maps, colouring, ordering, inverses (Section 4.2) -----------
int build_patches(Ctx& C, Level& L) {
  const int maxnodes = 96;
  int rc;
  if ((rc = upload(C, &L.d_cells, L.mesh.cells))) return rc;
  if ((rc = upload(C, &L.d_cell_edges, L.mesh.cell_edges))) return rc;
  if ((rc = upload(C, &L.d_vc_ptr, L.mesh.vc_ptr))) return rc;
  if ((rc = upload(C, &L.d_vc_idx, L.mesh.vc_idx))) return rc;
  if ((rc = upload(C, &L.d_vv_ptr, L.mesh.vv_ptr))) return rc;
  if ((rc = upload(C, &L.d_vv_idx, L.mesh.vv_idx))) return rc;
  if ((rc = upload(C, &L.d_p2_to_free, L.mesh.p2_to_free))) return rc;
  int32_t *d_tmp = nullptr, *d_cnt = nullptr;
  CK(cudaMalloc(&d_tmp, sizeof(int32_t) * L.nv * maxnodes));
  CK(cudaMalloc(&d_cnt, sizeof(int32_t) * (L.nv + 1)));
  if ((rc = dalloc(C, &L.d_patch_ptr, L.nv + 1))) return rc;
  CK(launch_patch_maps(L, C.stream, maxnodes, d_tmp, d_cnt));
  std::vector<int32_t> cnt(L.nv);
  CK(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * L.nv, cudaMemcpyDeviceToHost, C.stream));
  CK(cudaStreamSynchronize(C.stream));
  for (int64_t v = 0; v < L.nv; ++v)
    if (cnt[v] < 0) {
      cudaFree(d_tmp);
      cudaFree(d_cnt);
      return fail(IRKMG_EINVAL, "vertex star too large for the patch builder");
    }
  CK(launch_scan(d_cnt, L.d_patch_ptr, L.nv, C.stream));
  L.h_patch_ptr.resize(L.nv + 1);
  CK(cudaMemcpyAsync(L.h_patch_ptr.data(), L.d_patch_ptr, sizeof(int32_t) * (L.nv + 1),
                     cudaMemcpyDeviceToHost, C.stream));
  CK(cudaStreamSynchronize(C.stream));
  if ((rc = dalloc(C, &L.d_patch_nodes, L.h_patch_ptr[L.nv]))) return rc;
  CK(launch_compact_patches(L, C.stream, maxnodes, d_tmp, d_cnt));
  L.h_patch_nodes.resize(L.h_patch_ptr[L.nv]);
  CK(cudaMemcpyAsync(L.h_patch_nodes.data(), L.d_patch_nodes,
                     sizeof(int32_t) * L.h_patch_nodes.size(), cudaMemcpyDeviceToHost, C.stream));
  // colouring: Jones–Plassmann rounds until every vertex is coloured
  if ((rc = dalloc(C, &L.d_colour, L.nv))) return rc;
  CK(cudaMemsetAsync(L.d_colour, 0xff, sizeof(int32_t) * L.nv, C.stream));
  int* d_flags = d_cnt;  // reuse: [0] remaining, [1] overflow
  int h_flags[2] = {1, 0};
  int64_t rounds = 0;
  while (h_flags[0] > 0) {
    CK(cudaMemsetAsync(d_flags, 0, sizeof(int) * 2, C.stream));
    for (int k = 0; k < 8; ++k) {
      if (k == 7) CK(cudaMemsetAsync(d_flags, 0, sizeof(int), C.stream));
      CK(launch_colour_round(L, C.stream, d_flags, d_flags + 1));
    }
    CK(cudaMemcpyAsync(h_flags, d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, C.stream));
    CK(cudaStreamSynchronize(C.stream));
    rounds += 8;
    if (h_flags[1]) return fail(IRKMG_EINVAL, "colouring needs more than 256 colours");
    if (rounds > 8 * (L.nv + 8)) return fail(IRKMG_ETIMEOUT, "colouring did not finish");
  }
  cudaFree(d_tmp);
  cudaFree(d_cnt);
  L.h_colour.resize(L.nv);
  CK(cudaMemcpy(L.h_colour.data(), L.d_colour, sizeof(int32_t) * L.nv, cudaMemcpyDeviceToHost));
  // order patches by (colour, vertex id); factor offsets in that order
  L.ncolours = 0;
  for (int32_t c : L.h_colour) L.ncolours = std::max(L.ncolours, c + 1);
  std::vector<int64_t> start(L.ncolours + 1, 0);
  for (int32_t c : L.h_colour) start[c + 1]++;
  for (int c = 0; c < L.ncolours; ++c) start[c + 1] += start[c];
  std::vector<int32_t> order(L.nv);
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t v = 0; v < L.nv; ++v) order[fill[L.h_colour[v]]++] = (int32_t)v;
  }
  L.colour_start = start;
  // Each ordered patch owns one 16-byte-aligned block: its n_p x n_p inverse
  // (column-major, padded to 16 bytes) followed by its n_p global DoF indices
  // (int32, padded to 16 bytes), so one bulk copy brings both.
  // Large patches (3D) keep LU factors and pivots instead of an inverse.
  std::vector<int64_t> off(L.nv + 1, 0);
  std::vector<int32_t> npv(L.nv);
  L.max_np = 0;
  const int64_t w = C.opt.patch_precision == 64 ? 8 : 4;
  for (int64_t i = 0; i < L.nv; ++i) {
    const int32_t v = order[i];
    const int64_t np = (int64_t)C.s * (L.dim * (L.h_patch_ptr[v + 1] - L.h_patch_ptr[v]) + 1);
    L.max_np = std::max<int>(L.max_np, (int)np);
    npv[i] = (int32_t)np;
  }
  L.big = L.max_np > kMaxSmallNp;
  // Decoupled patch factors: inverted in shared memory where the largest
  // block (2n for a complex pair) fits, else by the blocked LU up to
  // kMaxBigNp; the dense form otherwise.
  L.kron = false;
  L.kron_big = false;
  if (C.kron) {
    int q = 1;
    for (int b = 0; b < C.kplan.nblk; ++b) q = std::max(q, C.kplan.blk_size[b]);
    const int nmax = L.max_np / C.s;
    const bool small = q * nmax <= kMaxSmallNp && C.kplan.nt * nmax <= 32 * kron_max_slots();
    const bool big = !small && q * nmax <= kMaxBigNp && nmax <= kron_big_max_n();
    if (small || big) {
      L.kron = true;
      L.kron_big = big;
      L.big = big;
      L.kron_nmax = nmax;
      for (int64_t i = 0; i < L.nv; ++i) npv[i] /= C.s;
    }
  }
  if (!L.kron && L.max_np > kMaxBigNp)
    return fail(IRKMG_ENOTIMPL, "patches above " + std::to_string(kMaxBigNp) + " DoFs");
  // explicit inverses of every patch block: 2 m³ flops for an m × m block (LU
  // 2/3 m³ and the inverse from it 4/3 m³; Gauss–Jordan takes the same)
  L.factor_flops = 0.0;
  for (int64_t i = 0; i < L.nv; ++i) {
    const double n = (double)npv[i];
    if (L.kron)
      for (int b = 0; b < C.kplan.nblk; ++b) {
        const double q = (double)C.kplan.blk_size[b] * n;
        L.factor_flops += 2.0 * q * q * q;
      }
    else
      L.factor_flops += 2.0 * n * n * n;
  }
  for (int64_t i = 0; i < L.nv; ++i) {
    const int64_t np = npv[i];
    if (L.kron) {
      const int64_t xbytes = (C.kplan.nm * np * np * w + 15) / 16 * 16;
      off[i + 1] = off[i] + (xbytes + (np * 4 + 15) / 16 * 16) / w;
      continue;
    }
    const int64_t xbytes = (np * np * w + 15) / 16 * 16, gbytes = (np * 4 + 15) / 16 * 16;
    off[i + 1] = off[i] + (xbytes + gbytes * (L.big ? 2 : 1)) / w;
  }
  L.fac_elems = off[L.nv];
  if ((rc = upload(C, &L.d_order, order))) return rc;
  if ((rc = upload(C, &L.d_np, npv))) return rc;
  off.pop_back();
  if ((rc = upload(C, &L.d_fac_off, off))) return rc;
  const size_t esz = C.opt.patch_precision == 64 ? 8 : 4;
  void* fac = nullptr;
  cudaError_t e = cudaMalloc(&fac, esz * std::max<int64_t>(L.fac_elems, 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(IRKMG_ENOMEM, "patch inverses: " + std::to_string(esz * L.fac_elems) + " bytes");
  }
  C.allocs.push_back(fac);
  C.dev_bytes += esz * L.fac_elems;
  L.d_fac = fac;
  L.fixed = L.kron && C.opt.patch_fixed && fixed_fits(C, L);
  if (L.fixed) {
    std::vector<int16_t> ex((size_t)L.nv * C.kplan.nm * L.kron_nmax, 0);
    if ((rc = upload(C, &L.d_fexp, ex))) return rc;
  }
  if (L.kron)
    CK(launch_patch_gidx_kron(C, L));
  else
    CK(launch_patch_gidx(C, L));
  if (L.kron) {
    // one-launch relaxation, warp-per-patch (2D) levels: the results of the
    // patch of vertex v at i·ystride + v (local row i), and, per spatial DoF
    // d, its entries in ordered-patch (colour) order.  The per-DoF sum then
    // reads the results of neighbouring vertices from adjacent addresses,
    // and the launch takes the patches in vertex order, so that the writes
    // of one 32-byte sector come from neighbouring warps at about the same
    // time.  Levels of large (3D) patches, a CTA per patch streaming a
    // quarter-megabyte block, keep the patches in colour order (one
    // sequential stream of blocks) with each patch's results contiguous at
    // qoff[p] + i: measured at 32³, their apply took 1.92 ms per launch in
    // vertex order against 1.60 ms in colour order.
    const bool vorder = !L.kron_big;
    const int64_t ys = vorder ? (L.nv + 31) / 32 * 32 : 1;
    std::vector<int64_t> qoff(L.nv);
    std::vector<int32_t> perm(L.nv);
    int64_t Qent = 0, nloc = 0;
    for (int64_t p = 0; p < L.nv; ++p) {
      qoff[p] = vorder ? order[p] : Qent;
      perm[order[p]] = (int32_t)p;
      Qent += npv[p];
      nloc = std::max<int64_t>(nloc, npv[p]);
    }
    const int64_t Q = vorder ? nloc * ys : Qent;
    if (Q > INT32_MAX) return fail(IRKMG_ENOTIMPL, "patch results exceed 2^31 entries");
    std::vector<int32_t> cptr(L.m + 1, 0), cidx(Qent);
    auto dof = [&](int32_t v, int64_t i) -> int64_t {
      const int32_t nb = L.h_patch_ptr[v], nl = L.h_patch_ptr[v + 1] - nb;
      if (i < (int64_t)L.dim * nl) {
        const int64_t c = i / nl;
        return c * L.nf + L.h_patch_nodes[nb + i - c * nl];
      }
      return L.dim * L.nf + v;
    };
    for (int64_t p = 0; p < L.nv; ++p)
      for (int64_t i = 0; i < npv[p]; ++i) cptr[dof(order[p], i) + 1]++;
    for (int64_t d = 0; d < L.m; ++d) cptr[d + 1] += cptr[d];
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t p = 0; p < L.nv; ++p)
      for (int64_t i = 0; i < npv[p]; ++i)
        cidx[fill[dof(order[p], i)]++] = (int32_t)(i * ys + qoff[p]);
    if ((rc = upload(C, &L.d_qoff, qoff))) return rc;
    if (vorder && (rc = upload(C, &L.d_perm, perm))) return rc;
    if ((rc = upload(C, &L.d_cptr, cptr))) return rc;
    if ((rc = upload(C, &L.d_cidx, cidx))) return rc;
    L.Q = Q;
    L.Qent = Qent;
    L.ystride = ys;
    // the reduction reads every result and its index once, and out per DoF
    L.reduce_bytes = (double)C.s * (8.0 * Qent + 16.0 * L.m) + 4.0 * Qent + 4.0 * L.m;
  }
  return IRKMG_OK;
}

int factor_level(Ctx& C, Level& L) {
  if (L.kron && L.kron_big) {
    int q = 1;
    for (int b = 0; b < C.kplan.nblk; ++b) q = std::max(q, C.kplan.blk_size[b]);
    const int ctas = (int)std::min<int64_t>(L.nv, 2 * 152);
    const int64_t ws = kron_big_workspace(q * L.kron_nmax, L.kron_nmax, C.opt.patch_precision);
    const size_t esz = C.opt.patch_precision == 64 ? 8 : 4;
    void* work = nullptr;
    cudaError_t e = cudaMallocAsync(&work, esz * ws * ctas, C.stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(IRKMG_ENOMEM, "workspace for the decoupled large-patch factors");
    }
    e = launch_patch_factor_kron_big(C, L, work, ws, ctas);
    cudaError_t e2 = cudaFreeAsync(work, C.stream);
    CK(e);
    CK(e2);
    return IRKMG_OK;
  }
  if (L.kron) {
    CK(launch_patch_invert_kron(C, L));
    if (L.fixed) CK(launch_patch_to_fixed(C, L));
    return IRKMG_OK;
  }
  if (!L.big) {
    CK(launch_patch_invert(C, L, C.opt.patch_precision));
    return IRKMG_OK;
  }
  // large patches: blocked LU in place, then the explicit inverse from it
  CK(launch_patch_lu_big(C, L));
  const int ctas = (int)std::min<int64_t>(L.nv, 2 * 152);
  const int64_t ws = (int64_t)L.max_np * L.max_np;
  const size_t esz = C.opt.patch_precision == 64 ? 8 : 4;
  void* work = nullptr;
  cudaError_t e = cudaMallocAsync(&work, esz * ws * ctas, C.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(IRKMG_ENOMEM, "workspace for the large-patch inverses");
  }
  e = launch_patch_inv_from_lu(C, L, work, ws, ctas);
  cudaError_t e2 = cudaFreeAsync(work, C.stream);
  CK(e);
  CK(e2);
  return IRKMG_OK;
}

int factor_coarse(Ctx& C) {
  CK(launch_coarse_build(C, C.d_coarse_inv));
  CK(coarse_invert(C, C.d_coarse_inv, C.nb));
  return IRKMG_OK;
}

int assemble_all(Ctx& C) {
  const int nl = (int)C.L.size();
  std::vector<std::vector<double>> winds(nl);
  if (!C.wind.empty()) {
    winds[nl - 1] = C.wind;
    for (int l = nl - 2; l >= 0; --l)
      winds[l].assign(winds[l + 1].begin(), winds[l + 1].begin() + 2 * C.L[l].np2);
  }
  for (int l = 0; l < nl; ++l)
    assemble_level(C.L[l].mesh, C.nu, winds[l].empty() ? nullptr : winds[l].data(), C.L[l].hops);
  return IRKMG_OK;
}

int factor_all(Ctx& C) {
  int rc;
  for (size_t l = 1; l < C.L.size(); ++l) {
    cudaEvent_t a = nullptr, b = nullptr;
    const bool traced = C.trace_on && l + 1 == C.L.size();  // the finest level
    if (traced) {
      if ((rc = trace_pair(C, 5, 0.0, &a, &b, C.L[l].factor_flops))) return rc;
      CK(cudaEventRecord(a, C.stream));
    }
    if ((rc = factor_level(C, C.L[l]))) return rc;
    if (traced) CK(cudaEventRecord(b, C.stream));
  }
  if ((rc = factor_coarse(C))) return rc;
  CK(cudaStreamSynchronize(C.stream));
  return check_err(C, "factorisation");
}

int vanka_all(Ctx& C, Level& L, const double* r, double* out, double scale, int tr,
              const ChebFuse* fuse = nullptr);

// Choose the Vanka apply kernel of every level: the option forces one, or
// (apply_variant 0) both are timed on one sweep of the level (after a warm-up
// sweep) with CUDA events on the context stream and the faster is kept.
int tune_apply(Ctx& C) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  const bool saved = C.trace_on;
  C.trace_on = false;
  int rc = IRKMG_OK;
  for (size_t l = 1; l < C.L.size() && rc == IRKMG_OK; ++l) {
    Level& L = C.L[l];
    if (L.big && !L.kron) {
      L.apply_kernel = 3;
      continue;
    }
    if (L.kron_big) {
      // one kernel (CTA per patch); per-colour launches or one launch + sum
      L.apply_kernel = 6;
      L.single = false;
      const int av = C.opt.apply_variant;
      if (av != 0) {
        L.single = av >= 3;
        continue;
      }
      cudaError_t ez = cudaMemsetAsync(L.t, 0, sizeof(double) * L.N, C.stream);
      if (ez != cudaSuccess) { rc = fail(IRKMG_ECUDA, cudaGetErrorString(ez)); break; }
      float t2[2] = {0.f, 0.f};
      for (int single = 0; single < 2 && rc == IRKMG_OK; ++single) {
        L.single = single != 0;
        float best = 1e30f;
        for (int rep = 0; rep < 3 && rc == IRKMG_OK; ++rep) {
          cudaEventRecord(a, C.stream);
          rc = vanka_all(C, L, L.t, L.d, 1.0, 0);
          cudaEventRecord(b, C.stream);
          cudaError_t e2 = cudaEventSynchronize(b);
          if (e2 != cudaSuccess) { rc = fail(IRKMG_ECUDA, cudaGetErrorString(e2)); break; }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, a, b);
          if (rep > 0 && ms < best) best = ms;
        }
        t2[single] = best;
      }
      L.single = t2[1] < t2[0];
      L.apply_ms[1] = 0.f;
      L.apply_ms[2] = std::min(t2[0], t2[1]);
      continue;
    }
    if (L.fixed) {
      // one kernel (warp per patch, fixed point): its launch shapes and both
      // relaxation modes timed, unless the variant fixes the mode
      L.apply_kernel = 8;
      L.single = false;
      L.kron_shape = 0;
      const int av = C.opt.apply_variant;
      if (av != 0) {
        L.single = av == 3 || av == 4 || av == 6;
        continue;
      }
      cudaError_t ez = cudaMemsetAsync(L.t, 0, sizeof(double) * L.N, C.stream);
      if (ez != cudaSuccess) { rc = fail(IRKMG_ECUDA, cudaGetErrorString(ez)); break; }
      float best_all = 1e30f;
      int pick_shape = 0;
      bool pick_single = false;
      for (int single = 0; single < 2 && rc == IRKMG_OK; ++single)
        for (int shape = 0; shape < fixed_shapes() && rc == IRKMG_OK; ++shape) {
          if (!fixed_shape_fits(C, L, shape)) continue;
          L.single = single != 0;
          L.kron_shape = shape;
          L.apply_kernel = fixed_shape_kernel(shape);
          float best = 1e30f;
          for (int rep = 0; rep < 3 && rc == IRKMG_OK; ++rep) {
            cudaEventRecord(a, C.stream);
            rc = vanka_all(C, L, L.t, L.d, 1.0, 0);
            cudaEventRecord(b, C.stream);
            cudaError_t e2 = cudaEventSynchronize(b);
            if (e2 != cudaSuccess) { rc = fail(IRKMG_ECUDA, cudaGetErrorString(e2)); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < best) best = ms;
          }
          if (best < best_all) {
            best_all = best;
            pick_shape = shape;
            pick_single = single != 0;
          }
        }
      L.single = pick_single;
      L.kron_shape = pick_shape;
      L.apply_kernel = fixed_shape_kernel(pick_shape);
      L.apply_ms[1] = 0.f;
      L.apply_ms[2] = best_all;
      continue;
    }
    // candidates: staged (TMA) and warp-per-patch kernels, dense or decoupled;
    // on decoupled levels each staged launch shape, and both relaxation
    // modes (one launch per colour, or one launch and the per-DoF reduction)
    const int ks = L.kron ? 5 : 1, kw = L.kron ? 4 : 2;
    L.kron_shape = 0;
    L.single = false;
    const bool fits = L.kron ? kron_staged_fits(C, L, 0) : vanka_staged_fits(C, L);
    const int av = C.opt.apply_variant;
    if (av != 0) {
      const bool staged = (av == 1 || av == 3) && fits;
      L.apply_kernel = staged ? ks : kw;
      if (av >= 5 && L.kron && kron_ws_fits(C, L)) L.apply_kernel = 7;
      L.single = L.kron && (av == 3 || av == 4 || av == 6);
      continue;
    }
    struct Cand { int kern, shape; bool single; };
    std::vector<Cand> cands;
    for (int single = 0; single <= (L.kron ? 1 : 0); ++single) {
      if (fits)
        for (int shape = 0; shape < (L.kron ? 2 : 1); ++shape) cands.push_back({ks, shape, single != 0});
      cands.push_back({kw, 0, single != 0});
      if (L.kron && L.kron_nmax <= kron_big_max_n()) cands.push_back({6, 0, single != 0});
      if (L.kron && kron_ws_fits(C, L)) cands.push_back({7, 0, single != 0});
    }
    cudaError_t e = cudaMemsetAsync(L.t, 0, sizeof(double) * L.N, C.stream);
    if (e != cudaSuccess) { rc = fail(IRKMG_ECUDA, cudaGetErrorString(e)); break; }
    float best_all = 1e30f;
    Cand pick = cands.back();
    L.apply_ms[1] = L.apply_ms[2] = 0.f;
    float best_kind[2] = {1e30f, 1e30f};
    for (const Cand& cd : cands) {
      if (rc != IRKMG_OK) break;
      L.apply_kernel = cd.kern;
      L.kron_shape = cd.shape;
      L.single = cd.single;
      float best = 1e30f;
      for (int rep = 0; rep < 3 && rc == IRKMG_OK; ++rep) {
        cudaEventRecord(a, C.stream);
        rc = vanka_all(C, L, L.t, L.d, 1.0, 0);
        cudaEventRecord(b, C.stream);
        cudaError_t e2 = cudaEventSynchronize(b);
        if (e2 != cudaSuccess) { rc = fail(IRKMG_ECUDA, cudaGetErrorString(e2)); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;   // rep 0 is the warm-up
      }
      const int kind = cd.kern == kw ? 1 : 0;  // [0]: staged or CTA-per-patch, [1]: warp
      best_kind[kind] = std::min(best_kind[kind], best);
      if (best < best_all) {
        best_all = best;
        pick = cd;
      }
    }
    L.apply_ms[1] = best_kind[0] < 1e29f ? best_kind[0] : 0.f;
    L.apply_ms[2] = best_kind[1] < 1e29f ? best_kind[1] : 0.f;
    L.apply_kernel = pick.kern;
    L.kron_shape = pick.shape;
    L.single = pick.single;
  }
  C.trace_on = saved;
  C.launches = 0;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  CK(cudaStreamSynchronize(C.stream));
  return check_err(C, "apply autotuning");
}

// --- smoothers and V-cycle -------------------------------------------------
// fuse (one-launch levels only, L.kron && L.single): the Chebyshev update
// carried out by the per-DoF sum (ChebFuse).
int vanka_all(Ctx& C, Level& L, const double* r, double* out, double scale, int tr,
              const ChebFuse* fuse) {
  if (L.big && tr)
    return fail(IRKMG_ENOTIMPL, "transposed patch solves of LU-factored (3D) patches");
  const bool timed = C.trace_on && &L == &C.L.back();
  if (L.kron && L.single) {
    // one launch over all patches into d_Y, then the deterministic per-DoF sum
    cudaEvent_t a = nullptr, b = nullptr, c2 = nullptr, d2 = nullptr;
    if (timed) {
      double bytes = 0.0, flops = 0.0;
      for (int c = 0; c < L.ncolours; ++c) {
        bytes += L.colour_bytes[c];
        flops += L.colour_flops[c];
      }
      // the colour bytes count r and out per DoF; here the launch reads r and
      // writes its results once (24 B per stage DoF either way)
      int rc = trace_pair(C, 0, bytes, &a, &b, flops);
      if (rc) return rc;
      CK(cudaEventRecord(a, C.stream));
    }
    CK(launch_vanka_kron(C, L, -1, r, out, scale, tr));
    C.launches++;
    if (timed) {
      CK(cudaEventRecord(b, C.stream));
      // fused: x read (added) and written, d not read when zeroed
      const double xb = fuse ? 8.0 * (double)L.N * ((fuse->xadd ? 2.0 : 1.0) - (fuse->dzero ? 1.0 : 0.0))
                             : 0.0;
      int rc = trace_pair(C, 2, L.reduce_bytes + xb, &c2, &d2, 0.0);
      if (rc) return rc;
      CK(cudaEventRecord(c2, C.stream));
    }
    CK(launch_vanka_reduce(C, L, out, scale, fuse));
    C.launches++;
    if (timed) CK(cudaEventRecord(d2, C.stream));
    return IRKMG_OK;
  }
  if (fuse) return fail(IRKMG_EINVAL, "fused Chebyshev step on a per-colour level");
  for (int c = 0; c < L.ncolours; ++c) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) {
      int rc = trace_pair(C, 0, L.colour_bytes[c], &a, &b, L.colour_flops[c]);
      if (rc) return rc;
      CK(cudaEventRecord(a, C.stream));
    }
    if (L.kron)
      CK(launch_vanka_kron(C, L, c, r, out, scale, tr));
    else if (L.big)
      CK(launch_vanka_big(C, L, c, r, out, scale));
    else
      CK(launch_vanka(C, L, c, r, out, scale, tr));
    C.launches++;
    if (timed) CK(cudaEventRecord(b, C.stream));
  }
  return IRKMG_OK;
}

// nsteps relaxation steps on J x = b from x (x == 0 on entry if zero_init).
int smooth(Ctx& C, Level& L, const double* b, double* x, int nsteps, bool zero_init, int tr) {
  if (nsteps <= 0) {
    if (zero_init) CK(launch_fill(x, 0.0, L.N, C.stream));
    C.launches += zero_init ? 1 : 0;
    return IRKMG_OK;
  }
  int rc;
  if (C.opt.smoother == 0) {
    if (zero_init) {
      CK(launch_fill(x, 0.0, L.N, C.stream));
      C.launches++;
    }
    for (int k = 0; k < nsteps; ++k) {
      const double* res = b;
      if (!(zero_init && k == 0)) {
        { int rc_ = op(C, L, b, x, L.t, tr); if (rc_) return rc_; }
        res = L.t;
      }
      if ((rc = vanka_all(C, L, res, x, C.opt.omega, tr))) return rc;
    }
    return IRKMG_OK;
  }
  const double theta = 0.5 * (L.cheb_hi + L.cheb_lo);
  const double delta = 0.5 * (L.cheb_hi - L.cheb_lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const double* res = b;
  if (!zero_init) {
    { int rc_ = op(C, L, b, x, L.t, tr); if (rc_) return rc_; }
    res = L.t;
  }
  if (L.kron && L.single) {
    // one-launch levels: the per-DoF sum also scales d and updates x (the
    // same roundings as the fill / axpby launches below)
    ChebFuse f{0.0, true, !zero_init, x};
    if ((rc = vanka_all(C, L, res, L.d, 1.0 / theta, tr, &f))) return rc;
    for (int k = 1; k < nsteps; ++k) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      { int rc_ = op(C, L, b, x, L.t, tr); if (rc_) return rc_; }
      ChebFuse g{rho_new * rho, false, true, x};
      if ((rc = vanka_all(C, L, L.t, L.d, 2.0 * rho_new / delta, tr, &g))) return rc;
      rho = rho_new;
    }
    return IRKMG_OK;
  }
  CK(launch_fill(L.d, 0.0, L.N, C.stream));
  C.launches++;
  if ((rc = vanka_all(C, L, res, L.d, 1.0 / theta, tr))) return rc;
  if (zero_init) {
    CK(cudaMemcpyAsync(x, L.d, sizeof(double) * L.N, cudaMemcpyDeviceToDevice, C.stream));
  } else {
    CK(launch_axpby(x, L.d, 1.0, 1.0, L.N, C.stream));
    C.launches++;
  }
  for (int k = 1; k < nsteps; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    { int rc_ = op(C, L, b, x, L.t, tr); if (rc_) return rc_; }
    CK(launch_axpby(L.d, L.d, rho_new * rho, 0.0, L.N, C.stream));
    if ((rc = vanka_all(C, L, L.t, L.d, 2.0 * rho_new / delta, tr))) return rc;
    CK(launch_axpby(x, L.d, 1.0, 1.0, L.N, C.stream));
    C.launches += 2;
    rho = rho_new;
  }
  return IRKMG_OK;
}

int coarse_graph(Ctx& C, int tr);
int coarse_correction(Ctx& C, int l, const double* b, double* z, int tr);

int vcycle_level(Ctx& C, int l, const double* b, double* z, int tr) {
  if (l == 0) {
    CK(launch_coarse_apply(C, b, z, tr));
    C.launches++;
    return IRKMG_OK;
  }
  int rc;
  if ((rc = smooth(C, C.L[l], b, z, C.opt.nu_pre, true, tr))) return rc;
  if ((rc = coarse_correction(C, l, b, z, tr))) return rc;
  return smooth(C, C.L[l], b, z, C.opt.nu_post, false, tr);
}

// z += (I_s ⊗ P) V-cycle_{l-1}((I_s ⊗ P)ᵀ (b - J z)) on level l >= 1: the
// residual, its restriction, the coarse levels (one graph launch below the
// finest level), the prolongation added into z.
int coarse_correction(Ctx& C, int l, const double* b, double* z, int tr) {
  Level& L = C.L[l];
  Level& Lc = C.L[l - 1];
  int rc;
  { int rc_ = op(C, L, b, z, L.t, tr); if (rc_) return rc_; }
  const bool timed = C.trace_on && l == (int)C.L.size() - 1;
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (timed) {  // restriction reads the fine vector and writes the coarse one
    if ((rc = trace_pair(C, 3, 8.0 * (double)(L.N + Lc.N), &ta, &tb))) return rc;
    CK(cudaEventRecord(ta, C.stream));
  }
  CK(launch_restrict(C, L, L.t, Lc.r));
  if (timed) CK(cudaEventRecord(tb, C.stream));
  if (l == (int)C.L.size() - 1 && l >= 2 && !C.capturing) {
    // everything below the finest level: one graph launch
    if ((rc = coarse_graph(C, tr))) return rc;
    CK(cudaEventRecord(C.gev[0], C.stream));
    CK(cudaStreamWaitEvent(C.gstream, C.gev[0], 0));
    CK(cudaGraphLaunch(C.cgraph[tr], C.gstream));
    CK(cudaEventRecord(C.gev[1], C.gstream));
    CK(cudaStreamWaitEvent(C.stream, C.gev[1], 0));
    C.launches += C.cgraph_launches[tr];
  } else if ((rc = vcycle_level(C, l - 1, Lc.r, Lc.z, tr))) {
    return rc;
  }
  if (timed) {  // prolongation reads the coarse vector and updates the fine one
    if ((rc = trace_pair(C, 3, 8.0 * (double)(Lc.N + 2 * L.N), &ta, &tb))) return rc;
    CK(cudaEventRecord(ta, C.stream));
  }
  CK(launch_prolong(C, L, Lc.z, z, 1));
  if (timed) CK(cudaEventRecord(tb, C.stream));
  C.launches += 2;
  return IRKMG_OK;
}

// --- FGMRES (Section 4) -----------------------------------------------------
int fgmres(Ctx& C, const double* F, double* x, irkmg_stats* st, int tr) {
  Level& L = C.L.back();
  const int64_t n = L.N;
  const int m = C.opt.restart;
  const double t0 = now();
  double* V = C.d_V;
  double* Z = C.d_Z;
  double* w = C.d_w;
  double* hd = C.d_h;       // device: [0..m] h1, [64..] h2, [128] norm
  double* hh = C.h_h;       // pinned host mirror
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
  auto norm = [&](const double* v, double* out) -> int {
    CK(launch_multidot(v, 0, 1, v, n, C.d_part, hd + 192, C.stream));
    C.launches += 2;
    CK(cudaMemcpyAsync(hh + 192, hd + 192, sizeof(double), cudaMemcpyDeviceToHost, C.stream));
    CK(cudaStreamSynchronize(C.stream));
    *out = std::sqrt(hh[192]);
    return IRKMG_OK;
  };
  int rc;
  double bnorm;
  if ((rc = norm(F, &bnorm))) return rc;
  const double target = std::max(C.opt.rtol * bnorm, C.opt.atol);
  if ((rc = op(C, L, F, x, V, tr))) return rc;
  double beta;
  if ((rc = norm(V, &beta))) return rc;
  if (st) {
    st->r0 = beta;
    st->iters = 0;
  }
  int its = 0;
  while (beta > target && its < C.opt.maxit) {
    CK(launch_axpby(V, V, 1.0 / beta, 0.0, n, C.stream));
    C.launches++;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (int64_t)j * n;
      double* zj = Z + (int64_t)j * n;
      if ((rc = vcycle_level(C, (int)C.L.size() - 1, vj, zj, tr))) return rc;
      CK(launch_pressure_mean_remove(C, L, zj));
      C.launches++;
      if ((rc = op(C, L, nullptr, zj, w, tr))) return rc;
      // classical Gram–Schmidt, twice
      cudaEvent_t ga = nullptr, gb = nullptr;
      if (C.trace_on) {
        // k = j + 1 basis vectors: the dot products read V and w; each update
        // reads V and w and writes w, fused with the next dot products (or
        // ||w||²) when k <= 16; otherwise every update and reduction reads
        // its vectors again
        const double k1 = (double)(j + 1), nb = 8.0 * (double)n;
        const double bytes = j + 1 <= 16 ? nb * (3.0 * k1 + 5.0)
                                         : 2.0 * (nb * (k1 + 1.0) + nb * (k1 + 2.0)) + nb;
        if ((rc = trace_pair(C, 4, bytes, &ga, &gb))) return rc;
        CK(cudaEventRecord(ga, C.stream));
      }
      CK(launch_multidot(V, n, j + 1, w, n, C.d_part, hd, C.stream));
      CK(launch_multiaxpy_dot(w, V, n, j + 1, hd, -1.0, n, C.d_part, hd + 64, false, C.stream));
      CK(launch_multiaxpy_dot(w, V, n, j + 1, hd + 64, -1.0, n, C.d_part, hd + 128, true,
                              C.stream));
      if (C.trace_on) CK(cudaEventRecord(gb, C.stream));
      C.launches += j + 1 <= 16 ? 6 : 10;
      CK(cudaMemcpyAsync(hh, hd, sizeof(double) * 129, cudaMemcpyDeviceToHost, C.stream));
      CK(cudaMemcpyAsync(C.h_err, C.d_err, sizeof(int) * 2, cudaMemcpyDeviceToHost, C.stream));
      CK(cudaStreamSynchronize(C.stream));
      if (C.h_err[0] != 0) {
        const int code = C.h_err[0];
        CK(cudaMemsetAsync(C.d_err, 0, sizeof(int) * 2, C.stream));
        if (st) st->status = code;
        return fail(code, "a bounded device-side wait expired during the V-cycle");
      }
      double* Hj = &H[(size_t)j * (m + 1)];  // column j, length m+1
      for (int i = 0; i <= j; ++i) Hj[i] = hh[i] + hh[64 + i];
      const double hn = std::sqrt(hh[128]);
      Hj[j + 1] = hn;
      if (hn > 0.0) {
        CK(launch_axpby(V + (int64_t)(j + 1) * n, w, 1.0 / hn, 0.0, n, C.stream));
        C.launches++;
      }
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
        Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
        Hj[i] = a;
      }
      const double den = std::hypot(Hj[j], Hj[j + 1]);
      cs[j] = Hj[j] / den;
      sn[j] = Hj[j + 1] / den;
      Hj[j] = den;
      Hj[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) <= target || its >= C.opt.maxit || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jdone; ++k) s -= H[(size_t)k * (m + 1) + i] * y[k];
      y[i] = s / H[(size_t)i * (m + 1) + i];
    }
    std::copy(y.begin(), y.begin() + jdone, hh + 256);
    CK(cudaMemcpyAsync(hd + 256, hh + 256, sizeof(double) * jdone, cudaMemcpyHostToDevice,
                       C.stream));
    CK(launch_multiaxpy(x, Z, n, jdone, hd + 256, 1.0, n, C.stream));
    C.launches++;
    if ((rc = op(C, L, F, x, V, tr))) return rc;
    if ((rc = norm(V, &beta))) return rc;
  }
  if (st) {
    st->iters = its;
    st->rfinal = beta;
    st->t_solve = now() - t0;
    st->status = beta <= target ? IRKMG_OK : IRKMG_ENOCONV;
    st->bad_index = -1;
  }
  if (beta > target) return fail(IRKMG_ENOCONV, "FGMRES reached maxit");
  return IRKMG_OK;
}

int validate(const irkmg_mesh* mesh, const irkmg_tableau* tab, double dt, double nu,
             const irkmg_options* o) {
  if (!mesh || !tab || !o) return fail(IRKMG_EINVAL, "null argument");
  if (mesh->dim != 2 && mesh->dim != 3)
    return fail(IRKMG_ENOTIMPL, "dim must be 2 (triangles) or 3 (tetrahedra)");
  if (mesh->dim == 3 && o->wind)
    return fail(IRKMG_ENOTIMPL, "the Oseen wind is built for 2D meshes only");
  if (!mesh->coords || !mesh->cells || !mesh->bnd_vertex) return fail(IRKMG_EINVAL, "mesh arrays");
  if (tab->s < 1 || tab->s > 3 || !tab->A || !tab->b || !tab->c)
    return fail(IRKMG_EINVAL, "tableau: 1 <= s <= 3 and A, b, c required");
  double sb = 0.0;
  for (int j = 0; j < tab->s; ++j) sb += tab->b[j];
  if (std::fabs(sb - 1.0) > 1e-12) return fail(IRKMG_EINVAL, "tableau: sum b != 1");
  for (int i = 0; i < tab->s; ++i) {
    double sa = 0.0;
    for (int j = 0; j < tab->s; ++j) sa += tab->A[i * tab->s + j];
    if (std::fabs(sa - tab->c[i]) > 1e-12) return fail(IRKMG_EINVAL, "tableau: row sum != c");
  }
  if (!(dt > 0.0) || !(nu > 0.0)) return fail(IRKMG_EINVAL, "dt and nu must be positive");
  if (o->nlevels < 2 || o->nlevels > 12) return fail(IRKMG_EINVAL, "nlevels in [2, 12]");
  if (o->nu_pre < 0 || o->nu_post < 0) return fail(IRKMG_EINVAL, "negative sweep count");
  if (o->smoother != 0 && o->smoother != 1) return fail(IRKMG_EINVAL, "smoother is 0 or 1");
  if (o->smoother == 1 && !o->cheb_auto && !(o->cheb_hi > o->cheb_lo && o->cheb_lo > 0.0))
    return fail(IRKMG_EINVAL, "Chebyshev interval needs 0 < lo < hi");
  if (o->cheb_auto != 0 && o->cheb_auto != 1) return fail(IRKMG_EINVAL, "cheb_auto is 0 or 1");
  if (o->cheb_auto && o->smoother != 1) return fail(IRKMG_EINVAL, "cheb_auto needs smoother 1");
  if (o->restart < 1 || o->restart > 60) return fail(IRKMG_EINVAL, "restart in [1, 60]");
  if (o->maxit < 1) return fail(IRKMG_EINVAL, "maxit >= 1");
  if (o->patch_precision != 64 && o->patch_precision != 32)
    return fail(IRKMG_EINVAL, "patch_precision is 64 or 32");
  if (o->apply_variant < 0 || o->apply_variant > 6)
    return fail(IRKMG_EINVAL, "apply_variant is 0 .. 6");
  if (o->patch_form < 0 || o->patch_form > 3)
    return fail(IRKMG_EINVAL, "patch_form is 0, 1, 2 or 3");
  if (o->patch_lu_tc != 0 && o->patch_lu_tc != 1) return fail(IRKMG_EINVAL, "patch_lu_tc is 0 or 1");
  if (o->patch_fixed != 0 && o->patch_fixed != 1) return fail(IRKMG_EINVAL, "patch_fixed is 0 or 1");
  if (o->op_fixed != 0 && o->op_fixed != 1) return fail(IRKMG_EINVAL, "op_fixed is 0 or 1");
  if (o->patch_form != 0) {
    KronSplit K;
    if (kron_split(tab->s, tab->A, &K) != IRKMG_OK)
      return fail(IRKMG_ENOTIMPL,
                  "decoupled patch solves need a Butcher matrix with distinct eigenvalues");
  }
  if (o->timeout_spins < 0) return fail(IRKMG_EINVAL, "timeout_spins >= 0");
  return IRKMG_OK;
}

int set_chebyshev_intervals(Ctx& C);
void drop_graphs(Ctx& C);
int estimate_lambda(Ctx& C, Level& L, int k, const double* x0, double* ritz_re, double* ritz_im,
                    double* lambda);

int setup_impl(irkmg_ctx* C, const irkmg_mesh* mesh, const irkmg_tableau* tab, double dt,
               double nu, const irkmg_options* opt) {
  const double t0 = now();
  C->opt = *opt;
  C->s = tab->s;
  std::memcpy(C->A, tab->A, sizeof(double) * tab->s * tab->s);
  std::memcpy(C->b, tab->b, sizeof(double) * tab->s);
  std::memcpy(C->c, tab->c, sizeof(double) * tab->s);
  C->dt = dt;
  C->nu = nu;
  C->stream = (cudaStream_t)opt->cuda_stream;
  int rc;
  if (opt->patch_form != 0) {
    KronSplit K;
    if (kron_split(C->s, C->A, &K) != IRKMG_OK) return fail(IRKMG_ENOTIMPL, "Butcher matrix split");
    // patch_form 1: the complex layout (s·n² entries) where the apply is
    // bound by memory traffic (FP32 entries, and 2D FP64 entries applied in
    // fixed point), the three-product layout (fewest FP64 multiply-adds)
    // where the FP64 pipe bounds it
    const bool traffic_bound =
        opt->patch_precision == 32 || (opt->patch_fixed == 1 && mesh->dim == 2);
    const int layout = opt->patch_form == 2 ? 1
                       : opt->patch_form == 3 ? 2
                                              : (traffic_bound ? 1 : 2);
    if ((rc = kron_plan(K, layout, &C->kplan))) return fail(rc, "decoupled patch plan");
    C->kron = true;
  }
  const int nl = opt->nlevels;
  C->L.resize(nl);
  C->dim = mesh->dim;
  std::string why = build_mesh(mesh->coords, mesh->cells, mesh->bnd_vertex, mesh->nverts,
                               mesh->ncells, mesh->dim, C->L[0].mesh);
  if (!why.empty()) return fail(IRKMG_EINVAL, why);
  for (int l = 1; l < nl; ++l) {
    if (C->L[l - 1].mesh.np2 > (1LL << 30)) return fail(IRKMG_EINVAL, "hierarchy too large");
    refine_mesh(C->L[l - 1].mesh, C->L[l].mesh);
  }
  if (opt->wind) C->wind.assign(opt->wind, opt->wind + 2 * C->L[nl - 1].mesh.np2);
  for (int l = 0; l < nl; ++l) {
    Level& L = C->L[l];
    L.dim = C->dim;
    L.nv = L.mesh.nv;
    L.nf = L.mesh.nf;
    L.np2 = L.mesh.np2;
    L.m = L.dim * L.nf + L.nv;
    L.N = C->s * L.m;
  }
  if ((rc = assemble_all(*C))) return rc;
  CK(cudaMalloc(&C->d_err, sizeof(int) * 2));
  C->allocs.push_back(C->d_err);
  CK(cudaMemset(C->d_err, 0, sizeof(int) * 2));
  for (int l = 0; l < nl; ++l) {
    Level& L = C->L[l];
    if ((rc = upload_csr(*C, L.vel, L.hops.vel, 3))) return rc;
    if ((rc = upload_csr(*C, L.b, L.hops.b, L.dim))) return rc;
    if ((rc = upload_csr(*C, L.bt, L.hops.bt, L.dim))) return rc;
    if ((rc = upload_sell(*C, L.svel, L.hops.vel, 3))) return rc;
    if ((rc = upload_sell(*C, L.sb, L.hops.b, L.dim))) return rc;
    if ((rc = upload_sell(*C, L.sbt, L.hops.bt, L.dim))) return rc;
    if (l == nl - 1 && (rc = upload_csr(*C, L.mall, L.hops.mall, 2))) return rc;
    if (l == nl - 1 && (rc = upload_csr(*C, L.btall, L.hops.btall, L.dim))) return rc;
    if (op_fixed_fits(*C, L)) {  // fixed-point copies of the operator rows
      FxOpLevel& X = L.fxop;
      if ((rc = dalloc(*C, &X.qM, L.svel.stored))) return rc;
      if ((rc = dalloc(*C, &X.qK, L.svel.stored))) return rc;
      if ((rc = dalloc(*C, &X.qB[0], L.sb.stored))) return rc;
      if ((rc = dalloc(*C, &X.qB[1], L.sb.stored))) return rc;
      if ((rc = dalloc(*C, &X.qT[0], L.sbt.stored))) return rc;
      if ((rc = dalloc(*C, &X.qT[1], L.sbt.stored))) return rc;
      if ((rc = dalloc(*C, &X.eM, L.nf))) return rc;
      if ((rc = dalloc(*C, &X.eK, L.nf))) return rc;
      if ((rc = dalloc(*C, &X.eB[0], L.nf))) return rc;
      if ((rc = dalloc(*C, &X.eB[1], L.nf))) return rc;
      if ((rc = dalloc(*C, &X.eT, L.nv))) return rc;
      if ((rc = dalloc(*C, &X.xl, L.N))) return rc;
      if ((rc = dalloc(*C, &X.bmax, 6))) return rc;
      CK(launch_op_fixed_convert(*C, L));
      L.fxop_on = true;
    }
    if ((rc = dalloc(*C, &L.r, L.N))) return rc;
    if ((rc = dalloc(*C, &L.z, L.N))) return rc;
    if ((rc = dalloc(*C, &L.t, L.N))) return rc;
    if ((rc = dalloc(*C, &L.d, L.N))) return rc;
    if (l > 0) {
      HostCSR Pu, Pp;
      build_prolongation(C->L[l - 1].mesh, L.mesh, Pu, Pp);
      if ((rc = upload_sell(*C, L.pu, Pu, 1, true))) return rc;
      if ((rc = upload_sell(*C, L.put, transpose_csr(Pu, 1), 1, true))) return rc;
      if ((rc = upload_sell(*C, L.pp, Pp, 1, true))) return rc;
      if ((rc = upload_sell(*C, L.ppt, transpose_csr(Pp, 1), 1, true))) return rc;
      if ((rc = build_patches(*C, L))) return rc;
      level_trace_bytes(*C, L);
    }
    L.op_bytes = 20.0 * (double)L.vel.nnz + 20.0 * (double)(L.b.nnz + L.bt.nnz) + 24.0 * (double)L.N;
    {
      const double s = (double)C->s;
      L.op_flops = 2.0 * (4.0 * s * (double)L.vel.nnz + 2.0 * s * (double)(L.b.nnz + L.bt.nnz) +
                          2.0 * s * s * (double)L.nf + s * s * (double)L.nv);
    }
  }
  {
    Level& Lf = C->L[nl - 1];
    HostCSR cl;
    assemble_cell_load(Lf.mesh, cl);
    if ((rc = upload_csr(*C, C->cload, cl, 1))) return rc;
    if ((rc = upload_csr(*C, C->cloadt, transpose_csr(cl, 1), 1))) return rc;
    if ((rc = dalloc(*C, &C->d_F, Lf.N))) return rc;
    if ((rc = dalloc(*C, &C->d_kb, Lf.N))) return rc;
    if ((rc = dalloc(*C, &C->d_lam, Lf.N))) return rc;
    if ((rc = dalloc(*C, &C->d_scalar, 8))) return rc;
  }
  if (C->kron) {
    int64_t qmax = 0;
    for (const Level& L : C->L) qmax = std::max(qmax, L.Q);
    if (qmax > 0 && (rc = dalloc(*C, &C->d_Y, (size_t)C->s * qmax))) return rc;
  }
  C->nb = C->L[0].N + C->s;
  if (C->nb > 20000) return fail(IRKMG_EINVAL, "coarsest level too large for the dense solve");
  if ((rc = dalloc(*C, &C->d_coarse_inv, (size_t)C->nb * C->nb))) return rc;
  if ((rc = dalloc(*C, &C->d_coarse_perm, C->nb))) return rc;
  const int64_t n = C->L.back().N;
  const int m = opt->restart;
  if ((rc = dalloc(*C, &C->d_V, (size_t)(m + 1) * n))) return rc;
  if ((rc = dalloc(*C, &C->d_Z, (size_t)m * n))) return rc;
  if ((rc = dalloc(*C, &C->d_w, n))) return rc;
  if ((rc = dalloc(*C, &C->d_part, (size_t)kMultidotBlocks * 64))) return rc;
  if ((rc = dalloc(*C, &C->d_h, 512))) return rc;
  CK(cudaMallocHost(&C->h_h, sizeof(double) * 512));
  CK(cudaMallocHost(&C->h_err, sizeof(int) * 2));
  if ((rc = factor_all(*C))) return rc;
  if ((rc = tune_apply(*C))) return rc;
  if ((rc = set_chebyshev_intervals(*C))) return rc;
  (void)t0;
  return IRKMG_OK;
}

bool level_ok(const irkmg_ctx* ctx, int level) {
  return ctx && level >= 0 && level < (int)ctx->L.size();
}

// --- relaxation without device allocation -----------------------------------
// Work vectors for irkmg_smooth_noalloc: [0, kNoallocMaxN) holds the residual,
// [kNoallocMaxN, 2 kNoallocMaxN) the Chebyshev direction.  Host code cannot
// use the symbol as an address: the device address is looked up with the
// device current.  A call outside stream capture looks it up again (the
// module, and so the array, moves if the device's context was torn down and
// re-created); a call during capture, when no lookup that might load a module
// is wanted, uses the address the last uncaptured call on that device found.
constexpr int64_t kNoallocMaxN = 1 << 19;
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxN];
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoallocMaxDevices] = {};

int noalloc_scratch(cudaStream_t st, double** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(IRKMG_EINVAL, "device index out of range");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = (double*)p;
  } else if (!g_noalloc_ptr[dev]) {
    return fail(IRKMG_EINVAL, "the first no-allocation call on a device must come before any "
                              "stream capture");
  }
  *out = g_noalloc_ptr[dev];
  return IRKMG_OK;
}

// nsteps relaxation steps on J x = b from x, with the residual in t and the
// Chebyshev direction in d (both caller-provided, length >= L.N).
int smooth_in(Ctx& C, Level& L, const double* b, double* x, int nsteps, int tr, double* t,
              double* d) {
  if (nsteps <= 0) return IRKMG_OK;
  int rc;
  if (C.opt.smoother == 0) {
    for (int k = 0; k < nsteps; ++k) {
      if ((rc = op(C, L, b, x, t, tr))) return rc;
      if ((rc = vanka_all(C, L, t, x, C.opt.omega, tr))) return rc;
    }
    return IRKMG_OK;
  }
  const double theta = 0.5 * (L.cheb_hi + L.cheb_lo);
  const double delta = 0.5 * (L.cheb_hi - L.cheb_lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  if ((rc = op(C, L, b, x, t, tr))) return rc;
  CK(launch_fill(d, 0.0, L.N, C.stream));
  C.launches++;
  if ((rc = vanka_all(C, L, t, d, 1.0 / theta, tr))) return rc;
  CK(launch_axpby(x, d, 1.0, 1.0, L.N, C.stream));
  C.launches++;
  for (int k = 1; k < nsteps; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    if ((rc = op(C, L, b, x, t, tr))) return rc;
    CK(launch_axpby(d, d, rho_new * rho, 0.0, L.N, C.stream));
    if ((rc = vanka_all(C, L, t, d, 2.0 * rho_new / delta, tr))) return rc;
    CK(launch_axpby(x, d, 1.0, 1.0, L.N, C.stream));
    C.launches += 2;
    rho = rho_new;
  }
  return IRKMG_OK;
}

// Ritz values of k Arnoldi steps on the relaxation-preconditioned operator
// D⁻¹J of level L (D⁻¹ = Σ_v R_vᵀ A_v⁻¹ R_v, the additive Vanka step), from
// x0 (device, length L.N) or, if null, x0_i = sin(i + 1); modified
// Gram–Schmidt applied twice.  The basis lives in the FGMRES storage
// (k <= restart).  lambda = the largest real part among the Ritz values
// (Section 5.1: the Chebyshev interval is chosen as [λ/4, λ] from such an
// estimate).  ritz_re / ritz_im (host, k each) may be null.
int estimate_lambda(Ctx& C, Level& L, int k, const double* x0, double* ritz_re, double* ritz_im,
                    double* lambda) {
  if (k < 2 || k > C.opt.restart) return fail(IRKMG_EINVAL, "Arnoldi steps in [2, restart]");
  const int64_t n = L.N;
  double* V = C.d_V;
  double* hd = C.d_h;
  double* hh = C.h_h;
  if (x0)
    CK(cudaMemcpyAsync(V, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.stream));
  else
    CK(launch_fill_sin(V, n, C.stream));
  auto dot_self = [&](const double* v, double* out) -> int {
    CK(launch_multidot(v, 0, 1, v, n, C.d_part, hd + 192, C.stream));
    CK(cudaMemcpyAsync(hh + 192, hd + 192, sizeof(double), cudaMemcpyDeviceToHost, C.stream));
    CK(cudaStreamSynchronize(C.stream));
    *out = std::sqrt(hh[192]);
    return IRKMG_OK;
  };
  int rc;
  double nrm;
  if ((rc = dot_self(V, &nrm))) return rc;
  if (!(nrm > 0.0)) return fail(IRKMG_EINVAL, "zero Arnoldi start vector");
  CK(launch_axpby(V, V, 1.0 / nrm, 0.0, n, C.stream));
  std::vector<double> H((size_t)k * k, 0.0);  // row-major k x k Hessenberg
  int kk = k;
  for (int j = 0; j < k; ++j) {
    double* vj = V + (int64_t)j * n;
    double* w = C.d_w;
    // w = D⁻¹ J v_j
    if ((rc = op(C, L, nullptr, vj, L.t, 0))) return rc;
    CK(launch_fill(w, 0.0, n, C.stream));
    if ((rc = vanka_all(C, L, L.t, w, 1.0, 0))) return rc;
    for (int pass = 0; pass < 2; ++pass) {
      CK(launch_multidot(V, n, j + 1, w, n, C.d_part, hd, C.stream));
      CK(launch_multiaxpy(w, V, n, j + 1, hd, -1.0, n, C.stream));
      CK(cudaMemcpyAsync(hh, hd, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, C.stream));
      CK(cudaStreamSynchronize(C.stream));
      for (int i = 0; i <= j; ++i) H[(size_t)i * k + j] += hh[i];
    }
    double hn;
    if ((rc = dot_self(w, &hn))) return rc;
    if (j + 1 == k) break;
    if (!(hn > 1e-14 * std::fabs(H[(size_t)j * k + j]) + 1e-300)) {  // invariant subspace
      kk = j + 1;
      break;
    }
    H[(size_t)(j + 1) * k + j] = hn;
    CK(launch_axpby(V + (int64_t)(j + 1) * n, w, 1.0 / hn, 0.0, n, C.stream));
  }
  std::vector<double> Hk((size_t)kk * kk), wr(kk), wi(kk);
  for (int i = 0; i < kk; ++i)
    for (int j = 0; j < kk; ++j) Hk[(size_t)i * kk + j] = H[(size_t)i * k + j];
  if ((rc = hessenberg_eigvals(kk, Hk.data(), wr.data(), wi.data())))
    return fail(rc, "Ritz values did not converge");
  double lam = -1e300;
  for (int i = 0; i < kk; ++i) lam = std::max(lam, wr[i]);
  for (int i = 0; i < k; ++i) {
    if (ritz_re) ritz_re[i] = i < kk ? wr[i] : 0.0;
    if (ritz_im) ritz_im[i] = i < kk ? wi[i] : 0.0;
  }
  *lambda = lam;
  return check_err(C, "Arnoldi on the Vanka-preconditioned operator");
}

// Per-level Chebyshev intervals: the fixed [cheb_lo, cheb_hi], or with
// cheb_auto [λ_l/4, λ_l] from 20 Arnoldi steps on level l.
int set_chebyshev_intervals(Ctx& C) {
  for (size_t l = 1; l < C.L.size(); ++l) {
    Level& L = C.L[l];
    L.cheb_lo = C.opt.cheb_lo;
    L.cheb_hi = C.opt.cheb_hi;
    if (!C.opt.cheb_auto) continue;
    double lam = 0.0;
    int rc = estimate_lambda(C, L, std::min(20, C.opt.restart), nullptr, nullptr, nullptr, &lam);
    if (rc) return rc;
    if (!(lam > 0.0)) return fail(IRKMG_ENOCONV, "no positive Ritz value for the Chebyshev interval");
    L.cheb_lo = 0.25 * lam;
    L.cheb_hi = lam;
  }
  C.launches = 0;
  return IRKMG_OK;
}

// --- Navier-Stokes: Newton on the stage equations (Section 3.2) ------------
// Once per context: the topology the GPU assembly of the Newton blocks needs
// on every level (vertex coordinates, P2 node -> cells, free -> P2 node), the
// SELL slot of every velocity CSR entry, and the block storage.
int ns_prepare(Ctx& C) {
  if (C.d_ns_U) return IRKMG_OK;
  int rc;
  for (Level& L : C.L) {
    const HostMesh& m = L.mesh;
    if (!L.d_cells && (rc = upload(C, &L.d_cells, m.cells))) return rc;
    if (!L.d_cell_edges && (rc = upload(C, &L.d_cell_edges, m.cell_edges))) return rc;
    if (!L.d_p2_to_free && (rc = upload(C, &L.d_p2_to_free, m.p2_to_free))) return rc;
    if ((rc = upload(C, &L.d_xy, m.xy))) return rc;
    if ((rc = upload(C, &L.d_free_to_p2, m.free_to_p2))) return rc;
    std::vector<int32_t> ptr(m.np2 + 1, 0), idx;
    for (int64_t c = 0; c < m.nc; ++c) {
      for (int i = 0; i < 3; ++i) ptr[m.cells[3 * c + i] + 1]++;
      for (int i = 0; i < 3; ++i) ptr[m.nv + m.cell_edges[3 * c + i] + 1]++;
    }
    for (int64_t n = 0; n < m.np2; ++n) ptr[n + 1] += ptr[n];
    idx.resize(ptr[m.np2]);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t c = 0; c < m.nc; ++c) {
      for (int i = 0; i < 3; ++i) idx[fill[m.cells[3 * c + i]]++] = (int32_t)c;
      for (int i = 0; i < 3; ++i) idx[fill[m.nv + m.cell_edges[3 * c + i]]++] = (int32_t)c;
    }
    if ((rc = upload(C, &L.d_nc_ptr, ptr))) return rc;
    if ((rc = upload(C, &L.d_nc_idx, idx))) return rc;
    const HostCSR& V = L.hops.vel;
    std::vector<int64_t> perm(V.col.size());
    HostSELL S = to_sell(V, 0);
    for (int64_t r = 0; r < V.nrows; ++r)
      for (int32_t p = V.ptr[r]; p < V.ptr[r + 1]; ++p)
        perm[p] = S.ptr[r / 32] + r % 32 + 32 * (int64_t)(p - V.ptr[r]);
    if ((rc = upload(C, &L.d_sell_perm, perm))) return rc;
    for (int t = 0; t < C.s; ++t)
      for (int k = 0; k < 4; ++k) {
        if ((rc = dalloc(C, &L.d_ns_csr[t][k], V.col.size()))) return rc;
        if ((rc = dalloc(C, &L.d_ns_sell[t][k], S.col.size()))) return rc;
        CK(cudaMemsetAsync(L.d_ns_sell[t][k], 0, sizeof(double) * S.col.size(), C.stream));
      }
  }
  Level& F = C.L.back();
  if ((rc = dalloc(C, &C.d_ns_g, (size_t)C.s * 2 * F.nf))) return rc;
  if ((rc = dalloc(C, &C.d_ns_U, (size_t)C.s * 2 * F.np2))) return rc;
  return IRKMG_OK;
}

// Newton blocks W_t,dc = δ_dc C(U_t) + R_dc(U_t) on every level from the stage
// velocities in C.d_ns_U (finest P2 nodes; a coarse level's P2 nodes are the
// first ones of the finer level, with the same ids, so its U is a prefix),
// g_t = C(U_t) U_t on the finest level, then the patches and the coarsest
// solve are refactored with them.  All on the GPU.
int ns_set_state(Ctx& C) {
  const int nl = (int)C.L.size();
  const int64_t np2f = C.L.back().np2;
  for (int l = 0; l < nl; ++l) {
    Level& L = C.L[l];
    for (int t = 0; t < C.s; ++t)
      CK(launch_ns_assemble(C, L, t, C.d_ns_U + (int64_t)t * 2 * np2f, np2f,
                            l == nl - 1 ? C.d_ns_g + (int64_t)t * 2 * L.nf : nullptr));
  }
  C.ns = true;
  drop_graphs(C);
  int rc;
  if ((rc = factor_all(C))) return rc;
  return set_chebyshev_intervals(C);
}

// Newton residual of the stage equations at k (finest level):
// F = J_S k - R_S + g with J_S the Stokes stage operator, R_S the stage
// right-hand side with u^n at every node and g = C(U_t) U_t from the state
// last set (which must be that of k).
int ns_residual(Ctx& C, const double* un_all, const double* pn, const double* f, const double* k,
                double* F) {
  Level& L = C.L.back();
  double* tmp = C.d_w;
  CK(launch_stage_rhs_full(C, un_all, pn, f, tmp));
  C.ns_active = false;
  cudaError_t e = launch_residual(C, L, tmp, k, F, 0);  // F = R_S - J_S k
  C.ns_active = true;
  CK(e);
  CK(launch_axpby(F, F, -1.0, 0.0, L.N, C.stream));
  for (int t = 0; t < C.s; ++t)
    CK(launch_axpby(F + (int64_t)t * L.m, C.d_ns_g + (int64_t)t * 2 * L.nf, 1.0, 1.0, 2 * L.nf,
                    C.stream));
  C.launches += 3 + C.s;
  return IRKMG_OK;
}

// Eisenstat–Walker forcing term, choice 2 (gamma 0.9, alpha 2) with its
// safeguard and the cap 0.9.
double ew_eta(double eta_prev, double fn, double fprev) {
  double eta = 0.9 * (fn / fprev) * (fn / fprev);
  const double safe = 0.9 * eta_prev * eta_prev;
  if (safe > 0.1) eta = std::max(eta, safe);
  return std::min(eta, 0.9);
}

int ns_newton(Ctx& C, const double* un_all, const double* pn, const double* f, double* k,
              double atol, int maxit, irkmg_ns_stats* st) {
  const double t0 = now();
  const int64_t N = C.L.back().N;
  int rc;
  if ((rc = ns_prepare(C))) return rc;
  double* Fb = C.d_F;
  double* db = C.d_kb;
  double eta = 0.5, fprev = 0.0, fn = 0.0;
  int its = 0, lin = 0;
  for (;; ++its) {
    CK(launch_ns_stage_velocity(C, un_all, k, C.d_ns_U));
    if ((rc = ns_set_state(C))) return rc;
    if ((rc = ns_residual(C, un_all, pn, f, k, Fb))) return rc;
    CK(launch_multidot(Fb, 0, 1, Fb, N, C.d_part, C.d_h + 192, C.stream));
    CK(cudaMemcpyAsync(C.h_h + 192, C.d_h + 192, sizeof(double), cudaMemcpyDeviceToHost, C.stream));
    CK(cudaStreamSynchronize(C.stream));
    fn = std::sqrt(C.h_h[192]);
    if (st && its == 0) st->f0 = fn;
    if (fn <= atol || its >= maxit) break;
    if (its > 0) eta = ew_eta(eta, fn, fprev);
    fprev = fn;
    // J δ = -F to the relative tolerance eta
    CK(launch_axpby(Fb, Fb, -1.0, 0.0, N, C.stream));
    CK(cudaMemsetAsync(db, 0, sizeof(double) * N, C.stream));
    const double rtol = C.opt.rtol;
    C.opt.rtol = eta;
    irkmg_stats ls{};
    rc = fgmres(C, Fb, db, &ls, 0);
    C.opt.rtol = rtol;
    lin += ls.iters;
    if (rc && rc != IRKMG_ENOCONV) return rc;
    CK(launch_axpby(k, db, 1.0, 1.0, N, C.stream));
  }
  const int status = fn <= atol ? IRKMG_OK : IRKMG_ENOCONV;
  if (st) {
    st->newton_iters = its;
    st->linear_iters = lin;
    st->ffinal = fn;
    st->status = status;
    st->t_solve = now() - t0;
  }
  if (status) return fail(status, "Newton reached maxit on the Navier-Stokes stage equations");
  return IRKMG_OK;
}

// Levels 0 .. nl-2 of the V-cycle as one CUDA graph (from L[nl-2].r to
// L[nl-2].z), captured on the library's own non-blocking stream the first time
// it is needed: the hundreds of short colour launches of the coarse levels
// then cost one graph launch.  Kernel parameters (dt·A among them) are baked
// in, so irkmg_update drops the graphs.
int coarse_graph(Ctx& C, int tr) {
  if (C.cgraph[tr]) return IRKMG_OK;
  if (!C.gstream) {
    CK(cudaStreamCreateWithFlags(&C.gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&C.gev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&C.gev[1], cudaEventDisableTiming));
  }
  const int lc = (int)C.L.size() - 2;
  cudaStream_t saved_stream = C.stream;
  const bool saved_trace = C.trace_on;
  const int64_t l0 = C.launches;
  C.stream = C.gstream;
  C.trace_on = false;
  C.capturing = true;
  cudaGraph_t g = nullptr;
  int rc = IRKMG_OK;
  cudaError_t e = cudaStreamBeginCapture(C.gstream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = vcycle_level(C, lc, C.L[lc].r, C.L[lc].z, tr);
    e = cudaStreamEndCapture(C.gstream, &g);
  }
  C.stream = saved_stream;
  C.trace_on = saved_trace;
  C.capturing = false;
  C.cgraph_launches[tr] = C.launches - l0;
  C.launches = l0;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(e);
  e = cudaGraphInstantiate(&C.cgraph[tr], g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return IRKMG_OK;
}

void drop_graphs(Ctx& C) {
  if (C.vgraph) cudaGraphExecDestroy(C.vgraph);
  C.vgraph = nullptr;
  for (int t = 0; t < 2; ++t) {
    if (C.cgraph[t]) cudaGraphExecDestroy(C.cgraph[t]);
    C.cgraph[t] = nullptr;
  }
}

// --- batched solves ----------------------------------------------------------
// One V-cycle of C captured as a CUDA graph that reads d_gin and writes
// d_gout; captured once, on the context's (non-default) stream.
int capture_vcycle(Ctx& C) {
  if (C.vgraph) return IRKMG_OK;
  const int64_t n = C.L.back().N;
  int rc;
  if (!C.d_gin && (rc = dalloc(C, &C.d_gin, n))) return rc;
  if (!C.d_gout && (rc = dalloc(C, &C.d_gout, n))) return rc;
  const bool saved = C.trace_on;
  C.trace_on = false;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(C.stream, cudaStreamCaptureModeThreadLocal));
  C.capturing = true;
  rc = vcycle_level(C, (int)C.L.size() - 1, C.d_gin, C.d_gout, 0);
  C.capturing = false;
  cudaError_t e = cudaStreamEndCapture(C.stream, &g);
  C.trace_on = saved;
  if (rc) {
    if (e == cudaSuccess && g) cudaGraphDestroy(g);
    return rc;
  }
  CK(e);
  e = cudaGraphInstantiate(&C.vgraph, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return IRKMG_OK;
}

// Per-system state of the lock-step FGMRES (the same recurrences as fgmres()).
struct FState {
  Ctx* C = nullptr;
  const double* F = nullptr;
  double* x = nullptr;
  irkmg_stats* st = nullptr;
  int m = 0, j = 0, its = 0;
  double bnorm = 0, beta = 0, target = 0, t0 = 0;
  bool done = false, finishing = false;
  std::vector<double> H, cs, sn, g, y;
};

int issue_norm(Ctx& C, const double* v, int slot) {
  const int64_t n = C.L.back().N;
  CK(launch_multidot(v, 0, 1, v, n, C.d_part, C.d_h + slot, C.stream));
  CK(cudaMemcpyAsync(C.h_h + slot, C.d_h + slot, sizeof(double), cudaMemcpyDeviceToHost, C.stream));
  C.launches += 2;
  return IRKMG_OK;
}

// What a batch owns besides its contexts: one stream per system; with a
// persistent plan, the batch stream and events ordering the persistent
// launches against the systems' streams, and the relaxation mode each finest
// level had before the batch pinned it to one launch.
struct BatchLink {
  BatchPlan* plan = nullptr;
  bool on = false;  // relax through the plan (else per-system V-cycle graphs)
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> ready;
};

// One V-cycle per active system (b_i -> z_i) with the finest-level smoothing
// of all of them in two persistent launches (before and after the coarse
// corrections, which run on the systems' own streams).
int batch_vcycles(BatchLink& K, std::vector<FState>& S, const std::vector<int>& act,
                  const std::vector<const double*>& b, const std::vector<double*>& z) {
  auto join = [&]() -> int {  // every active system's stream -> the batch stream
    for (int i : act) {
      CK(cudaEventRecord(K.ready[i], S[i].C->stream));
      CK(cudaStreamWaitEvent(K.stream, K.ready[i], 0));
    }
    return IRKMG_OK;
  };
  auto fork = [&]() -> int {  // the batch stream -> every active system's stream
    CK(cudaEventRecord(K.done, K.stream));
    for (int i : act) CK(cudaStreamWaitEvent(S[i].C->stream, K.done, 0));
    return IRKMG_OK;
  };
  Ctx& C0 = *S[act[0]].C;
  int rc;
  if ((rc = join())) return rc;
  CK(batch_plan_smooth(K.plan, act, b, z, C0.opt.nu_pre, true, C0.opt.timeout_spins, C0.d_err,
                       K.stream));
  C0.launches++;
  if ((rc = fork())) return rc;
  for (size_t k = 0; k < act.size(); ++k) {
    Ctx& C = *S[act[k]].C;
    if ((rc = coarse_correction(C, (int)C.L.size() - 1, b[k], z[k], 0))) return rc;
  }
  if ((rc = join())) return rc;
  CK(batch_plan_smooth(K.plan, act, b, z, C0.opt.nu_post, false, C0.opt.timeout_spins, C0.d_err,
                       K.stream));
  C0.launches++;
  return fork();
}

int batch_fgmres(std::vector<FState>& S, BatchLink* K) {
  int rc;
  if (K && K->plan && (rc = batch_plan_refresh(K->plan, K->stream))) return fail(rc, "batch plan");
  for (FState& f : S) {  // initial residuals and norms
    Ctx& C = *f.C;
    const int64_t n = C.L.back().N;
    f.m = C.opt.restart;
    f.H.assign((size_t)(f.m + 1) * f.m, 0.0);
    f.cs.assign(f.m, 0.0);
    f.sn.assign(f.m, 0.0);
    f.g.assign(f.m + 1, 0.0);
    f.y.assign(f.m, 0.0);
    f.t0 = now();
    if (!(K && K->plan) && (rc = capture_vcycle(C))) return rc;
    if ((rc = issue_norm(C, f.F, 192))) return rc;
    if ((rc = op(C, C.L.back(), f.F, f.x, C.d_V, 0))) return rc;
    if ((rc = issue_norm(C, C.d_V, 193))) return rc;
    (void)n;
  }
  for (FState& f : S) {
    CK(cudaStreamSynchronize(f.C->stream));
    f.bnorm = std::sqrt(f.C->h_h[192]);
    f.beta = std::sqrt(f.C->h_h[193]);
    f.target = std::max(f.C->opt.rtol * f.bnorm, f.C->opt.atol);
    if (f.st) f.st->r0 = f.beta;
    f.done = !(f.beta > f.target && f.its < f.C->opt.maxit);
    f.finishing = false;
    f.j = -1;  // a new cycle starts
  }
  std::vector<int> act;
  std::vector<const double*> vb;
  std::vector<double*> vz;
  for (;;) {
    bool any = false;
    act.clear();
    vb.clear();
    vz.clear();
    for (size_t i = 0; i < S.size(); ++i) {  // new cycles start; the V-cycles' inputs
      FState& f = S[i];
      if (f.done) continue;
      Ctx& C = *f.C;
      const int64_t n = C.L.back().N;
      if (f.j < 0) {
        CK(launch_axpby(C.d_V, C.d_V, 1.0 / f.beta, 0.0, n, C.stream));
        C.launches++;
        std::fill(f.g.begin(), f.g.end(), 0.0);
        f.g[0] = f.beta;
        f.j = 0;
      }
      act.push_back((int)i);
      vb.push_back(C.d_V + (int64_t)f.j * n);
      vz.push_back(C.d_Z + (int64_t)f.j * n);
    }
    if (K && K->plan && !act.empty() && (rc = batch_vcycles(*K, S, act, vb, vz))) return rc;
    for (FState& f : S) {  // issue the rest of one Arnoldi step per active system
      if (f.done) continue;
      any = true;
      Ctx& C = *f.C;
      Level& L = C.L.back();
      const int64_t n = L.N;
      double* vj = C.d_V + (int64_t)f.j * n;
      double* zj = C.d_Z + (int64_t)f.j * n;
      if (!(K && K->plan)) {  // the whole V-cycle as one graph on the system's stream
        CK(cudaMemcpyAsync(C.d_gin, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.stream));
        CK(cudaGraphLaunch(C.vgraph, C.stream));
        CK(cudaMemcpyAsync(zj, C.d_gout, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.stream));
      }
      CK(launch_pressure_mean_remove(C, L, zj));
      if ((rc = op(C, L, nullptr, zj, C.d_w, 0))) return rc;
      CK(launch_multidot(C.d_V, n, f.j + 1, C.d_w, n, C.d_part, C.d_h, C.stream));
      CK(launch_multiaxpy_dot(C.d_w, C.d_V, n, f.j + 1, C.d_h, -1.0, n, C.d_part, C.d_h + 64,
                              false, C.stream));
      CK(launch_multiaxpy_dot(C.d_w, C.d_V, n, f.j + 1, C.d_h + 64, -1.0, n, C.d_part,
                              C.d_h + 128, true, C.stream));
      C.launches += f.j + 1 <= 16 ? 7 : 11;
      CK(cudaMemcpyAsync(C.h_h, C.d_h, sizeof(double) * 129, cudaMemcpyDeviceToHost, C.stream));
      CK(cudaMemcpyAsync(C.h_err, C.d_err, sizeof(int) * 2, cudaMemcpyDeviceToHost, C.stream));
    }
    if (!any) break;
    for (FState& f : S) {  // Givens updates, cycle ends
      if (f.done) continue;
      Ctx& C = *f.C;
      const int64_t n = C.L.back().N;
      CK(cudaStreamSynchronize(C.stream));
      if (C.h_err[0] != 0) {
        const int code = C.h_err[0];
        CK(cudaMemsetAsync(C.d_err, 0, sizeof(int) * 2, C.stream));
        if (f.st) f.st->status = code;
        return fail(code, "a bounded device-side wait expired during a batched V-cycle");
      }
      const int j = f.j, m = f.m;
      double* Hj = &f.H[(size_t)j * (m + 1)];
      for (int i = 0; i <= j; ++i) Hj[i] = C.h_h[i] + C.h_h[64 + i];
      const double hn = std::sqrt(C.h_h[128]);
      Hj[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = f.cs[i] * Hj[i] + f.sn[i] * Hj[i + 1];
        Hj[i + 1] = -f.sn[i] * Hj[i] + f.cs[i] * Hj[i + 1];
        Hj[i] = a;
      }
      const double den = std::hypot(Hj[j], Hj[j + 1]);
      f.cs[j] = Hj[j] / den;
      f.sn[j] = Hj[j + 1] / den;
      Hj[j] = den;
      Hj[j + 1] = 0.0;
      f.g[j + 1] = -f.sn[j] * f.g[j];
      f.g[j] = f.cs[j] * f.g[j];
      ++f.its;
      const bool end = std::fabs(f.g[j + 1]) <= f.target || f.its >= C.opt.maxit || hn == 0.0 ||
                       j + 1 == m;
      if (!end) {
        CK(launch_axpby(C.d_V + (int64_t)(j + 1) * n, C.d_w, 1.0 / hn, 0.0, n, C.stream));
        C.launches++;
        f.j = j + 1;
        continue;
      }
      const int jdone = j + 1;
      for (int i = jdone - 1; i >= 0; --i) {
        double sum = f.g[i];
        for (int k = i + 1; k < jdone; ++k) sum -= f.H[(size_t)k * (m + 1) + i] * f.y[k];
        f.y[i] = sum / f.H[(size_t)i * (m + 1) + i];
      }
      std::copy(f.y.begin(), f.y.begin() + jdone, C.h_h + 256);
      CK(cudaMemcpyAsync(C.d_h + 256, C.h_h + 256, sizeof(double) * jdone, cudaMemcpyHostToDevice,
                         C.stream));
      CK(launch_multiaxpy(f.x, C.d_Z, n, jdone, C.d_h + 256, 1.0, n, C.stream));
      C.launches++;
      if ((rc = op(C, C.L.back(), f.F, f.x, C.d_V, 0))) return rc;
      if ((rc = issue_norm(C, C.d_V, 193))) return rc;
      f.finishing = true;
    }
    for (FState& f : S) {  // restarts: true residual decides
      if (f.done || !f.finishing) continue;
      CK(cudaStreamSynchronize(f.C->stream));
      f.beta = std::sqrt(f.C->h_h[193]);
      f.finishing = false;
      f.j = -1;
      if (!(f.beta > f.target && f.its < f.C->opt.maxit)) f.done = true;
    }
  }
  int worst = IRKMG_OK;
  for (FState& f : S) {
    const int status = f.beta <= f.target ? IRKMG_OK : IRKMG_ENOCONV;
    if (f.st) {
      f.st->iters = f.its;
      f.st->rfinal = f.beta;
      f.st->t_solve = now() - f.t0;
      f.st->status = status;
      f.st->bad_index = -1;
    }
    if (status != IRKMG_OK) worst = status;
  }
  if (worst) return fail(worst, "FGMRES reached maxit in at least one system of the batch");
  return IRKMG_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void irkmg_default_options(irkmg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->nlevels = 3;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->smoother = 1;
  o->omega = 0.5;
  o->cheb_lo = 2.0;
  o->cheb_hi = 8.0;
  o->rtol = 1e-10;
  o->atol = 1e-30;
  o->restart = 30;
  o->maxit = 200;
  o->patch_precision = 64;
  o->wind = nullptr;
  o->cuda_stream = nullptr;
  o->timeout_spins = 0;
  o->apply_variant = 0;
  o->patch_form = 0;
  o->patch_lu_tc = 1;
}

int irkmg_radau_iia(int s, double* A, double* b, double* c) {
  if (!A || !b || !c) return fail(IRKMG_EINVAL, "null output");
  int rc = radau_iia(s, A, b, c);
  if (rc) return fail(rc, "Radau IIA closed forms exist here for s = 1, 2, 3");
  return IRKMG_OK;
}

int irkmg_gauss(int s, double* A, double* b, double* c) {
  if (!A || !b || !c) return fail(IRKMG_EINVAL, "null output");
  int rc = gauss_tableau(s, A, b, c);
  if (rc) return fail(rc, "Gauss closed forms exist here for s = 2, 3");
  return IRKMG_OK;
}

int irkmg_lobatto_iiic(int s, double* A, double* b, double* c) {
  if (!A || !b || !c) return fail(IRKMG_EINVAL, "null output");
  int rc = lobatto_iiic_tableau(s, A, b, c);
  if (rc) return fail(rc, "LobattoIIIC closed forms exist here for s = 2, 3");
  return IRKMG_OK;
}

int irkmg_kron_split(int s, const double* A, double* T, double* Tinv, double* D) {
  if (!A || !T || !Tinv || !D) return fail(IRKMG_EINVAL, "null argument");
  if (s < 1 || s > 3) return fail(IRKMG_EINVAL, "s in [1, 3]");
  KronSplit K;
  if (kron_split(s, A, &K) != IRKMG_OK)
    return fail(IRKMG_ENOTIMPL, "no real block diagonalisation with distinct eigenvalues");
  for (int i = 0; i < s * s; ++i) {
    T[i] = K.T[i];
    Tinv[i] = K.Tinv[i];
    D[i] = 0.0;
  }
  for (int b = 0; b < K.nblk; ++b) {
    const int c0 = K.col0[b], q = K.blk_size[b];
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) D[(c0 + i) * s + c0 + j] = K.blk[b][i * q + j];
  }
  return IRKMG_OK;
}

int irkmg_hessenberg_eigvals(int n, const double* H, double* wr, double* wi) {
  if (!H || !wr || !wi || n < 1 || n > 512) return fail(IRKMG_EINVAL, "bad arguments");
  const int rc = hessenberg_eigvals(n, H, wr, wi);
  if (rc) return fail(rc, "QR iteration did not converge");
  return IRKMG_OK;
}

int irkmg_estimate_lambda(irkmg_ctx* C, int level, int nsteps, const double* d_x0, double* ritz_re,
                          double* ritz_im, double* lambda) {
  if (!level_ok(C, level) || level == 0 || !lambda) return fail(IRKMG_EINVAL, "bad level");
  return estimate_lambda(*C, C->L[level], nsteps, d_x0, ritz_re, ritz_im, lambda);
}

int irkmg_setup(const irkmg_mesh* mesh, const irkmg_tableau* tab, double dt, double nu,
                const irkmg_options* opt, irkmg_ctx** out) {
  if (!out) return fail(IRKMG_EINVAL, "null out");
  *out = nullptr;
  int rc = validate(mesh, tab, dt, nu, opt);
  if (rc) return rc;
  irkmg_ctx* C = new (std::nothrow) irkmg_ctx();
  if (!C) return fail(IRKMG_ENOMEM, "context");
  rc = setup_impl(C, mesh, tab, dt, nu, opt);
  if (rc) {
    std::string msg = g_last_error;
    irkmg_destroy(C);
    g_last_error = msg;
    return rc;
  }
  *out = C;
  return IRKMG_OK;
}

int irkmg_update(irkmg_ctx* C, double dt, double nu) {
  if (!C || !(dt > 0.0) || !(nu > 0.0)) return fail(IRKMG_EINVAL, "bad update");
  CK(C->stream ? cudaStreamSynchronize(C->stream) : cudaDeviceSynchronize());
  C->dt = dt;
  C->nu = nu;
  drop_graphs(*C);
  int rc;
  if ((rc = assemble_all(*C))) return rc;
  for (size_t l = 0; l < C->L.size(); ++l) {
    Level& L = C->L[l];
    if ((rc = refresh_csr_values(*C, L.vel, L.hops.vel, 3))) return rc;
    if ((rc = refresh_csr_values(*C, L.b, L.hops.b, L.dim))) return rc;
    if ((rc = refresh_csr_values(*C, L.bt, L.hops.bt, L.dim))) return rc;
    if ((rc = refresh_sell_values(*C, L.svel, L.hops.vel, 3))) return rc;
    if ((rc = refresh_sell_values(*C, L.sb, L.hops.b, L.dim))) return rc;
    if ((rc = refresh_sell_values(*C, L.sbt, L.hops.bt, L.dim))) return rc;
    if (L.fxop_on) CK(launch_op_fixed_convert(*C, L));
    if (l + 1 == C->L.size() && (rc = refresh_csr_values(*C, L.mall, L.hops.mall, 2))) return rc;
    if (l + 1 == C->L.size() && (rc = refresh_csr_values(*C, L.btall, L.hops.btall, L.dim)))
      return rc;
  }
  if ((rc = factor_all(*C))) return rc;
  return set_chebyshev_intervals(*C);
}

int irkmg_set_wind(irkmg_ctx* C, const double* wind) {
  if (!C) return fail(IRKMG_EINVAL, "null ctx");
  if (C->dim != 2 && wind) return fail(IRKMG_ENOTIMPL, "the Oseen wind is built for 2D meshes only");
  CK(C->stream ? cudaStreamSynchronize(C->stream) : cudaDeviceSynchronize());
  if (wind)
    C->wind.assign(wind, wind + 2 * C->L.back().np2);
  else
    C->wind.clear();
  return irkmg_update(C, C->dt, C->nu);
}

int irkmg_level_info_get(const irkmg_ctx* C, int level, irkmg_level_info* info) {
  if (!level_ok(C, level) || !info) return fail(IRKMG_EINVAL, "bad level");
  const Level& L = C->L[level];
  info->nv = L.nv;
  info->ne = L.mesh.ne;
  info->nc = L.mesh.nc;
  info->np2 = L.np2;
  info->nf = L.nf;
  info->m = L.m;
  info->N = L.N;
  info->npatch = level > 0 ? L.nv : 0;
  info->ncolours = L.ncolours;
  info->max_patch_dofs = L.max_np;
  info->factor_bytes = L.fac_elems * (C->opt.patch_precision == 64 ? 8 : 4);
  info->apply_kernel = level > 0 ? L.apply_kernel : 0;
  info->dim = L.dim;
  info->apply_ms[0] = L.apply_ms[1];
  info->apply_ms[1] = L.apply_ms[2];
  info->single_launch = level > 0 && L.kron && L.single ? 1 : 0;
  info->cheb[0] = level > 0 ? L.cheb_lo : 0.0;
  info->cheb[1] = level > 0 ? L.cheb_hi : 0.0;
  info->apply_shape =
      level > 0 && (L.apply_kernel == 5 || L.apply_kernel >= 8) ? L.kron_shape : 0;
  return IRKMG_OK;
}

int irkmg_level_set_apply(irkmg_ctx* C, int level, int shape, int single_launch) {
  if (!level_ok(C, level) || level < 1) return fail(IRKMG_EINVAL, "bad level (relaxed levels are 1 ..)");
  Level& L = C->L[level];
  if (single_launch != 0 && single_launch != 1) return fail(IRKMG_EINVAL, "single_launch is 0 or 1");
  if (single_launch && !L.kron) return fail(IRKMG_EINVAL, "one-launch relaxation needs decoupled patches");
  const int nshape = L.fixed ? fixed_shapes() : L.apply_kernel == 5 ? 2 : 1;
  if (shape < 0 || shape >= nshape) return fail(IRKMG_EINVAL, "no such launch shape for the level's kernel");
  if ((L.apply_kernel == 5 && !kron_staged_fits(*C, L, shape)) || (L.fixed && !fixed_shape_fits(*C, L, shape)))
    return fail(IRKMG_EINVAL, "launch shape does not fit in shared memory");
  L.kron_shape = shape;
  if (L.fixed) L.apply_kernel = fixed_shape_kernel(shape);
  L.single = single_launch != 0;
  drop_graphs(*C);  // captured coarse levels hold the previous launches
  return IRKMG_OK;
}

int irkmg_set_timeout(irkmg_ctx* C, int64_t timeout_spins) {
  if (!C) return fail(IRKMG_EINVAL, "null ctx");
  if (timeout_spins < 0) return fail(IRKMG_EINVAL, "timeout_spins >= 0");
  C->opt.timeout_spins = timeout_spins;
  drop_graphs(*C);  // captured coarse levels hold the previous bound
  return IRKMG_OK;
}

int irkmg_p2_coords(const irkmg_ctx* C, int level, double* xy) {
  if (!level_ok(C, level) || !xy) return fail(IRKMG_EINVAL, "bad level");
  const HostMesh& m = C->L[level].mesh;
  const int d = m.dim;
  std::copy(m.xy.begin(), m.xy.end(), xy);
  for (int64_t e = 0; e < m.ne; ++e) {
    const int32_t a = m.edges[2 * e], b = m.edges[2 * e + 1];
    for (int k = 0; k < d; ++k) xy[d * (m.nv + e) + k] = 0.5 * (m.xy[d * a + k] + m.xy[d * b + k]);
  }
  return IRKMG_OK;
}

int irkmg_free_nodes(const irkmg_ctx* C, int level, int64_t* ids) {
  if (!level_ok(C, level) || !ids) return fail(IRKMG_EINVAL, "bad level");
  const HostMesh& m = C->L[level].mesh;
  for (int64_t i = 0; i < m.nf; ++i) ids[i] = m.free_to_p2[i];
  return IRKMG_OK;
}

int irkmg_patch_map(const irkmg_ctx* C, int level, int64_t* ptr, int32_t* nodes) {
  if (!level_ok(C, level) || level == 0 || !ptr || !nodes)
    return fail(IRKMG_EINVAL, "bad level (patches exist on levels >= 1)");
  const Level& L = C->L[level];
  for (int64_t v = 0; v <= L.nv; ++v) ptr[v] = L.h_patch_ptr[v];
  std::copy(L.h_patch_nodes.begin(), L.h_patch_nodes.end(), nodes);
  return IRKMG_OK;
}

int irkmg_colouring(const irkmg_ctx* C, int level, int32_t* colour) {
  if (!level_ok(C, level) || level == 0 || !colour)
    return fail(IRKMG_EINVAL, "bad level (patches exist on levels >= 1)");
  const Level& L = C->L[level];
  std::copy(L.h_colour.begin(), L.h_colour.end(), colour);
  return IRKMG_OK;
}

int irkmg_apply(irkmg_ctx* C, int level, const double* x, double* y, int transpose) {
  if (!level_ok(C, level) || !x || !y) return fail(IRKMG_EINVAL, "bad arguments");
  return op(*C, C->L[level], nullptr, x, y, transpose ? 1 : 0);
}

int irkmg_vanka_correction(irkmg_ctx* C, int level, const double* r, double* c, int transpose) {
  if (!level_ok(C, level) || level == 0 || !r || !c) return fail(IRKMG_EINVAL, "bad arguments");
  Level& L = C->L[level];
  CK(launch_fill(c, 0.0, L.N, C->stream));
  C->launches++;
  return vanka_all(*C, L, r, c, 1.0, transpose ? 1 : 0);
}

int irkmg_smooth(irkmg_ctx* C, int level, const double* F, double* x, int nsteps, int transpose) {
  if (!level_ok(C, level) || level == 0 || !F || !x || nsteps < 0)
    return fail(IRKMG_EINVAL, "bad arguments");
  return smooth(*C, C->L[level], F, x, nsteps, false, transpose ? 1 : 0);
}

int irkmg_smooth_noalloc(irkmg_ctx* C, int level, const double* F, double* x, int nsteps,
                         int transpose) {
  if (!level_ok(C, level) || level == 0 || !F || !x || nsteps < 0)
    return fail(IRKMG_EINVAL, "bad arguments");
  Level& L = C->L[level];
  if (L.N > kNoallocMaxN)
    return fail(IRKMG_EINVAL, "level has " + std::to_string(L.N) +
                                  " unknowns; the static work array holds at most " +
                                  std::to_string(kNoallocMaxN));
  double* scratch = nullptr;
  int rc = noalloc_scratch(C->stream, &scratch);
  if (rc) return rc;
  return smooth_in(*C, L, F, x, nsteps, transpose ? 1 : 0, scratch, scratch + kNoallocMaxN);
}

int irkmg_restrict(irkmg_ctx* C, int level, const double* fine, double* coarse) {
  if (!level_ok(C, level) || level == 0 || !fine || !coarse)
    return fail(IRKMG_EINVAL, "bad arguments");
  CK(launch_restrict(*C, C->L[level], fine, coarse));
  return IRKMG_OK;
}

int irkmg_prolong(irkmg_ctx* C, int level, const double* coarse, double* fine) {
  if (!level_ok(C, level) || level == 0 || !fine || !coarse)
    return fail(IRKMG_EINVAL, "bad arguments");
  CK(launch_prolong(*C, C->L[level], coarse, fine, 0));
  return IRKMG_OK;
}

int irkmg_coarse_solve(irkmg_ctx* C, const double* r, double* x, int transpose) {
  if (!C || !r || !x) return fail(IRKMG_EINVAL, "bad arguments");
  CK(launch_coarse_apply(*C, r, x, transpose ? 1 : 0));
  return IRKMG_OK;
}

int irkmg_vcycle(irkmg_ctx* C, const double* r, double* z, int transpose) {
  if (!C || !r || !z) return fail(IRKMG_EINVAL, "bad arguments");
  return vcycle_level(*C, (int)C->L.size() - 1, r, z, transpose ? 1 : 0);
}

int irkmg_solve(irkmg_ctx* C, const double* F, double* k, irkmg_stats* st) {
  if (!C || !F || !k) return fail(IRKMG_EINVAL, "bad arguments");
  return fgmres(*C, F, k, st, 0);
}

int ns_check(irkmg_ctx* C) {
  if (!C) return fail(IRKMG_EINVAL, "null ctx");
  if (C->dim != 2) return fail(IRKMG_ENOTIMPL, "Navier-Stokes stages are built for 2D");
  if (C->kron) return fail(IRKMG_ENOTIMPL, "Newton blocks depend on the stage: dense patches only");
  if (!C->wind.empty()) return fail(IRKMG_EINVAL, "a frozen Oseen wind and Newton blocks exclude each other");
  return IRKMG_OK;
}

int irkmg_ns_set_state(irkmg_ctx* C, const double* U) {
  int rc = ns_check(C);
  if (rc) return rc;
  if (!U) return fail(IRKMG_EINVAL, "null state");
  if ((rc = ns_prepare(*C))) return rc;
  const Level& F = C->L.back();
  CK(cudaMemcpyAsync(C->d_ns_U, U, sizeof(double) * C->s * 2 * F.np2, cudaMemcpyHostToDevice,
                     C->stream));
  return ns_set_state(*C);
}

int irkmg_ns_residual(irkmg_ctx* C, const double* un_all, const double* pn, const double* f,
                      const double* k, double* F) {
  int rc = ns_check(C);
  if (rc) return rc;
  if (!C->ns) return fail(IRKMG_EINVAL, "irkmg_ns_set_state first");
  if (!un_all || !pn || !f || !k || !F) return fail(IRKMG_EINVAL, "bad arguments");
  return ns_residual(*C, un_all, pn, f, k, F);
}

int irkmg_ns_newton(irkmg_ctx* C, const double* un_all, const double* pn, const double* f,
                    double* k, double atol, int maxit, irkmg_ns_stats* st) {
  int rc = ns_check(C);
  if (rc) return rc;
  if (!un_all || !pn || !f || !k || !(atol > 0.0) || maxit < 1)
    return fail(IRKMG_EINVAL, "bad arguments");
  return ns_newton(*C, un_all, pn, f, k, atol, maxit, st);
}

int irkmg_adjoint_solve(irkmg_ctx* C, const double* G, double* lam, irkmg_stats* st) {
  if (!C || !G || !lam) return fail(IRKMG_EINVAL, "bad arguments");
  return fgmres(*C, G, lam, st, 1);
}

int irkmg_stage_rhs(irkmg_ctx* C, const double* un, const double* pn, const double* f,
                    double* F) {
  if (!C || !un || !pn || !f || !F) return fail(IRKMG_EINVAL, "bad arguments");
  CK(launch_stage_rhs(*C, un, pn, f, F));
  C->launches++;
  return IRKMG_OK;
}

int irkmg_advance(irkmg_ctx* C, const double* k, double* un, double* pn) {
  if (!C || !k || !un || !pn) return fail(IRKMG_EINVAL, "bad arguments");
  CK(launch_advance(*C, k, un, pn));
  C->launches++;
  return IRKMG_OK;
}

int irkmg_forcing_load(irkmg_ctx* C, const double* theta, double* g) {
  if (!C || !theta || !g) return fail(IRKMG_EINVAL, "bad arguments");
  if (C->dim != 2) return fail(IRKMG_ENOTIMPL, "the adjoint form is built for 2D meshes");
  CK(launch_cell_load(*C, theta, g));
  C->launches++;
  return IRKMG_OK;
}

int irkmg_step(irkmg_ctx* C, double* un, double* pn, const double* f, const double* g, double* k,
               irkmg_stats* st) {
  if (!C || !un || !pn || !f || !k) return fail(IRKMG_EINVAL, "bad arguments");
  Level& L = C->L.back();
  CK(launch_stage_rhs(*C, un, pn, f, C->d_F));
  C->launches++;
  if (g) {
    CK(launch_add_to_stages(*C, g, C->d_F));
    C->launches++;
  }
  CK(cudaMemsetAsync(k, 0, sizeof(double) * L.N, C->stream));
  int rc = fgmres(*C, C->d_F, k, st, 0);
  if (rc) return rc;
  CK(launch_advance(*C, k, un, pn));
  C->launches++;
  return IRKMG_OK;
}

int irkmg_adjoint_step(irkmg_ctx* C, double* ub, double* pb, const double* k, const double* un,
                       double* thb, double* dnu, irkmg_stats* st) {
  if (!C || !ub || !pb || !k || !un) return fail(IRKMG_EINVAL, "bad arguments");
  if (C->dim != 2) return fail(IRKMG_ENOTIMPL, "the adjoint form is built for 2D meshes");
  Level& L = C->L.back();
  CK(launch_kbar(*C, ub, pb, C->d_kb));
  CK(cudaMemsetAsync(C->d_lam, 0, sizeof(double) * L.N, C->stream));
  C->launches++;
  int rc = fgmres(*C, C->d_kb, C->d_lam, st, 1);
  if (rc) return rc;
  if (dnu) {
    CK(launch_dnu(*C, C->d_lam, k, un, C->d_part, C->d_scalar));
    C->launches += 2;
  }
  CK(launch_adjoint_update(*C, C->d_lam, ub, pb));
  C->launches++;
  if (thb) {
    CK(launch_theta_bar(*C, C->d_lam, thb));
    C->launches++;
  }
  if (dnu) {
    double h = 0.0;
    CK(cudaMemcpyAsync(&h, C->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    *dnu += h;
  }
  return IRKMG_OK;
}

int irkmg_tracking(irkmg_ctx* C, const double* u, const double* ut, double* grad, double* value) {
  if (!C || !u || !ut || !value) return fail(IRKMG_EINVAL, "bad arguments");
  if (C->dim != 2) return fail(IRKMG_ENOTIMPL, "the adjoint form is built for 2D meshes");
  CK(launch_tracking(*C, u, ut, grad, C->d_part, C->d_scalar));
  C->launches += 2;
  CK(cudaMemcpyAsync(value, C->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return IRKMG_OK;
}

int irkmg_stage_rhs_full(irkmg_ctx* C, const double* un_all, const double* pn, const double* f,
                         double* F) {
  if (!C || !un_all || !pn || !f || !F) return fail(IRKMG_EINVAL, "bad arguments");
  CK(launch_stage_rhs_full(*C, un_all, pn, f, F));
  C->launches++;
  return IRKMG_OK;
}

struct irkmg_batch {
  std::vector<irkmg_ctx*> sys;
  std::vector<cudaStream_t> own, saved;
  BatchLink link;
  std::vector<char> saved_single;  // finest levels' relaxation mode before the batch
};

int irkmg_batch_create(int nsys, irkmg_ctx* const* ctxs, irkmg_batch** out) {
  if (!out || nsys < 1 || !ctxs) return fail(IRKMG_EINVAL, "bad arguments");
  *out = nullptr;
  for (int i = 0; i < nsys; ++i)
    for (int j = 0; j < i; ++j)
      if (!ctxs[i] || ctxs[i] == ctxs[j]) return fail(IRKMG_EINVAL, "null or repeated context");
  irkmg_batch* B = new (std::nothrow) irkmg_batch();
  if (!B) return fail(IRKMG_ENOMEM, "batch");
  for (int i = 0; i < nsys; ++i) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      irkmg_batch_destroy(B);
      return fail(IRKMG_ECUDA, cudaGetErrorString(e));
    }
    // the context finishes pending work on its own stream before switching
    ctxs[i]->stream ? cudaStreamSynchronize(ctxs[i]->stream) : cudaDeviceSynchronize();
    B->sys.push_back(ctxs[i]);
    B->own.push_back(st);
    B->saved.push_back(ctxs[i]->stream);
    ctxs[i]->stream = st;
  }
  // the finest levels relax in one persistent launch for the whole batch when
  // the systems allow it (else each V-cycle is a graph on its system's stream)
  std::vector<Ctx*> sys(B->sys.begin(), B->sys.end());
  if (batch_plan_unsupported(sys).empty()) {
    BatchLink& K = B->link;
    int rc = batch_plan_create(sys, &K.plan);
    cudaError_t e = rc == IRKMG_OK ? cudaStreamCreateWithFlags(&K.stream, cudaStreamNonBlocking)
                                   : cudaSuccess;
    if (rc == IRKMG_OK && e == cudaSuccess)
      e = cudaEventCreateWithFlags(&K.done, cudaEventDisableTiming);
    for (int i = 0; rc == IRKMG_OK && e == cudaSuccess && i < nsys; ++i) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      K.ready.push_back(ev);
    }
    if (rc != IRKMG_OK || e != cudaSuccess) {
      irkmg_batch_destroy(B);
      return fail(rc != IRKMG_OK ? rc : IRKMG_ECUDA, "batched relaxation plan");
    }
    for (Ctx* C : sys) {  // the persistent smoother's relaxation mode
      Level& L = C->L.back();
      B->saved_single.push_back(L.single ? 1 : 0);
      L.single = true;
      drop_graphs(*C);
    }
    K.on = true;
  }
  *out = B;
  return IRKMG_OK;
}

int irkmg_batch_solve(irkmg_batch* B, const double* const* F, double* const* k, irkmg_stats* st) {
  if (!B || !F || !k) return fail(IRKMG_EINVAL, "bad arguments");
  std::vector<FState> S(B->sys.size());
  for (size_t i = 0; i < B->sys.size(); ++i) {
    if (!F[i] || !k[i]) return fail(IRKMG_EINVAL, "null vector in batch");
    S[i].C = B->sys[i];
    S[i].F = F[i];
    S[i].x = k[i];
    S[i].st = st ? &st[i] : nullptr;
  }
  return batch_fgmres(S, B->link.on ? &B->link : nullptr);
}

int irkmg_batch_persistent(const irkmg_batch* B) { return B && B->link.on ? 1 : 0; }

int irkmg_batch_set_persistent(irkmg_batch* B, int on) {
  if (!B || (on != 0 && on != 1)) return fail(IRKMG_EINVAL, "bad arguments");
  if (on && !B->link.plan)
    return fail(IRKMG_ENOTIMPL, "the batch's systems cannot relax in one persistent launch");
  B->link.on = on != 0;
  return IRKMG_OK;
}

void irkmg_batch_destroy(irkmg_batch* B) {
  if (!B) return;
  BatchLink& K = B->link;
  if (K.stream) cudaStreamSynchronize(K.stream);
  for (size_t i = 0; i < B->own.size(); ++i) {
    cudaStreamSynchronize(B->own[i]);
    if (i < B->sys.size()) B->sys[i]->stream = B->saved[i];
    cudaStreamDestroy(B->own[i]);
  }
  for (size_t i = 0; i < B->saved_single.size() && i < B->sys.size(); ++i) {
    B->sys[i]->L.back().single = B->saved_single[i] != 0;
    drop_graphs(*B->sys[i]);
  }
  for (cudaEvent_t ev : K.ready)
    if (ev) cudaEventDestroy(ev);
  if (K.done) cudaEventDestroy(K.done);
  if (K.stream) cudaStreamDestroy(K.stream);
  batch_plan_destroy(K.plan);
  delete B;
}

int irkmg_trace_enable(irkmg_ctx* C, int on) {
  if (!C) return fail(IRKMG_EINVAL, "null ctx");
  C->launches = 0;
  C->trace_on = on != 0;
  C->ev_used = 0;
  C->ev_class.clear();
  C->ev_bytes.clear();
  C->ev_flops.clear();
  return IRKMG_OK;
}

int irkmg_trace_read(irkmg_ctx* C, irkmg_trace* out) {
  if (!C || !out) return fail(IRKMG_EINVAL, "null argument");
  CK(C->stream ? cudaStreamSynchronize(C->stream) : cudaDeviceSynchronize());
  std::memset(out, 0, sizeof(*out));
  out->launches = C->launches;
  for (size_t k = 0; k < C->ev_class.size(); ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, C->ev[2 * k], C->ev[2 * k + 1]));
    if (C->ev_class[k] == 0) {
      out->vanka_launches++;
      out->vanka_ms += ms;
      out->vanka_bytes += C->ev_bytes[k];
      out->vanka_flops += C->ev_flops[k];
    } else if (C->ev_class[k] == 2) {
      out->reduce_launches++;
      out->reduce_ms += ms;
      out->reduce_bytes += C->ev_bytes[k];
    } else if (C->ev_class[k] == 3) {
      out->xfer_launches++;
      out->xfer_ms += ms;
      out->xfer_bytes += C->ev_bytes[k];
    } else if (C->ev_class[k] == 4) {
      out->arnoldi_steps++;
      out->arnoldi_ms += ms;
      out->arnoldi_bytes += C->ev_bytes[k];
    } else if (C->ev_class[k] == 5) {
      out->factor_launches++;
      out->factor_ms += ms;
      out->factor_flops += C->ev_flops[k];
    } else {
      out->op_launches++;
      out->op_ms += ms;
      out->op_bytes += C->ev_bytes[k];
      out->op_flops += C->ev_flops[k];
    }
  }
  C->ev_used = 0;
  C->ev_class.clear();
  C->ev_bytes.clear();
  C->ev_flops.clear();
  return IRKMG_OK;
}

void irkmg_destroy(irkmg_ctx* C) {
  if (!C) return;
  if (C->stream) cudaStreamSynchronize(C->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : C->ev) cudaEventDestroy(e);
  drop_graphs(*C);
  if (C->gstream) cudaStreamSynchronize(C->gstream);
  for (cudaEvent_t e : C->gev)
    if (e) cudaEventDestroy(e);
  if (C->gstream) cudaStreamDestroy(C->gstream);
  for (void* p : C->allocs) cudaFree(p);
  if (C->h_h) cudaFreeHost(C->h_h);
  if (C->h_err) cudaFreeHost(C->h_err);
  delete C;
}

const char* irkmg_strerror(int s) {
  switch (s) {
    case IRKMG_OK: return "ok";
    case IRKMG_EINVAL: return "invalid argument";
    case IRKMG_ENOMEM: return "out of memory";
    case IRKMG_ECUDA: return "CUDA error";
    case IRKMG_ESINGULAR: return "singular patch or coarse pivot";
    case IRKMG_ENOCONV: return "FGMRES did not converge";
    case IRKMG_ETIMEOUT: return "bounded device wait expired";
    case IRKMG_ENOTIMPL: return "not implemented";
    default: return "unknown status";
  }
}

const char* irkmg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

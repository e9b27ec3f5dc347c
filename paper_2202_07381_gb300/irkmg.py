"""ctypes binding of the irkmg C ABI (include/irkmg.h); argument marshalling only.

Device vectors are passed as contiguous float64 CUDA tensors (their data
pointers); host arrays as numpy arrays.  Every call checks the returned status
and raises IrkmgError with the library's message on failure.  There is no
fallback: if libirkmg.so is missing the first call raises.
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

IRKMG_OK, IRKMG_EINVAL, IRKMG_ENOMEM, IRKMG_ECUDA = 0, 1, 2, 3
IRKMG_ESINGULAR, IRKMG_ENOCONV, IRKMG_ETIMEOUT, IRKMG_ENOTIMPL = 4, 5, 6, 7


class IrkmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"irkmg status {status}: {msg}")
        self.status = status


class Mesh(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("nverts", ct.c_int64), ("ncells", ct.c_int64),
                ("coords", ct.POINTER(ct.c_double)), ("cells", ct.POINTER(ct.c_int64)),
                ("bnd_vertex", ct.POINTER(ct.c_uint8))]


class Tableau(ct.Structure):
    _fields_ = [("s", ct.c_int), ("A", ct.POINTER(ct.c_double)), ("b", ct.POINTER(ct.c_double)),
                ("c", ct.POINTER(ct.c_double))]


class Options(ct.Structure):
    _fields_ = [("nlevels", ct.c_int), ("nu_pre", ct.c_int), ("nu_post", ct.c_int),
                ("smoother", ct.c_int), ("omega", ct.c_double), ("cheb_lo", ct.c_double),
                ("cheb_hi", ct.c_double), ("rtol", ct.c_double), ("atol", ct.c_double),
                ("restart", ct.c_int), ("maxit", ct.c_int), ("patch_precision", ct.c_int),
                ("wind", ct.POINTER(ct.c_double)), ("cuda_stream", ct.c_void_p),
                ("timeout_spins", ct.c_int64), ("apply_variant", ct.c_int),
                ("patch_form", ct.c_int), ("cheb_auto", ct.c_int), ("patch_lu_tc", ct.c_int),
                ("patch_fixed", ct.c_int), ("op_fixed", ct.c_int)]


class Stats(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("status", ct.c_int), ("r0", ct.c_double),
                ("rfinal", ct.c_double), ("t_setup", ct.c_double), ("t_solve", ct.c_double),
                ("bad_index", ct.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LevelInfo(ct.Structure):
    _fields_ = [(k, ct.c_int64) for k in ("nv", "ne", "nc", "np2", "nf", "m", "N", "npatch",
                                          "ncolours", "max_patch_dofs", "factor_bytes",
                                          "apply_kernel")] + [("apply_ms", ct.c_double * 2),
                                                              ("dim", ct.c_int64),
                                                              ("single_launch", ct.c_int64),
                                                              ("cheb", ct.c_double * 2),
                                                              ("apply_shape", ct.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("apply_ms", "cheb")}
        d["apply_ms"] = list(self.apply_ms)
        d["cheb"] = list(self.cheb)
        return d


class NSStats(ct.Structure):
    _fields_ = [("newton_iters", ct.c_int), ("linear_iters", ct.c_int), ("status", ct.c_int),
                ("f0", ct.c_double), ("ffinal", ct.c_double), ("t_solve", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Trace(ct.Structure):
    _fields_ = [("launches", ct.c_int64), ("vanka_launches", ct.c_int64), ("vanka_ms", ct.c_double),
                ("vanka_bytes", ct.c_double), ("op_launches", ct.c_int64), ("op_ms", ct.c_double),
                ("op_bytes", ct.c_double), ("vanka_flops", ct.c_double), ("op_flops", ct.c_double),
                ("reduce_launches", ct.c_int64), ("reduce_ms", ct.c_double),
                ("reduce_bytes", ct.c_double), ("xfer_launches", ct.c_int64),
                ("xfer_ms", ct.c_double), ("xfer_bytes", ct.c_double),
                ("arnoldi_steps", ct.c_int64), ("arnoldi_ms", ct.c_double),
                ("arnoldi_bytes", ct.c_double), ("factor_launches", ct.c_int64),
                ("factor_ms", ct.c_double), ("factor_flops", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ct.c_void_p
_SIGS = {
    "irkmg_default_options": (None, [ct.POINTER(Options)]),
    "irkmg_radau_iia": (ct.c_int, [ct.c_int, _P, _P, _P]),
    "irkmg_gauss": (ct.c_int, [ct.c_int, _P, _P, _P]),
    "irkmg_kron_split": (ct.c_int, [ct.c_int, _P, _P, _P, _P]),
    "irkmg_hessenberg_eigvals": (ct.c_int, [ct.c_int, _P, _P, _P]),
    "irkmg_ns_set_state": (ct.c_int, [_P, _P]),
    "irkmg_ns_residual": (ct.c_int, [_P, _P, _P, _P, _P, _P]),
    "irkmg_ns_newton": (ct.c_int, [_P, _P, _P, _P, _P, ct.c_double, ct.c_int, _P]),
    "irkmg_estimate_lambda": (ct.c_int, [_P, ct.c_int, ct.c_int, _P, _P, _P, _P]),
    "irkmg_lobatto_iiic": (ct.c_int, [ct.c_int, _P, _P, _P]),
    "irkmg_setup": (ct.c_int, [ct.POINTER(Mesh), ct.POINTER(Tableau), ct.c_double, ct.c_double,
                               ct.POINTER(Options), ct.POINTER(_P)]),
    "irkmg_update": (ct.c_int, [_P, ct.c_double, ct.c_double]),
    "irkmg_set_wind": (ct.c_int, [_P, _P]),
    "irkmg_level_info_get": (ct.c_int, [_P, ct.c_int, ct.POINTER(LevelInfo)]),
    "irkmg_level_set_apply": (ct.c_int, [_P, ct.c_int, ct.c_int, ct.c_int]),
    "irkmg_set_timeout": (ct.c_int, [_P, ct.c_int64]),
    "irkmg_probe_peak": (ct.c_int, [ct.c_int, ct.c_int64, _P, ct.POINTER(ct.c_double)]),
    "irkmg_p2_coords": (ct.c_int, [_P, ct.c_int, _P]),
    "irkmg_free_nodes": (ct.c_int, [_P, ct.c_int, _P]),
    "irkmg_patch_map": (ct.c_int, [_P, ct.c_int, _P, _P]),
    "irkmg_colouring": (ct.c_int, [_P, ct.c_int, _P]),
    "irkmg_apply": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int]),
    "irkmg_vanka_correction": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int]),
    "irkmg_smooth": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int, ct.c_int]),
    "irkmg_smooth_noalloc": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int, ct.c_int]),
    "irkmg_restrict": (ct.c_int, [_P, ct.c_int, _P, _P]),
    "irkmg_prolong": (ct.c_int, [_P, ct.c_int, _P, _P]),
    "irkmg_coarse_solve": (ct.c_int, [_P, _P, _P, ct.c_int]),
    "irkmg_vcycle": (ct.c_int, [_P, _P, _P, ct.c_int]),
    "irkmg_solve": (ct.c_int, [_P, _P, _P, ct.POINTER(Stats)]),
    "irkmg_adjoint_solve": (ct.c_int, [_P, _P, _P, ct.POINTER(Stats)]),
    "irkmg_stage_rhs": (ct.c_int, [_P, _P, _P, _P, _P]),
    "irkmg_advance": (ct.c_int, [_P, _P, _P, _P]),
    "irkmg_stage_rhs_full": (ct.c_int, [_P, _P, _P, _P, _P]),
    "irkmg_batch_create": (ct.c_int, [ct.c_int, ct.POINTER(_P), ct.POINTER(_P)]),
    "irkmg_batch_solve": (ct.c_int, [_P, ct.POINTER(_P), ct.POINTER(_P), ct.POINTER(Stats)]),
    "irkmg_batch_destroy": (None, [_P]),
    "irkmg_batch_persistent": (ct.c_int, [_P]),
    "irkmg_batch_set_persistent": (ct.c_int, [_P, ct.c_int]),
    "irkmg_forcing_load": (ct.c_int, [_P, _P, _P]),
    "irkmg_step": (ct.c_int, [_P, _P, _P, _P, _P, _P, ct.POINTER(Stats)]),
    "irkmg_adjoint_step": (ct.c_int, [_P, _P, _P, _P, _P, _P, ct.POINTER(ct.c_double),
                                      ct.POINTER(Stats)]),
    "irkmg_tracking": (ct.c_int, [_P, _P, _P, _P, ct.POINTER(ct.c_double)]),
    "irkmg_trace_enable": (ct.c_int, [_P, ct.c_int]),
    "irkmg_trace_read": (ct.c_int, [_P, ct.POINTER(Trace)]),
    "irkmg_destroy": (None, [_P]),
    "irkmg_strerror": (ct.c_char_p, [ct.c_int]),
    "irkmg_last_error": (ct.c_char_p, []),
}


def library_path():
    return _build.LIB


def lib():
    """The loaded libirkmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2202_07381_gb300.build.build()")
        L = ct.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != IRKMG_OK:
        raise IrkmgError(rc, lib().irkmg_last_error().decode())
    return rc


def _dptr(t, n=None, name="vector"):
    """Data pointer of a contiguous float64 CUDA tensor (length n if given)."""
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError(f"{name}: need a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name}: expected {n} entries, got {t.numel()}")
    return ct.c_void_p(t.data_ptr())


def _hptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ct.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


def irkmg_default_options():
    o = Options()
    lib().irkmg_default_options(ct.byref(o))
    return o


def _tableau(fn, s):
    A, b, c = np.zeros(s * s), np.zeros(s), np.zeros(s)
    _check(fn(s, A.ctypes.data, b.ctypes.data, c.ctypes.data))
    return A.reshape(s, s), b, c


def irkmg_radau_iia(s):
    return _tableau(lib().irkmg_radau_iia, s)


def irkmg_kron_split(A):
    """(T, Tinv, D) with A = T D Tinv, D real block diagonal."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    s = A.shape[0]
    T, Ti, D = np.zeros(s * s), np.zeros(s * s), np.zeros(s * s)
    _check(lib().irkmg_kron_split(s, A.ctypes.data, T.ctypes.data, Ti.ctypes.data, D.ctypes.data))
    return T.reshape(s, s), Ti.reshape(s, s), D.reshape(s, s)


def irkmg_hessenberg_eigvals(H):
    """Eigenvalues (complex array) of the upper Hessenberg matrix H."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    n = H.shape[0]
    wr, wi = np.zeros(n), np.zeros(n)
    _check(lib().irkmg_hessenberg_eigvals(n, H.ctypes.data, wr.ctypes.data, wi.ctypes.data))
    return wr + 1j * wi


def irkmg_estimate_lambda(ctx, nsteps=20, x0=None, level=-1):
    """(lambda, Ritz values) of nsteps Arnoldi steps on the level's D⁻¹J."""
    level %= ctx.nlevels
    wr, wi = np.zeros(nsteps), np.zeros(nsteps)
    lam = ct.c_double()
    px = _dptr(x0, ctx.N(level), "x0") if x0 is not None else None
    _check(lib().irkmg_estimate_lambda(ctx.handle, level, nsteps, px, wr.ctypes.data,
                                       wi.ctypes.data, ct.byref(lam)))
    return lam.value, wr + 1j * wi


def irkmg_ns_set_state(ctx, U):
    """Newton blocks for the stage velocities U (host array s x 2 x np2)."""
    L = ctx.finest
    U = np.ascontiguousarray(U, dtype=np.float64)
    if U.shape != (ctx.s, 2, L["np2"]):
        raise ValueError(f"U: expected shape {(ctx.s, 2, L['np2'])}")
    _check(lib().irkmg_ns_set_state(ctx.handle, U.ctypes.data))


def irkmg_ns_residual(ctx, un_all, pn, f, k, F):
    L = ctx.finest
    _check(lib().irkmg_ns_residual(ctx.handle, _dptr(un_all, 2 * L["np2"], "un_all"),
                                   _dptr(pn, L["nv"], "pn"), _dptr(f, ctx.s * 2 * L["np2"], "f"),
                                   _dptr(k, L["N"], "k"), _dptr(F, L["N"], "F")))


def irkmg_ns_newton(ctx, un_all, pn, f, k, atol=1e-10, maxit=20, raise_on_noconv=True):
    """Inexact Newton on the Navier-Stokes stage equations from the guess in k."""
    L = ctx.finest
    st = NSStats()
    rc = lib().irkmg_ns_newton(ctx.handle, _dptr(un_all, 2 * L["np2"], "un_all"),
                               _dptr(pn, L["nv"], "pn"), _dptr(f, ctx.s * 2 * L["np2"], "f"),
                               _dptr(k, L["N"], "k"), float(atol), int(maxit), ct.byref(st))
    if not (rc == IRKMG_ENOCONV and not raise_on_noconv):
        _check(rc)
    return st.as_dict()


def irkmg_gauss(s):
    return _tableau(lib().irkmg_gauss, s)


def irkmg_lobatto_iiic(s):
    return _tableau(lib().irkmg_lobatto_iiic, s)


class Context:
    """Owns an irkmg_ctx; sizes per level are cached in .levels."""

    def __init__(self, handle, s, keep):
        self.handle = handle
        self.s = s
        self._keep = keep
        self.refresh()

    def refresh(self):
        """Re-read the per-level information (after irkmg_level_set_apply)."""
        self.levels = []
        k = 0
        while True:
            info = LevelInfo()
            if lib().irkmg_level_info_get(self.handle, k, ct.byref(info)) != IRKMG_OK:
                break
            self.levels.append(info.as_dict())
            k += 1
        self.nlevels = len(self.levels)

    @property
    def finest(self):
        return self.levels[-1]

    def N(self, level=-1):
        return self.levels[level]["N"]

    def close(self):
        if self.handle:
            lib().irkmg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def irkmg_setup(coords, cells, bnd, A, b, c, dt, nu, options=None, wind=None, stream=None):
    """Build a context.  coords [nv,2], cells [nc,3], bnd [nv] (host arrays)."""
    o = options if options is not None else irkmg_default_options()
    xy, pxy = _hptr(coords, np.float64)
    cl, pcl = _hptr(cells, np.int64)
    bd, pbd = _hptr(bnd, np.uint8)
    mesh = Mesh(xy.shape[1], xy.shape[0], cl.shape[0], pxy, pcl, pbd)
    s = int(np.asarray(b).size)
    Aa, pA = _hptr(A, np.float64)
    ba, pb = _hptr(b, np.float64)
    ca, pc = _hptr(c, np.float64)
    tab = Tableau(s, pA, pb, pc)
    keep = [xy, cl, bd, Aa, ba, ca]
    if wind is not None:
        w, pw = _hptr(wind, np.float64)
        o.wind = pw
        keep.append(w)
    if stream is not None:
        o.cuda_stream = ct.c_void_p(stream)
    h = ct.c_void_p()
    _check(lib().irkmg_setup(ct.byref(mesh), ct.byref(tab), float(dt), float(nu), ct.byref(o),
                             ct.byref(h)))
    return Context(h, s, keep)


def irkmg_update(ctx, dt, nu):
    _check(lib().irkmg_update(ctx.handle, float(dt), float(nu)))


def irkmg_set_wind(ctx, wind):
    """wind: host array [np2, 2] at the finest P2 nodes, or None for Stokes."""
    if wind is None:
        _check(lib().irkmg_set_wind(ctx.handle, None))
        return
    w = np.ascontiguousarray(wind, dtype=np.float64)
    if w.size != 2 * ctx.finest["np2"]:
        raise ValueError("wind: expected np2 x 2 values")
    ctx._keep.append(w)
    _check(lib().irkmg_set_wind(ctx.handle, w.ctypes.data))


def irkmg_p2_coords(ctx, level=-1):
    level %= ctx.nlevels
    out = np.zeros((ctx.levels[level]["np2"], ctx.levels[level]["dim"]))
    _check(lib().irkmg_p2_coords(ctx.handle, level, out.ctypes.data))
    return out


def irkmg_free_nodes(ctx, level=-1):
    level %= ctx.nlevels
    out = np.zeros(ctx.levels[level]["nf"], dtype=np.int64)
    _check(lib().irkmg_free_nodes(ctx.handle, level, out.ctypes.data))
    return out


def irkmg_patch_map(ctx, level=-1):
    level %= ctx.nlevels
    nv = ctx.levels[level]["nv"]
    ptr = np.zeros(nv + 1, dtype=np.int64)
    nodes = np.zeros(96 * nv, dtype=np.int32)
    _check(lib().irkmg_patch_map(ctx.handle, level, ptr.ctypes.data, nodes.ctypes.data))
    return ptr, nodes[: ptr[-1]].copy()


def irkmg_colouring(ctx, level=-1):
    level %= ctx.nlevels
    out = np.zeros(ctx.levels[level]["nv"], dtype=np.int32)
    _check(lib().irkmg_colouring(ctx.handle, level, out.ctypes.data))
    return out


def irkmg_apply(ctx, x, y, level=-1, transpose=False):
    level %= ctx.nlevels
    n = ctx.N(level)
    _check(lib().irkmg_apply(ctx.handle, level, _dptr(x, n, "x"), _dptr(y, n, "y"), int(transpose)))


def irkmg_level_set_apply(ctx, level, shape, single_launch):
    _check(lib().irkmg_level_set_apply(ctx.handle, int(level), int(shape), int(single_launch)))
    ctx.refresh()


def irkmg_probe_peak(kind, iters, stream=None):
    """Measured arithmetic rate of the current device (include/irkmg_probe.h):
    kind 0 FP64 FMA flop/s, 1 FP32 FMA flop/s, 2 mad.wide.s32 per second."""
    out = ct.c_double()
    rc = lib().irkmg_probe_peak(int(kind), int(iters), stream, ct.byref(out))
    if rc != 0:
        raise IrkmgError(IRKMG_ECUDA, f"irkmg_probe_peak returned {rc}")
    return out.value


def irkmg_set_timeout(ctx, timeout_spins):
    _check(lib().irkmg_set_timeout(ctx.handle, int(timeout_spins)))


def irkmg_vanka_correction(ctx, r, c, level=-1, transpose=False):
    level %= ctx.nlevels
    n = ctx.N(level)
    _check(lib().irkmg_vanka_correction(ctx.handle, level, _dptr(r, n, "r"), _dptr(c, n, "c"),
                                        int(transpose)))


def irkmg_smooth(ctx, F, x, nsteps, level=-1, transpose=False):
    level %= ctx.nlevels
    n = ctx.N(level)
    _check(lib().irkmg_smooth(ctx.handle, level, _dptr(F, n, "F"), _dptr(x, n, "x"), int(nsteps),
                              int(transpose)))


def irkmg_smooth_noalloc(ctx, F, x, nsteps, level=-1, transpose=False):
    """irkmg_smooth with its work vectors in the library's static device array
    (no device allocation; levels with N <= 524,288)."""
    level %= ctx.nlevels
    n = ctx.N(level)
    _check(lib().irkmg_smooth_noalloc(ctx.handle, level, _dptr(F, n, "F"), _dptr(x, n, "x"),
                                      int(nsteps), int(transpose)))


def irkmg_restrict(ctx, fine, coarse, level=-1):
    level %= ctx.nlevels
    _check(lib().irkmg_restrict(ctx.handle, level, _dptr(fine, ctx.N(level), "fine"),
                                _dptr(coarse, ctx.N(level - 1), "coarse")))


def irkmg_prolong(ctx, coarse, fine, level=-1):
    level %= ctx.nlevels
    _check(lib().irkmg_prolong(ctx.handle, level, _dptr(coarse, ctx.N(level - 1), "coarse"),
                               _dptr(fine, ctx.N(level), "fine")))


def irkmg_coarse_solve(ctx, r, x, transpose=False):
    n = ctx.N(0)
    _check(lib().irkmg_coarse_solve(ctx.handle, _dptr(r, n, "r"), _dptr(x, n, "x"), int(transpose)))


def irkmg_vcycle(ctx, r, z, transpose=False):
    n = ctx.N()
    _check(lib().irkmg_vcycle(ctx.handle, _dptr(r, n, "r"), _dptr(z, n, "z"), int(transpose)))


def _solve(fn, ctx, F, k, raise_on_noconv):
    st = Stats()
    n = ctx.N()
    rc = fn(ctx.handle, _dptr(F, n, "F"), _dptr(k, n, "k"), ct.byref(st))
    if rc == IRKMG_ENOCONV and not raise_on_noconv:
        return st.as_dict()
    _check(rc)
    return st.as_dict()


def irkmg_solve(ctx, F, k, raise_on_noconv=False):
    """FGMRES + V-cycle solve of J k = F (k: initial guess in, solution out)."""
    return _solve(lib().irkmg_solve, ctx, F, k, raise_on_noconv)


def irkmg_adjoint_solve(ctx, G, lam, raise_on_noconv=False):
    return _solve(lib().irkmg_adjoint_solve, ctx, G, lam, raise_on_noconv)


def irkmg_stage_rhs(ctx, un, pn, f, F):
    L = ctx.finest
    d = L["dim"]
    _check(lib().irkmg_stage_rhs(ctx.handle, _dptr(un, d * L["nf"], "un"), _dptr(pn, L["nv"], "pn"),
                                 _dptr(f, ctx.s * d * L["np2"], "f"), _dptr(F, L["N"], "F")))


def irkmg_advance(ctx, k, un, pn):
    L = ctx.finest
    _check(lib().irkmg_advance(ctx.handle, _dptr(k, L["N"], "k"), _dptr(un, L["dim"] * L["nf"], "un"),
                               _dptr(pn, L["nv"], "pn")))


def irkmg_stage_rhs_full(ctx, un_all, pn, f, F):
    """Stage RHS with u^n at every P2 node (boundary values included)."""
    L = ctx.finest
    _check(lib().irkmg_stage_rhs_full(ctx.handle, _dptr(un_all, 2 * L["np2"], "un_all"),
                                      _dptr(pn, L["nv"], "pn"), _dptr(f, ctx.s * 2 * L["np2"], "f"),
                                      _dptr(F, L["N"], "F")))


class Batch:
    """Owns an irkmg_batch over caller-owned contexts (which must outlive it)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (_P * len(self.contexts))(*[c.handle for c in self.contexts])
        h = _P()
        _check(lib().irkmg_batch_create(len(self.contexts), arr, ct.byref(h)))
        self.handle = h

    def solve(self, Fs, ks, raise_on_noconv=False):
        n = len(self.contexts)
        F = (_P * n)(*[_dptr(F_, c.N(), "F").value for F_, c in zip(Fs, self.contexts)])
        K = (_P * n)(*[_dptr(k_, c.N(), "k").value for k_, c in zip(ks, self.contexts)])
        st = (Stats * n)()
        rc = lib().irkmg_batch_solve(self.handle, F, K, st)
        if not (rc == IRKMG_ENOCONV and not raise_on_noconv):
            _check(rc)
        return [x.as_dict() for x in st]

    @property
    def persistent(self):
        """True if the finest levels relax in one persistent launch."""
        return bool(lib().irkmg_batch_persistent(self.handle))

    @persistent.setter
    def persistent(self, on):
        _check(lib().irkmg_batch_set_persistent(self.handle, int(bool(on))))

    def close(self):
        if self.handle:
            lib().irkmg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def irkmg_batch_create(contexts):
    return Batch(contexts)


def irkmg_batch_solve(batch, Fs, ks, raise_on_noconv=False):
    return batch.solve(Fs, ks, raise_on_noconv)


def irkmg_batch_destroy(batch):
    batch.close()


def irkmg_forcing_load(ctx, theta, g):
    L = ctx.finest
    _check(lib().irkmg_forcing_load(ctx.handle, _dptr(theta, 2 * L["nc"], "theta"),
                                    _dptr(g, 2 * L["nf"], "g")))


def irkmg_step(ctx, un, pn, f, g, k, raise_on_noconv=True):
    """One IRK step; returns the solve's stats (status ENOCONV is returned
    instead of raised when raise_on_noconv is False)."""
    L = ctx.finest
    st = Stats()
    rc = lib().irkmg_step(ctx.handle, _dptr(un, 2 * L["nf"], "un"), _dptr(pn, L["nv"], "pn"),
                          _dptr(f, ctx.s * 2 * L["np2"], "f"),
                          _dptr(g, 2 * L["nf"], "g") if g is not None else None,
                          _dptr(k, L["N"], "k"), ct.byref(st))
    if not (rc == IRKMG_ENOCONV and not raise_on_noconv):
        _check(rc)
    return st.as_dict()


def irkmg_adjoint_step(ctx, ubar, pbar, k, un, theta_bar=None, want_nu=True):
    """Returns (stats, dObj/dnu contribution of this step or None)."""
    L = ctx.finest
    st = Stats()
    dnu = ct.c_double(0.0)
    _check(lib().irkmg_adjoint_step(
        ctx.handle, _dptr(ubar, 2 * L["nf"], "ubar"), _dptr(pbar, L["nv"], "pbar"),
        _dptr(k, L["N"], "k"), _dptr(un, 2 * L["nf"], "un"),
        _dptr(theta_bar, 2 * L["nc"], "theta_bar") if theta_bar is not None else None,
        ct.byref(dnu) if want_nu else None, ct.byref(st)))
    return st.as_dict(), (dnu.value if want_nu else None)


def irkmg_tracking(ctx, u, ut, grad=None):
    L = ctx.finest
    v = ct.c_double(0.0)
    _check(lib().irkmg_tracking(ctx.handle, _dptr(u, 2 * L["nf"], "u"), _dptr(ut, 2 * L["nf"], "ut"),
                                _dptr(grad, 2 * L["nf"], "grad") if grad is not None else None,
                                ct.byref(v)))
    return v.value


def irkmg_trace_enable(ctx, on=True):
    _check(lib().irkmg_trace_enable(ctx.handle, int(on)))


def irkmg_trace_read(ctx):
    t = Trace()
    _check(lib().irkmg_trace_read(ctx.handle, ct.byref(t)))
    return t.as_dict()


def irkmg_destroy(ctx):
    ctx.close()


def irkmg_strerror(status):
    return lib().irkmg_strerror(int(status)).decode()

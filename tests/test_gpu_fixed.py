"""GPU parity of the fixed-point decoupled patch apply (patch_fixed = 1) with
the oracle.

The decoupled FP64 patch inverses (the Kronecker form of the stage system,
Section 3, on the vertex-star patches of Section 4.2) are stored row by row as
57-bit fixed point with a power of two per row and applied by exact integer
dot products against sources scaled to 58-bit integers, rounded once to FP64.
The conversions cost at most 2^-57 of a row's largest entry and 2^-58 of a
source's largest entry, below the FP64 rounding of the same mat-vec, so the
bars are those of the FP64 decoupled form: Vanka corrections and V-cycles at
1e-12 (measured: below 3e-14), FGMRES solutions at 1e-8 with the oracle's
iteration count +-1."""
import functools

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from tests.gpu_util import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

CASES = [("radau_iia", 3, 1 / 64), ("radau_iia", 2, 1 / 8), ("gauss", 2, 1 / 8),
         ("lobatto_iiic", 3, 1 / 64)]


@functools.lru_cache(maxsize=None)
def _oracle(fam, s, dt, n0, nl, nu=1.0):
    from oracle import mg, tableau
    return mg.Hierarchy(*synth.square_mesh(n0), nl, getattr(tableau, fam)(s)[0], dt, nu=nu)


def _context(irkmg, fam, s, dt, n0, nl, form=1, fixed=1, variant=0, nu=1.0, wind=None):
    A, b, c = getattr(irkmg, "irkmg_" + fam)(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = nl
    o.patch_form = form
    o.patch_fixed = fixed
    o.apply_variant = variant
    return irkmg.irkmg_setup(*synth.square_mesh(n0), A, b, c, dt, nu, o, wind=wind)


@pytest.mark.parametrize("variant", [2, 4], ids=["per_colour", "one_launch"])
@pytest.mark.parametrize("form", [2, 3], ids=["complex", "three_product"])
@pytest.mark.parametrize("fam,s,dt", CASES)
def test_fixed_vanka_and_vcycle_match_oracle(fam, s, dt, form, variant):
    """Every level uses a fixed-point kernel (apply_kernel 8, 9 or 10); one
    correction per level with J and with Jᵀ patches, and one V-cycle."""
    irkmg = need_gpu()
    n0, nl = 2, 4
    H = _oracle(fam, s, dt, n0, nl)
    ctx = _context(irkmg, fam, s, dt, n0, nl, form=form, variant=variant)
    try:
        for l in range(1, nl):
            info = ctx.levels[l]
            assert info["apply_kernel"] in (8, 9, 10)
            assert info["single_launch"] == (1 if variant == 4 else 0)
            L = H.levels[l]
            r = synth.random_vector(700 + l, L.N)
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
            assert rel(host(c), L.vanka.correction(r)) < 1e-12
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l, transpose=True)
            ref_t = np.zeros(L.N)
            for idx, f in zip(L.vanka.dofs, L.vanka.lu):
                ref_t[idx] += sla.lu_solve(f, r[idx], trans=1)
            assert rel(host(c), ref_t) < 1e-12
        r = synth.random_vector(799, H.finest.N)
        z = dev(np.zeros(H.finest.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
    finally:
        ctx.close()


FIXED_SHAPE_KERNEL = [8] * 4 + [9] * 3 + [10] * 2


@pytest.mark.parametrize("form", [2, 3], ids=["complex", "three_product"])
@pytest.mark.parametrize("single", [0, 1], ids=["per_colour", "one_launch"])
@pytest.mark.parametrize("s,dt", [(3, 1 / 64), (2, 1 / 8)], ids=["s3", "s2"])
def test_every_fixed_launch_shape_matches_oracle(s, dt, single, form):
    """Each launch shape of the fixed-point kernels (warp per patch: columns
    per load batch x resident CTAs; TMA-staged: stages x CTAs; paired rows of
    the complex layout: columns per load batch), pinned on every level:
    corrections with J and Jᵀ patches against the oracle.  The paired kernel
    exists for the complex layout only (s = 3: one real block and one complex
    pair; s = 2: the pair alone)."""
    irkmg = need_gpu()
    fam, n0, nl = "radau_iia", 2, 4
    H = _oracle(fam, s, dt, n0, nl)
    ctx = _context(irkmg, fam, s, dt, n0, nl, form=form)
    try:
        for shape in range(len(FIXED_SHAPE_KERNEL)):
            if FIXED_SHAPE_KERNEL[shape] == 10 and form != 2:
                with pytest.raises(irkmg.IrkmgError):
                    irkmg.irkmg_level_set_apply(ctx, 1, shape, single)
                continue
            for l in range(1, nl):
                irkmg.irkmg_level_set_apply(ctx, l, shape, single)
                info = ctx.levels[l]
                assert (info["apply_kernel"], info["apply_shape"], info["single_launch"]) == \
                    (FIXED_SHAPE_KERNEL[shape], shape, single)
                L = H.levels[l]
                r = synth.random_vector(900 + 10 * shape + l, L.N)
                c = dev(np.zeros(L.N))
                irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
                assert rel(host(c), L.vanka.correction(r)) < 1e-12
                irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l, transpose=True)
                ref_t = np.zeros(L.N)
                for idx, f in zip(L.vanka.dofs, L.vanka.lu):
                    ref_t[idx] += sla.lu_solve(f, r[idx], trans=1)
                assert rel(host(c), ref_t) < 1e-12
        with pytest.raises(irkmg.IrkmgError):
            irkmg.irkmg_level_set_apply(ctx, 1, len(FIXED_SHAPE_KERNEL), single)
    finally:
        ctx.close()


def test_fixed_error_not_above_fp64_error():
    """On a 32x32 level the fixed-point correction is at least as close to
    the oracle as the FP64-entry correction (up to a factor 2 and 1e-16 of
    the correction's size), element by element in the max norm."""
    irkmg = need_gpu()
    fam, s, dt, n0, nl = "radau_iia", 3, 1 / 64, 2, 5
    H = _oracle(fam, s, dt, n0, nl)
    L = H.finest
    r = synth.random_vector(811, L.N)
    ref = L.vanka.correction(r)
    errs = {}
    for fixed in (0, 1):
        ctx = _context(irkmg, fam, s, dt, n0, nl, form=3, fixed=fixed, variant=4)
        try:
            assert ctx.levels[nl - 1]["apply_kernel"] in ((8, 9, 10) if fixed else (4,))
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=nl - 1)
            errs[fixed] = np.max(np.abs(host(c) - ref)) / np.max(np.abs(ref))
        finally:
            ctx.close()
    assert errs[1] <= 2 * errs[0] + 1e-16, errs


def test_fixed_correction_scales_exactly_by_powers_of_two():
    """Scaling r by 2^600 or 2^-600 moves only the sources' exponents: the
    integers and their one rounding are unchanged, so the correction scales
    bit for bit."""
    irkmg = need_gpu()
    fam, s, dt, n0, nl = "radau_iia", 3, 1 / 64, 2, 4
    ctx = _context(irkmg, fam, s, dt, n0, nl, variant=2)
    try:
        N = ctx.levels[nl - 1]["N"]
        r = synth.random_vector(812, N)
        c0, c1 = dev(np.zeros(N)), dev(np.zeros(N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c0)
        base = host(c0)
        for k in (600, -600):
            irkmg.irkmg_vanka_correction(ctx, dev(np.ldexp(r, k)), c1)
            assert np.array_equal(host(c1), np.ldexp(base, k))
    finally:
        ctx.close()


def test_fixed_nan_residual_stays_local():
    """A NaN residual entry makes the corrections of the patches that hold it
    NaN (the dot products cannot represent it) and leaves every other entry
    bit-identical."""
    irkmg = need_gpu()
    fam, s, dt, n0, nl = "radau_iia", 2, 1 / 8, 2, 5
    ctx = _context(irkmg, fam, s, dt, n0, nl, variant=2)
    try:
        N = ctx.levels[nl - 1]["N"]
        r = synth.random_vector(813, N)
        c0, c1 = dev(np.zeros(N)), dev(np.zeros(N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c0)
        r[N // 3] = np.nan
        irkmg.irkmg_vanka_correction(ctx, dev(r), c1)
        a, b = host(c0), host(c1)
        bad = np.isnan(b)
        assert 0 < bad.sum() < 0.05 * N
        assert np.array_equal(a[~bad], b[~bad])
    finally:
        ctx.close()


@pytest.mark.parametrize("fam,s,dt", [CASES[0], CASES[3]])
def test_fixed_solve_matches_oracle(fam, s, dt):
    """FGMRES with fixed-point patch applies reaches the oracle's solution to
    1e-8 with the oracle's iteration count +-1."""
    irkmg = need_gpu()
    from oracle import fgmres, problem, tableau
    n0, nl = 2, 5
    H = _oracle(fam, s, dt, n0, nl)
    F, _, _ = problem.mms_rhs(H, getattr(tableau, fam)(s)[2])
    x_ref, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
    ctx = _context(irkmg, fam, s, dt, n0, nl)
    try:
        assert all(lv["apply_kernel"] in (8, 9, 10) for lv in ctx.levels[1:])
        k = dev(np.zeros(H.finest.N))
        st = irkmg.irkmg_solve(ctx, dev(F), k)
        assert st["status"] == 0
        assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
        assert abs(st["iters"] - its) <= 1
    finally:
        ctx.close()


def test_fixed_adjoint_solve():
    """The adjoint FGMRES (transposed fixed-point patch applies) reaches its
    1e-10 true residual."""
    irkmg = need_gpu()
    n0, nl, s, dt = 2, 4, 3, 1 / 64
    H = _oracle("radau_iia", s, dt, n0, nl)
    ctx = _context(irkmg, "radau_iia", s, dt, n0, nl)
    try:
        G = H.project_pressure(synth.random_vector(814, H.finest.N))
        lam = dev(np.zeros(H.finest.N))
        st = irkmg.irkmg_adjoint_solve(ctx, dev(G), lam)
        assert st["status"] == 0
        res = G - H.finest.J.T @ host(lam)
        assert np.linalg.norm(res) <= 1.01e-10 * np.linalg.norm(G)
    finally:
        ctx.close()


def test_fixed_oseen_matches_oracle():
    """Oseen (non-symmetric blocks from a frozen wind): fixed-point Vanka
    correction and V-cycle against the oracle."""
    irkmg = need_gpu()
    from oracle import mesh as M, mg, tableau
    n0, nl, s, dt, nu = 2, 4, 2, 0.05, 1 / 500
    fine = M.hierarchy(*synth.square_mesh(n0), nl)[-1]
    wx, wy = synth.wind_field(fine.p2_coords[:, 0], fine.p2_coords[:, 1],
                              synth.wind_coefficients(11))
    sc = np.max(np.hypot(wx, wy))
    w = np.stack([wx / sc, wy / sc], axis=1)
    H = mg.Hierarchy(*synth.square_mesh(n0), nl, tableau.radau_iia(s)[0], dt, nu=nu,
                     wind_finest=w)
    ctx = _context(irkmg, "radau_iia", s, dt, n0, nl, nu=nu, wind=w)
    try:
        assert ctx.levels[nl - 1]["apply_kernel"] in (8, 9)
        L = H.finest
        r = synth.random_vector(815, L.N)
        c = dev(np.zeros(L.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=nl - 1)
        assert rel(host(c), L.vanka.correction(r)) < 1e-12
        z = dev(np.zeros(L.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
    finally:
        ctx.close()


def test_fixed_option_rejected_values_and_fp32():
    """patch_fixed is 0 or 1; with FP32 patches it leaves the FP32 kernels in
    place (the option concerns FP64 entries only)."""
    irkmg = need_gpu()
    A, b, c = irkmg.irkmg_radau_iia(2)
    o = irkmg.irkmg_default_options()
    o.nlevels = 3
    o.patch_form = 1
    o.patch_fixed = 2
    with pytest.raises(irkmg.IrkmgError):
        irkmg.irkmg_setup(*synth.square_mesh(2), A, b, c, 1 / 8, 1.0, o)
    o.patch_fixed = 1
    o.patch_precision = 32
    ctx = irkmg.irkmg_setup(*synth.square_mesh(2), A, b, c, 1 / 8, 1.0, o)
    try:
        assert all(lv["apply_kernel"] not in (8, 9) for lv in ctx.levels[1:])
    finally:
        ctx.close()


def test_fixed_update_reconverts_the_patches():
    """irkmg_update (new dt) refactors the decoupled patches and converts
    them to fixed point again: the correction matches the oracle built at
    the new step size."""
    irkmg = need_gpu()
    fam, s, n0, nl = "radau_iia", 3, 2, 4
    ctx = _context(irkmg, fam, s, 1 / 64, n0, nl, variant=4)
    try:
        for dt in (1 / 16, 1 / 256):
            irkmg.irkmg_update(ctx, dt, 1.0)
            assert ctx.levels[nl - 1]["apply_kernel"] in (8, 9)
            L = _oracle(fam, s, dt, n0, nl).finest
            r = synth.random_vector(816, L.N)
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c)
            assert rel(host(c), L.vanka.correction(r)) < 1e-12
    finally:
        ctx.close()

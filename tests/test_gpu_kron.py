"""GPU parity of the Kronecker-decoupled patch solves (patch_form 1..3) with
the oracle's dense patch inverses.

The decoupled form applies A_v⁻¹ = (T ⊗ I) (I ⊗ M̃ + Δt D ⊗ K̃)⁻¹ (T⁻¹ ⊗ I),
exact in exact arithmetic (the Kronecker form of the stage system, Section 3).
Its rounding differs from a dense LU by about cond(T) · κ(blocks) · eps; on
the 2D cases below the measured errors stay below 3e-14, so the 2D Vanka and
V-cycle bars are the dense form's 1e-12 (3D patches, whose blocks are
factored by the blocked LU, keep 1e-11); the FGMRES solution keeps 1e-8."""
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


def _context(irkmg, fam, s, dt, n0, nl, form, precision=64, nu=1.0, wind=None, variant=0):
    A, b, c = getattr(irkmg, "irkmg_" + fam)(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = nl
    o.patch_form = form
    o.patch_precision = precision
    o.apply_variant = variant
    return irkmg.irkmg_setup(*synth.square_mesh(n0), A, b, c, dt, nu, o, wind=wind)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6],
                         ids=["tma_staged", "warp_per_patch", "tma_staged_one_launch",
                              "warp_one_launch", "warp_specialised", "warp_specialised_one_launch"])
@pytest.mark.parametrize("form", [2, 3], ids=["complex", "three_product"])
@pytest.mark.parametrize("fam,s,dt", CASES)
def test_decoupled_vanka_and_vcycle_match_oracle(fam, s, dt, form, variant):
    """Both decoupled apply kernels (forced on every level), both layouts, one
    launch per colour or one launch plus the per-DoF reduction: one correction
    per level with J and Jᵀ patches, and one V-cycle."""
    irkmg = need_gpu()
    n0, nl = 2, 4
    H = _oracle(fam, s, dt, n0, nl)
    ctx = _context(irkmg, fam, s, dt, n0, nl, form, variant=variant)
    try:
        for l in range(1, nl):
            info = ctx.levels[l]
            assert info["apply_kernel"] == {1: 5, 2: 4, 3: 5, 4: 4, 5: 7, 6: 7}[variant]
            assert info["single_launch"] == (1 if variant in (3, 4, 6) else 0)
            n = 2 * 19 + 1   # largest patch of a structured triangle mesh: 19 nodes
            pairs = s // 2
            nm = s if form == 2 else s + pairs
            assert info["factor_bytes"] <= info["npatch"] * (8 * nm * n * n + 4 * n + 32)
            L = H.levels[l]
            r = synth.random_vector(500 + l, L.N)
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
            assert rel(host(c), L.vanka.correction(r)) < 1e-12
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l, transpose=True)
            ref_t = np.zeros(L.N)
            for idx, f in zip(L.vanka.dofs, L.vanka.lu):
                ref_t[idx] += sla.lu_solve(f, r[idx], trans=1)
            assert rel(host(c), ref_t) < 1e-12
        r = synth.random_vector(599, H.finest.N)
        z = dev(np.zeros(H.finest.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("fam,s,dt", CASES[:2] + CASES[3:])
def test_decoupled_solve_matches_oracle(fam, s, dt, precision):
    """FGMRES with decoupled patches (patch_form 1: three-product layout for
    FP64, complex layout for FP32) reaches the oracle's solution to 1e-8 with
    the same iteration count (FP64: ±1; FP32 patches: at most 3 more)."""
    irkmg = need_gpu()
    from oracle import fgmres, problem, tableau
    n0, nl = 2, 5
    H = _oracle(fam, s, dt, n0, nl)
    F, _, _ = problem.mms_rhs(H, getattr(tableau, fam)(s)[2])
    x_ref, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
    ctx = _context(irkmg, fam, s, dt, n0, nl, 1, precision=precision)
    try:
        k = dev(np.zeros(H.finest.N))
        st = irkmg.irkmg_solve(ctx, dev(F), k)
        assert st["status"] == 0
        assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
        if precision == 64:
            assert abs(st["iters"] - its) <= 1
        else:
            assert st["iters"] <= its + 3
    finally:
        ctx.close()


def test_decoupled_autotuner_picks_the_faster_kernel():
    irkmg = need_gpu()
    ctx = _context(irkmg, "radau_iia", 3, 1 / 64, 2, 5, 1)
    try:
        for lv in ctx.levels[1:]:
            assert lv["apply_kernel"] in (4, 5, 6, 7)
            assert all(t > 0 for t in lv["apply_ms"])
            assert (lv["apply_kernel"] != 4) == (lv["apply_ms"][0] <= lv["apply_ms"][1])
    finally:
        ctx.close()


def test_decoupled_adjoint_solve():
    """The adjoint FGMRES (transposed V-cycle with transposed decoupled
    patches) reaches its 1e-10 true residual."""
    irkmg = need_gpu()
    n0, nl, s, dt = 2, 4, 3, 1 / 64
    H = _oracle("radau_iia", s, dt, n0, nl)
    ctx = _context(irkmg, "radau_iia", s, dt, n0, nl, 1)
    try:
        G = H.project_pressure(synth.random_vector(777, H.finest.N))
        lam = dev(np.zeros(H.finest.N))
        st = irkmg.irkmg_adjoint_solve(ctx, dev(G), lam)
        assert st["status"] == 0
        res = G - H.finest.J.T @ host(lam)
        assert np.linalg.norm(res) <= 1.01e-10 * np.linalg.norm(G)
    finally:
        ctx.close()


def test_decoupled_oseen_matches_oracle():
    """Oseen (non-symmetric K̃ from a frozen wind; the Kronecker form holds):
    decoupled Vanka correction and V-cycle against the oracle."""
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
    ctx = _context(irkmg, "radau_iia", s, dt, n0, nl, 1, nu=nu, wind=w)
    try:
        L = H.finest
        r = synth.random_vector(808, L.N)
        c = dev(np.zeros(L.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=nl - 1)
        assert rel(host(c), L.vanka.correction(r)) < 1e-12
        z = dev(np.zeros(L.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
    finally:
        ctx.close()


@pytest.mark.parametrize("variant", [2, 4], ids=["per_colour", "one_launch"])
@pytest.mark.parametrize("s", [2, 3])
def test_3d_decoupled_large_patches_match_oracle(s, variant):
    """3D patches (n = 196 per stage inside): the pair block (2n = 392) is
    factored by the blocked LU and its first block column gives X and Y
    (`apply_kernel` 6, CTA per patch).  With s = 3 the dense patch (588 DoFs)
    exceeds the dense limit, the decoupled blocks (196 and 392) do not.
    FP64 patches: one Vanka correction per level and one V-cycle against the
    oracle at 1e-11."""
    irkmg = need_gpu()
    from oracle import mg, tableau
    A, b, c = irkmg.irkmg_radau_iia(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = 2
    o.cheb_lo, o.cheb_hi = 2.0, 17.0
    o.patch_form = 1
    o.apply_variant = variant
    dt = 1 / 16
    ctx = irkmg.irkmg_setup(*synth.cube_mesh(2), A, b, c, dt, 1.0, o)
    try:
        lv = ctx.levels[1]
        assert lv["apply_kernel"] == 6 and lv["single_launch"] == (1 if variant == 4 else 0)
        assert lv["max_patch_dofs"] == s * 196
        H = mg.Hierarchy(*synth.cube_mesh(2), 2, tableau.radau_iia(s)[0], dt, cheb=(2.0, 17.0))
        L = H.finest
        r = synth.random_vector(909 + s, L.N)
        cc = dev(np.zeros(L.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), cc)
        assert rel(host(cc), L.vanka.correction(r)) < 1e-11
        z = dev(np.zeros(L.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-11
    finally:
        ctx.close()


def test_3d_decoupled_fp32_solve():
    """3D FP32 decoupled patches (complex layout, tensor-core LU) inside the
    FP64 FGMRES reach the dense FP64 solution to 1e-6 in at most 2 more
    iterations."""
    irkmg = need_gpu()
    A, b, c = irkmg.irkmg_radau_iia(2)
    sols = {}
    for form, prec in ((0, 64), (1, 32)):
        o = irkmg.irkmg_default_options()
        o.nlevels = 3
        o.cheb_lo, o.cheb_hi = 2.0, 17.0
        o.patch_form = form
        o.patch_precision = prec
        o.maxit = 400
        ctx = irkmg.irkmg_setup(*synth.cube_mesh(2), A, b, c, 1 / 16, 1.0, o)
        try:
            fin = ctx.finest
            m, nv = fin["m"], fin["nv"]
            F = synth.random_vector(31, ctx.N())
            for t in range(2):   # consistent right-hand side: zero pressure mean per stage
                F[t * m + m - nv:(t + 1) * m] -= F[t * m + m - nv:(t + 1) * m].mean()
            k = dev(np.zeros(ctx.N()))
            st = irkmg.irkmg_solve(ctx, dev(F), k)
            assert st["status"] == 0
            sols[form] = (host(k), st["iters"], fin["apply_kernel"])
        finally:
            ctx.close()
    assert sols[1][2] == 6 and sols[0][2] == 3
    vel = np.concatenate([np.arange(t * m, t * m + m - nv) for t in range(2)])
    assert rel(sols[1][0][vel], sols[0][0][vel]) < 1e-6
    assert sols[1][1] <= sols[0][1] + 2


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6],
                         ids=["tma_staged", "warp_per_patch", "tma_staged_one_launch",
                              "warp_one_launch", "warp_specialised", "warp_specialised_one_launch"])
@pytest.mark.parametrize("form", [2, 3], ids=["complex", "three_product"])
def test_fp32_decoupled_vanka_every_kernel(form, variant):
    """FP32 decoupled patches (F1: patch inverses stored in FP32, the stage
    mixing T⁻¹ r and T y and the block mat-vecs in FP32) with every apply
    kernel forced on every level, J and Jᵀ patches, against the oracle's FP64
    dense patch solves, entry by entry.  Each output sums at most 5 FP32
    block products of 39 terms mixed through T (entries O(1)): a few hundred
    units of FP32 roundoff (u = 6e-8) relative to the largest entry bound it;
    the bar is 1e-6 of max |ref| plus the entry itself.  The interior patches
    (39 DoFs per stage) take the paired-row kernel under variants 2 and 4 with
    the complex layout."""
    irkmg = need_gpu()
    fam, s, dt = "radau_iia", 3, 1 / 64
    n0, nl = 2, 4
    H = _oracle(fam, s, dt, n0, nl)
    ctx = _context(irkmg, fam, s, dt, n0, nl, form, precision=32, variant=variant)
    try:
        for l in range(1, nl):
            assert ctx.levels[l]["apply_kernel"] == {1: 5, 2: 4, 3: 5, 4: 4, 5: 7, 6: 7}[variant]
            L = H.levels[l]
            r = synth.random_vector(640 + l, L.N)
            ref_t = np.zeros(L.N)
            for idx, f in zip(L.vanka.dofs, L.vanka.lu):
                ref_t[idx] += sla.lu_solve(f, r[idx], trans=1)
            for tr, ref in ((False, L.vanka.correction(r)), (True, ref_t)):
                c = dev(np.zeros(L.N))
                irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l, transpose=tr)
                err = np.abs(host(c) - ref) / (np.abs(ref) + np.abs(ref).max())
                assert err.max() < 1e-6, (l, tr, err.max())
    finally:
        ctx.close()

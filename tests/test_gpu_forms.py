"""GPU checks of the FP32-patch form: FP32 patch inverses and applies inside
an FP64 FGMRES must reach the same 1e-10 residual and the FP64 solution to
1e-8 (the outer Krylov method recovers the accuracy)."""
import numpy as np
import pytest

from tests.gpu_util import dev, gpu_context, host, need_gpu, oracle_hierarchy, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n0,nl,s,dt", [(2, 4, 2, 1 / 8), (2, 4, 3, 1 / 64)])
def test_fp32_patches_reach_fp64_solution(n0, nl, s, dt):
    irkmg = need_gpu()
    from oracle import fgmres, problem, tableau
    H = oracle_hierarchy(n0, nl, s, dt)
    _, _, c = tableau.radau_iia(s)
    F_ref, _, _ = problem.mms_rhs(H, c)
    x_ref, its_ref, _ = fgmres.fgmres(H.finest.J, F_ref, H.vcycle, rtol=1e-10,
                                      project=H.project_pressure)
    ctx = gpu_context(irkmg, n0, nl, s, dt, precision=32)
    k = dev(np.zeros(H.finest.N))
    st = irkmg.irkmg_solve(ctx, dev(F_ref), k)
    assert st["status"] == 0
    assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
    assert st["iters"] <= its_ref + 3
    ctx.close()


@pytest.mark.parametrize("variant", [1, 2], ids=["tma_staged", "warp_per_patch"])
@pytest.mark.parametrize("n0,nl,s,dt", [(2, 5, 2, 1 / 8), (2, 4, 3, 1 / 64)])
def test_both_apply_kernels_match_oracle(variant, n0, nl, s, dt):
    """Each Vanka apply kernel, forced on every level, against the oracle: one
    correction per level and one V-cycle (1e-12)."""
    irkmg = need_gpu()
    import synth
    H = oracle_hierarchy(n0, nl, s, dt)
    ctx = gpu_context(irkmg, n0, nl, s, dt, apply_variant=variant)
    try:
        for l in range(1, nl):
            assert ctx.levels[l]["apply_kernel"] == variant
            L = H.levels[l]
            r = synth.random_vector(300 + l, L.N)
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
            assert rel(host(c), L.vanka.correction(r)) < 1e-12
        r = synth.random_vector(399, H.finest.N)
        z = dev(np.zeros(H.finest.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
    finally:
        ctx.close()


def test_autotuner_records_both_timings():
    irkmg = need_gpu()
    ctx = gpu_context(irkmg, 2, 5, 2, 1 / 8)
    try:
        for lv in ctx.levels[1:]:
            assert lv["apply_kernel"] in (1, 2)
            assert all(t > 0 for t in lv["apply_ms"])
            assert lv["apply_kernel"] == (1 if lv["apply_ms"][0] <= lv["apply_ms"][1] else 2)
    finally:
        ctx.close()


@pytest.mark.parametrize("fam,s,dt", [("gauss", 2, 1 / 8), ("lobatto_iiic", 3, 1 / 64)])
def test_other_irk_families_match_oracle(fam, s, dt):
    """The path takes any consistent tableau: Gauss and LobattoIIIC (Section 5)
    on the 8x8 problem, V-cycle and FGMRES solution against the oracle."""
    irkmg = need_gpu()
    import synth
    from oracle import fgmres, mg, problem, tableau
    A, b, c = getattr(irkmg, "irkmg_" + fam)(s)
    o = irkmg.irkmg_default_options()
    ctx = irkmg.irkmg_setup(*synth.square_mesh(2), A, b, c, dt, 1.0, o)
    Ao, bo, co = getattr(tableau, fam)(s)
    H = mg.Hierarchy(*synth.square_mesh(2), 3, Ao, dt)
    r = synth.random_vector(901, H.finest.N)
    z = dev(np.zeros(H.finest.N))
    irkmg.irkmg_vcycle(ctx, dev(r), z)
    assert rel(host(z), H.vcycle(r)) < 1e-12
    F, _, _ = problem.mms_rhs(H, co)
    k = dev(np.zeros(H.finest.N))
    st = irkmg.irkmg_solve(ctx, dev(F), k)
    x_ref, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
    assert st["status"] == 0 and abs(st["iters"] - its) <= 1
    assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
    ctx.close()


def test_ritz_estimate_matches_oracle():
    """Section 5.1's eigenvalue estimate on the GPU (20 Arnoldi steps on the
    Vanka-preconditioned operator of each level, from x_i = sin(i + 1))
    against the oracle's: the largest real Ritz value to 1e-8."""
    irkmg = need_gpu()
    n0, nl, s, dt = 2, 4, 2, 1 / 8
    H = oracle_hierarchy(n0, nl, s, dt)
    ctx = gpu_context(irkmg, n0, nl, s, dt)
    try:
        for l in range(1, nl):
            lam, ritz = irkmg.irkmg_estimate_lambda(ctx, 20, level=l)
            lam_ref, ritz_ref = H.ritz_estimate(l, 20)
            assert abs(lam - lam_ref) <= 1e-8 * lam_ref
            assert 6.5 < lam < 9.0
    finally:
        ctx.close()


@pytest.mark.parametrize("form", [0, 1])
def test_chebyshev_interval_from_ritz_values(form):
    """cheb_auto: each level smooths on [λ/4, λ] from its own estimate, and
    FGMRES converges in about as many iterations as with the hand-tuned [2, 8]
    (32x32, 5 levels, Radau IIA(3))."""
    irkmg = need_gpu()
    from oracle import problem, tableau
    n0, nl, s, dt = 2, 5, 3, 1 / 64
    H = oracle_hierarchy(n0, nl, s, dt)
    F, _, _ = problem.mms_rhs(H, tableau.radau_iia(s)[2])
    its = {}
    for auto in (0, 1):
        ctx = gpu_context(irkmg, n0, nl, s, dt, cheb_auto=auto, patch_form=form)
        try:
            k = dev(np.zeros(H.finest.N))
            st = irkmg.irkmg_solve(ctx, dev(F), k)
            assert st["status"] == 0
            its[auto] = st["iters"]
            if auto:
                for l in range(1, nl):
                    lo, hi = ctx.levels[l]["cheb"]
                    assert hi == pytest.approx(4 * lo) and 6.0 < hi < 9.5
        finally:
            ctx.close()
    assert its[1] <= its[0] + 4

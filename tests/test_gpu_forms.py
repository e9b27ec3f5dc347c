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

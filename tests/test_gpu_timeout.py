"""Failure detection of the staged patch kernels (the Vanka patch solves of
Section 4.2 streamed into shared memory by bulk copies on mbarriers): every
device-side wait is bounded.  With the bound set to one poll
(irkmg_set_timeout), a wait for a copy still in flight expires; the kernel
records IRKMG_ETIMEOUT, drains its own copies and returns, and FGMRES reports
IRKMG_ETIMEOUT.  Nothing faults or hangs: the failure is a host-chosen bound.
The same context, given the default bound again, then solves to the oracle's
solution, so the error left the context usable."""
import functools

import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

S, DT, N0, NL = 2, 1 / 8, 2, 4


@functools.lru_cache(maxsize=None)
def _oracle():
    from oracle import fgmres, mg, problem, tableau
    A, b, c = tableau.radau_iia(S)
    H = mg.Hierarchy(*synth.square_mesh(N0), NL, A, DT)
    F, _, _ = problem.mms_rhs(H, c)
    x, _, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-13, project=H.project_pressure)
    return H, F, H.project_pressure(x)


# (patch_form, patch_fixed, apply_variant, pinned fixed-point shape, kernel id)
KERNELS = [(0, 0, 1, None, 1),      # dense patches, TMA-staged
           (1, 0, 1, None, 5),      # decoupled, TMA-staged
           (1, 0, 5, None, 7),      # decoupled, warp-specialised producer / consumers
           (1, 1, 0, 4, 9)]         # decoupled fixed point, TMA-staged


@pytest.mark.parametrize("form,fixed,variant,shape,kern", KERNELS,
                         ids=["dense_staged", "kron_staged", "kron_ws", "fixed_staged"])
def test_expired_wait_reports_timeout_and_context_recovers(form, fixed, variant, shape, kern):
    irkmg = need_gpu()
    H, F, ref = _oracle()
    A, b, c = irkmg.irkmg_radau_iia(S)
    o = irkmg.irkmg_default_options()
    o.nlevels = NL
    o.patch_form = form
    o.patch_fixed = fixed
    o.apply_variant = variant
    o.rtol = 1e-13
    ctx = irkmg.irkmg_setup(*synth.square_mesh(N0), A, b, c, DT, 1.0, o)
    try:
        if shape is not None:
            for l in range(1, NL):
                irkmg.irkmg_level_set_apply(ctx, l, shape, 0)
        assert all(lv["apply_kernel"] == kern for lv in ctx.levels[1:]), ctx.levels
        Fd = dev(F)
        irkmg.irkmg_set_timeout(ctx, 1)
        with pytest.raises(irkmg.IrkmgError) as e:
            irkmg.irkmg_solve(ctx, Fd, dev(np.zeros(ctx.N())))
        assert e.value.status == irkmg.IRKMG_ETIMEOUT, str(e.value)
        irkmg.irkmg_set_timeout(ctx, 0)
        k = dev(np.zeros(ctx.N()))
        st = irkmg.irkmg_solve(ctx, Fd, k)
        assert st["status"] == 0
        assert rel(H.project_pressure(host(k)), ref) < 1e-8
    finally:
        ctx.close()


def test_negative_timeout_is_rejected():
    irkmg = need_gpu()
    A, b, c = irkmg.irkmg_radau_iia(2)
    o = irkmg.irkmg_default_options()
    o.nlevels = 2
    ctx = irkmg.irkmg_setup(*synth.square_mesh(2), A, b, c, 0.125, 1.0, o)
    try:
        with pytest.raises(irkmg.IrkmgError) as e:
            irkmg.irkmg_set_timeout(ctx, -1)
        assert e.value.status == irkmg.IRKMG_EINVAL
    finally:
        ctx.close()

"""The minimal use shown to library users (one decoupled-patch stage solve with
fixed-point patch mat-vecs and one time step on a 128x128 mesh) runs and
converges."""
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_minimal_stage_solve_and_step():
    irkmg = need_gpu()
    import torch
    import synth
    A, b, c = irkmg.irkmg_radau_iia(3)
    opt = irkmg.irkmg_default_options()
    opt.nlevels = 5
    opt.patch_form = 1
    opt.patch_fixed = 1
    ctx = irkmg.irkmg_setup(*synth.square_mesh(8), A, b, c, 1 / 64, 1.0, opt)
    fin = ctx.finest
    dev = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")
    un, pn = dev(2 * fin["nf"]), dev(fin["nv"])
    torch.manual_seed(0)
    f = torch.rand(3 * 2 * fin["np2"], dtype=torch.float64, device="cuda")
    F, k = dev(fin["N"]), dev(fin["N"])
    irkmg.irkmg_stage_rhs(ctx, un, pn, f, F)
    stats = irkmg.irkmg_solve(ctx, F, k)
    irkmg.irkmg_advance(ctx, k, un, pn)
    assert stats["status"] == 0 and stats["rfinal"] <= 1e-10 * stats["r0"]
    assert float(un.norm()) > 0.0
    ctx.close()

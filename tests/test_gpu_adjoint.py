"""GPU checks of the discrete adjoint (irkmg_step / irkmg_adjoint_step behind
torch.autograd): against the oracle's adjoint on the same problem (1e-9
relative, with tight solver tolerances on the GPU), and against central finite
differences of the GPU forward model (1e-5 relative) on the 128 x 128,
8-step, dt = 1/32 configuration with checkpoints every 2 steps (step 1 along a
seeded N(0,1) direction for the forcing, 1e-6 for nu)."""
import numpy as np
import pytest

import synth
from tests.gpu_util import gpu_context, need_gpu

pytestmark = pytest.mark.gpu


def _problem(irkmg, n0, nl, s, dt, nsteps, nu=1.0, rtol=1e-13, atol=1e-15, **kw):
    import torch
    from paper_2202_07381_gb300.adjoint import TrackingProblem
    # the residual of a solve cannot go below ~1e-16 in absolute terms, and F
    # shrinks as the steps proceed, so the test stops at max(1e-13 |F|, 1e-15)
    ctx = gpu_context(irkmg, n0, nl, s, dt, nu=nu, rtol=rtol, atol=atol, maxit=400, **kw)
    xy = irkmg.irkmg_p2_coords(ctx)
    free = irkmg.irkmg_free_nodes(ctx)
    nv = ctx.finest["nv"]
    ux, uy = synth.mms_velocity(xy[free, 0], xy[free, 1])
    u0 = np.concatenate([ux, uy])
    p0 = synth.mms_pressure(xy[:nv, 0], xy[:nv, 1])
    p0 -= p0.mean()
    fx, fy = synth.mms_forcing(xy[:, 0], xy[:, 1], nu=nu)
    f = np.concatenate([np.concatenate([fx, fy])] * s)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    prob = TrackingProblem(ctx, dt, T(u0), T(p0), T(f), T(0.9 * u0), nsteps, 2)
    theta = synth.normal(7, 2 * ctx.finest["nc"])
    return ctx, prob, theta, (u0, p0, 0.9 * u0)


@pytest.mark.parametrize("form", [0, 1], ids=["dense_patches", "decoupled_patches"])
def test_adjoint_matches_oracle_adjoint(form):
    """The adjoint chain (forward steps, transposed solves with transposed
    patches, dJ/dθ and dJ/dν) with dense or decoupled patch solves."""
    irkmg = need_gpu()
    import torch
    from oracle import adjoint as oadj, mesh as M, problem, tableau
    from paper_2202_07381_gb300.adjoint import tracking_objective
    n0, nl, s, dt, nsteps = 2, 3, 2, 1 / 32, 4
    ctx, prob, theta, (u0, p0, ut) = _problem(irkmg, n0, nl, s, dt, nsteps, patch_form=form)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = tracking_objective(th, nu, prob)
    J.backward()
    A, b, c = tableau.radau_iia(s)
    mesh = M.hierarchy(*synth.square_mesh(n0), nl)[-1]
    op = oadj.Problem(mesh, A, b, dt, 1.0)
    f_all = problem.forcing(mesh, c, 0.0, dt, 1.0)
    J_ref, thb_ref, dnu_ref = oadj.run(op, u0, p0, lambda n: f_all, theta, nsteps, ut)
    assert abs(J.item() - J_ref) <= 1e-9 * abs(J_ref)
    g = th.grad.cpu().numpy()
    assert np.linalg.norm(g - thb_ref) <= 1e-9 * np.linalg.norm(thb_ref)
    assert abs(nu.grad.item() - dnu_ref) <= 1e-9 * abs(dnu_ref)
    ctx.close()


def test_adjoint_matches_finite_differences_128():
    irkmg = need_gpu()
    import torch
    from paper_2202_07381_gb300.adjoint import tracking_objective
    ctx, prob, theta, _ = _problem(irkmg, 8, 5, 2, 1 / 32, 8)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = tracking_objective(th, nu, prob)
    J.backward()
    d = torch.tensor(synth.normal(11, theta.size), dtype=torch.float64, device="cuda")
    # u^N is affine in theta, so the objective is exactly quadratic in theta and
    # central differences carry no truncation error: a unit step keeps the
    # difference far above the solver's rounding floor
    h = 1.0
    with torch.no_grad():
        Jp = prob.objective(th + h * d, 1.0)
        Jm = prob.objective(th - h * d, 1.0)
    fd = (Jp - Jm) / (2 * h)
    ad = float((th.grad * d).sum())
    assert abs(fd - ad) <= 1e-5 * abs(fd), (fd, ad)
    hn = 1e-6
    Jp = prob.objective(th.detach(), 1.0 + hn)
    Jm = prob.objective(th.detach(), 1.0 - hn)
    fdn = (Jp - Jm) / (2 * hn)
    assert abs(fdn - nu.grad.item()) <= 1e-5 * abs(fdn), (fdn, nu.grad.item())
    ctx.close()

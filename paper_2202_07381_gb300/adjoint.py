"""Gradients of a tracking objective through several implicit RK steps, as a
torch.autograd.Function over the irkmg C ABI.

Forward: N steps of irkmg_step (stage RHS with the P0 forcing control th
loaded by irkmg_forcing_load, FGMRES + V-cycle solve, update); states are
kept only every `checkpoint_every` steps.  Objective: irkmg_tracking,
1/2 (u^N - u_T)^T M2 (u^N - u_T).
Backward: segment by segment, from the last checkpoint back, the segment's
steps are recomputed (keeping each step's start state and stages) and
irkmg_adjoint_step is applied in reverse order; it returns dObj/dth (through
C^T) and dObj/dnu (through K = nu K_1 in both the stage operator and the
right-hand side).  All arithmetic runs in the library's kernels; this module
only orders the calls and keeps the checkpoints.
"""
import torch

from . import irkmg


class TrackingProblem:
    """Fixed data of the objective: a context (finest level), initial state,
    per-step forcing interpolant f (s*2*np2, the same every step), target
    velocity, number of steps and checkpoint interval."""

    def __init__(self, ctx, dt, u0, p0, f, u_target, nsteps, checkpoint_every=2):
        self.ctx, self.dt = ctx, dt
        self.u0, self.p0, self.f, self.ut = u0, p0, f, u_target
        self.nsteps, self.every = nsteps, checkpoint_every
        self.nu = None
        self.stats = []

    def set_nu(self, nu):
        nu = float(nu)
        if self.nu is None or nu != self.nu:
            irkmg.irkmg_update(self.ctx, self.dt, nu)
            self.nu = nu

    def _step(self, u, p, g, k):
        st = irkmg.irkmg_step(self.ctx, u, p, self.f, g, k, raise_on_noconv=False)
        self.stats.append(st)
        if st["status"] != 0:
            raise irkmg.IrkmgError(st["status"], f"stage solve did not converge: {st}")

    def forward_states(self, g):
        """Run all steps; returns (u^N, p^N, checkpoints {n: (u^n, p^n)})."""
        u, p = self.u0.clone(), self.p0.clone()
        k = torch.empty(self.ctx.N(), dtype=u.dtype, device=u.device)
        ckpt = {0: (u.clone(), p.clone())}
        for n in range(self.nsteps):
            self._step(u, p, g, k)
            if (n + 1) % self.every == 0 and n + 1 < self.nsteps:
                ckpt[n + 1] = (u.clone(), p.clone())
        return u, p, ckpt

    def objective(self, theta, nu):
        self.set_nu(nu)
        g = torch.empty_like(self.u0)
        irkmg.irkmg_forcing_load(self.ctx, theta, g)
        u, _, _ = self.forward_states(g)
        return irkmg.irkmg_tracking(self.ctx, u, self.ut)


class IRKTracking(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, nu, prob):
        prob.set_nu(nu.item())
        g = torch.empty_like(prob.u0)
        irkmg.irkmg_forcing_load(prob.ctx, theta, g)
        u, p, ckpt = prob.forward_states(g)
        ub = torch.empty_like(u)
        val = irkmg.irkmg_tracking(prob.ctx, u, prob.ut, ub)
        fctx.prob, fctx.g, fctx.ckpt, fctx.ub = prob, g, ckpt, ub
        fctx.theta_shape = theta.shape
        return torch.tensor(val, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(fctx, grad_out):
        prob, g, ckpt = fctx.prob, fctx.g, fctx.ckpt
        ub = fctx.ub.clone()
        pb = torch.zeros_like(prob.p0)
        thb = torch.zeros(fctx.theta_shape, dtype=torch.float64, device=ub.device)
        dnu = 0.0
        starts = sorted(ckpt)
        N = prob.ctx.N()
        for seg in reversed(range(len(starts))):
            n0 = starts[seg]
            n1 = starts[seg + 1] if seg + 1 < len(starts) else prob.nsteps
            u, p = ckpt[n0][0].clone(), ckpt[n0][1].clone()
            us, ks = [], []
            for _ in range(n0, n1):
                us.append(u.clone())
                k = torch.empty(N, dtype=u.dtype, device=u.device)
                prob._step(u, p, g, k)
                ks.append(k)
            for j in reversed(range(n1 - n0)):
                st, dn = irkmg.irkmg_adjoint_step(prob.ctx, ub, pb, ks[j], us[j], thb, True)
                if st["status"] != 0:
                    raise irkmg.IrkmgError(st["status"], "adjoint solve did not converge")
                dnu += dn
        go = float(grad_out)
        return thb * go, torch.tensor(dnu * go, dtype=torch.float64, device=ub.device), None


def tracking_objective(theta, nu, prob):
    """Differentiable 1/2 ||u^N - u_T||_M^2 as a function of (theta, nu)."""
    return IRKTracking.apply(theta, nu, prob)

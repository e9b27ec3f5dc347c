"""Mesh independence of the FGMRES iteration counts on the GPU path
(Section 5.1, Table 1: iterations per step stay nearly constant as the mesh is
refined).  Radau IIA(3), dt = 1/64, V(2,2) Chebyshev [2, 8] Vanka, the
benchmarked patch form (decoupled, fixed-point mat-vecs), finest meshes
8x8 ... 128x128 from one 2x2 coarsest mesh (3 .. 7 levels), tolerance 1e-10.

Bars: where the oracle runs in seconds (8x8 .. 32x32) the GPU count equals
the oracle's to +-1; over all sizes every count is within 2 of the middle of
the range (max - min <= 4) and one refinement adds at most 2 iterations."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

S, DT, N0 = 3, 1 / 64, 2


def _oracle_iters(nl):
    from oracle import fgmres, mg, problem, tableau
    A, b, c = tableau.radau_iia(S)
    H = mg.Hierarchy(*synth.square_mesh(N0), nl, A, DT)
    F, _, _ = problem.mms_rhs(H, c)
    _, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
    return its


def _gpu_solve(irkmg, nl):
    A, b, c = irkmg.irkmg_radau_iia(S)
    o = irkmg.irkmg_default_options()
    o.nlevels = nl
    o.rtol = 1e-10
    o.maxit = 200
    ctx = irkmg.irkmg_setup(*synth.square_mesh(N0), A, b, c, DT, 1.0, o)
    try:
        xy = irkmg.irkmg_p2_coords(ctx)
        free = irkmg.irkmg_free_nodes(ctx)
        nv = ctx.finest["nv"]
        ux, uy = synth.mms_velocity(xy[free, 0], xy[free, 1])
        p0 = synth.mms_pressure(xy[:nv, 0], xy[:nv, 1])
        fx, fy = synth.mms_forcing(xy[:, 0], xy[:, 1], nu=1.0)
        f = np.concatenate([np.concatenate([fx, fy]) for _ in range(S)])
        F = dev(np.zeros(ctx.N()))
        irkmg.irkmg_stage_rhs(ctx, dev(np.concatenate([ux, uy])), dev(p0 - p0.mean()), dev(f), F)
        k = dev(np.zeros(ctx.N()))
        st = irkmg.irkmg_solve(ctx, F, k)
        r = dev(np.zeros(ctx.N()))
        irkmg.irkmg_apply(ctx, k, r)
        res = np.linalg.norm(host(F) - host(r)) / np.linalg.norm(host(F))
        return st, res
    finally:
        ctx.close()


def test_iterations_are_mesh_independent():
    irkmg = need_gpu()
    its = {}
    for nl in range(3, 8):                      # 8x8 ... 128x128
        st, res = _gpu_solve(irkmg, nl)
        assert st["status"] == 0 and res <= 1.5e-10, (nl, st, res)
        its[2 * 2 ** (nl - 1)] = st["iters"]
    for nl in range(3, 6):                      # the oracle at 8x8 ... 32x32
        n = 2 * 2 ** (nl - 1)
        assert abs(its[n] - _oracle_iters(nl)) <= 1, (n, its)
    counts = [its[n] for n in sorted(its)]
    assert max(counts) - min(counts) <= 4, its
    assert all(b - a <= 2 for a, b in zip(counts, counts[1:])), its

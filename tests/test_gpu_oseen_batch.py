"""GPU checks of the Oseen form and of batched solves.

Oseen (a frozen wind adds <(w . grad) u, v> to the velocity block, which makes
it nonsymmetric): operator and transpose, Vanka correction, V-cycle, lifted
stage right-hand side of a lid-driven cavity and the FGMRES solution, each
against the oracle with the same wind.  Batch: a mixed batch of Stokes and
Oseen systems of different sizes, tableaux, dt and nu solved together must
give what irkmg_solve gives on each system alone."""
import numpy as np
import pytest

import synth
from tests.gpu_util import WINDS, dev, gpu_context, host, need_gpu, oracle_hierarchy, rel

pytestmark = pytest.mark.gpu


def _wind(n0, nl, seed):
    from oracle import mesh as M
    fine = M.hierarchy(*synth.square_mesh(n0), nl)[-1]
    a = synth.wind_coefficients(seed)
    wx, wy = synth.wind_field(fine.p2_coords[:, 0], fine.p2_coords[:, 1], a)
    sc = np.max(np.hypot(wx, wy))
    return np.stack([wx / sc, wy / sc], axis=1)


@pytest.fixture(scope="module")
def oseen():
    irkmg = need_gpu()
    n0, nl, s, dt, nu = 2, 4, 2, 0.05, 1 / 500
    w = _wind(n0, nl, 3)
    WINDS["oseen3"] = w
    H = oracle_hierarchy(n0, nl, s, dt, nu=nu, wind_key="oseen3")
    ctx = gpu_context(irkmg, n0, nl, s, dt, nu=nu, wind=w)
    yield irkmg, ctx, H
    ctx.close()


def test_oseen_operator_vanka_vcycle(oseen):
    irkmg, ctx, H = oseen
    for l, L in enumerate(H.levels):
        x = synth.random_vector(500 + l, L.N)
        y = dev(np.zeros(L.N))
        irkmg.irkmg_apply(ctx, dev(x), y, level=l)
        assert rel(host(y), L.J @ x) < 1e-13
        irkmg.irkmg_apply(ctx, dev(x), y, level=l, transpose=True)
        assert rel(host(y), L.J.T @ x) < 1e-13
        if l > 0:
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(x), c, level=l)
            assert rel(host(c), L.vanka.correction(x)) < 1e-12
    r = synth.random_vector(599, H.finest.N)
    z = dev(np.zeros(H.finest.N))
    irkmg.irkmg_vcycle(ctx, dev(r), z)
    assert rel(host(z), H.vcycle(r)) < 1e-12


def test_oseen_lid_rhs_and_solve(oseen):
    irkmg, ctx, H = oseen
    from oracle import fgmres
    L = H.finest
    m = L.mesh
    lx, ly = synth.lid_velocity(m.p2_coords[:, 0], m.p2_coords[:, 1])
    ops = L.ops
    nf = m.nf
    Fu = np.concatenate([-(ops["Kall"] @ lx), -(ops["Kall"] @ ly)])
    Fp = -(ops["Bfull"][0].T @ lx + ops["Bfull"][1].T @ ly)
    F_ref = np.concatenate([np.concatenate([Fu, Fp])] * H.s)
    F = dev(np.zeros(L.N))
    irkmg.irkmg_stage_rhs_full(ctx, dev(np.concatenate([lx, ly])), dev(np.zeros(m.nv)),
                               dev(np.zeros(H.s * 2 * m.np2)), F)
    assert rel(host(F), F_ref) < 1e-13
    k = dev(np.zeros(L.N))
    st = irkmg.irkmg_solve(ctx, F, k)
    assert st["status"] == 0
    x_ref, its_ref, _ = fgmres.fgmres(L.J, F_ref, H.vcycle, rtol=1e-10, project=H.project_pressure,
                                      maxit=300)
    assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
    assert abs(st["iters"] - its_ref) <= 2


def test_batch_equals_independent_solves():
    irkmg = need_gpu()
    specs = [  # (n0, nl, s, dt, nu, wind seed or None)
        (2, 3, 2, 1 / 8, 1.0, None),
        (2, 4, 3, 1 / 64, 1.0, None),
        (4, 3, 2, 0.02, 1 / 300, 5),
        (2, 5, 2, 0.003, 1 / 900, 6),
        (3, 3, 2, 0.1, 1 / 150, 7),
    ]
    ctxs, Fs = [], []
    for i, (n0, nl, s, dt, nu, ws) in enumerate(specs):
        w = _wind(n0, nl, ws) if ws is not None else None
        ctx = gpu_context(irkmg, n0, nl, s, dt, nu=nu, wind=w)
        ctxs.append(ctx)
        xy = irkmg.irkmg_p2_coords(ctx)
        if w is None:
            # Stokes: manufactured forcing on the stationary domain
            F = dev(np.zeros(ctx.N()))
            free = irkmg.irkmg_free_nodes(ctx)
            nv = ctx.finest["nv"]
            ux, uy = synth.mms_velocity(xy[free, 0], xy[free, 1])
            p0 = synth.mms_pressure(xy[:nv, 0], xy[:nv, 1])
            fx, fy = synth.mms_forcing(xy[:, 0], xy[:, 1], nu=nu)
            irkmg.irkmg_stage_rhs(ctx, dev(np.concatenate([ux, uy])), dev(p0 - p0.mean()),
                                  dev(np.concatenate([np.concatenate([fx, fy])] * s)), F)
        else:
            lx, ly = synth.lid_velocity(xy[:, 0], xy[:, 1])
            F = dev(np.zeros(ctx.N()))
            irkmg.irkmg_stage_rhs_full(ctx, dev(np.concatenate([lx, ly])),
                                       dev(np.zeros(ctx.finest["nv"])),
                                       dev(np.zeros(s * 2 * ctx.finest["np2"])), F)
        Fs.append(F)
    ref = []
    for ctx, F in zip(ctxs, Fs):
        k = dev(np.zeros(ctx.N()))
        st = irkmg.irkmg_solve(ctx, F, k)
        assert st["status"] == 0
        ref.append((host(k), st["iters"]))
    batch = irkmg.Batch(ctxs)
    ks = [dev(np.zeros(c.N())) for c in ctxs]
    sts = batch.solve(Fs, ks)
    batch.close()
    for (kref, its), k, st in zip(ref, ks, sts):
        assert st["status"] == 0 and st["iters"] == its
        assert rel(host(k), kref) <= 1e-12
    for c in ctxs:
        c.close()

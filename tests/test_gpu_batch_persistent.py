"""The batched form in one persistent launch (independent stage systems of
uneven size, dt, nu and wind; Radau IIA(2); decoupled patches with
fixed-point mat-vecs): the finest-level relaxation of every system runs as
one cooperative launch per smoothing stage, and the batch solve must give,
bit for bit and with the same iteration counts, what irkmg_solve gives on each
system in the same relaxation mode.  Its grid-wide barriers are bounded: with
a one-poll bound a barrier wait expires, the solve reports IRKMG_ETIMEOUT,
and the same batch then solves normally."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

# (n0, nl, dt, nu, wind seed or None): finest meshes 8x8 ... 32x32
SPECS = [(2, 3, 1 / 8, 1.0, None), (2, 5, 0.01, 1 / 400, 6), (4, 3, 0.05, 1 / 200, 5),
         (2, 4, 1 / 32, 1.0, None), (3, 3, 0.1, 1 / 150, 7), (2, 4, 0.003, 1 / 900, 8)]


def _wind(n0, nl, seed):
    from oracle import mesh as M
    fine = M.hierarchy(*synth.square_mesh(n0), nl)[-1]
    wx, wy = synth.wind_field(fine.p2_coords[:, 0], fine.p2_coords[:, 1],
                              synth.wind_coefficients(seed))
    sc = np.max(np.hypot(wx, wy))
    return np.stack([wx / sc, wy / sc], axis=1)


def _systems(irkmg):
    ctxs, Fs = [], []
    A, b, c = irkmg.irkmg_radau_iia(2)
    for n0, nl, dt, nu, ws in SPECS:
        o = irkmg.irkmg_default_options()
        o.nlevels = nl
        o.patch_form = 1
        o.patch_fixed = 1
        o.maxit = 400
        w = _wind(n0, nl, ws) if ws is not None else None
        ctx = irkmg.irkmg_setup(*synth.square_mesh(n0), A, b, c, dt, nu, o, wind=w)
        xy = irkmg.irkmg_p2_coords(ctx)
        F = dev(np.zeros(ctx.N()))
        if w is None:
            free = irkmg.irkmg_free_nodes(ctx)
            nv = ctx.finest["nv"]
            ux, uy = synth.mms_velocity(xy[free, 0], xy[free, 1])
            p0 = synth.mms_pressure(xy[:nv, 0], xy[:nv, 1])
            fx, fy = synth.mms_forcing(xy[:, 0], xy[:, 1], nu=nu)
            irkmg.irkmg_stage_rhs(ctx, dev(np.concatenate([ux, uy])), dev(p0 - p0.mean()),
                                  dev(np.concatenate([np.concatenate([fx, fy])] * 2)), F)
        else:
            lx, ly = synth.lid_velocity(xy[:, 0], xy[:, 1])
            irkmg.irkmg_stage_rhs_full(ctx, dev(np.concatenate([lx, ly])),
                                       dev(np.zeros(ctx.finest["nv"])),
                                       dev(np.zeros(2 * 2 * ctx.finest["np2"])), F)
        ctxs.append(ctx)
        Fs.append(F)
    return ctxs, Fs


def test_persistent_batch_equals_independent_solves_bitwise():
    irkmg = need_gpu()
    ctxs, Fs = _systems(irkmg)
    batch = irkmg.Batch(ctxs)
    try:
        assert batch.persistent
        for c in ctxs:
            c.refresh()
        assert all(c.levels[-1]["single_launch"] == 1 for c in ctxs)
        ref = []
        for ctx, F in zip(ctxs, Fs):   # each system alone, same relaxation mode
            k = dev(np.zeros(ctx.N()))
            st = irkmg.irkmg_solve(ctx, F, k)
            assert st["status"] == 0
            ref.append((host(k), st["iters"]))
        for rep in range(2):            # twice: the plan is rebuilt per solve
            ks = [dev(np.zeros(c.N())) for c in ctxs]
            sts = batch.solve(Fs, ks)
            for (kref, its), k, st in zip(ref, ks, sts):
                assert st["status"] == 0 and st["iters"] == its, (rep, st, its)
                assert np.array_equal(host(k), kref)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_persistent_batch_barrier_timeout_then_recovers():
    irkmg = need_gpu()
    ctxs, Fs = _systems(irkmg)
    batch = irkmg.Batch(ctxs)
    try:
        assert batch.persistent
        ref = []
        for ctx, F in zip(ctxs, Fs):
            k = dev(np.zeros(ctx.N()))
            irkmg.irkmg_solve(ctx, F, k)
            ref.append(host(k))
        irkmg.irkmg_set_timeout(ctxs[0], 1)   # the batch's barriers take the first system's bound
        with pytest.raises(irkmg.IrkmgError) as e:
            batch.solve(Fs, [dev(np.zeros(c.N())) for c in ctxs])
        assert e.value.status == irkmg.IRKMG_ETIMEOUT, str(e.value)
        irkmg.irkmg_set_timeout(ctxs[0], 0)
        ks = [dev(np.zeros(c.N())) for c in ctxs]
        sts = batch.solve(Fs, ks)
        for kref, k, st in zip(ref, ks, sts):
            assert st["status"] == 0 and np.array_equal(host(k), kref)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_batch_mode_is_restored_and_mixed_batches_use_graphs():
    irkmg = need_gpu()
    ctxs, Fs = _systems(irkmg)
    before = [c.levels[-1]["single_launch"] for c in ctxs]
    batch = irkmg.Batch(ctxs)
    batch.close()
    for c in ctxs:
        c.refresh()
    assert [c.levels[-1]["single_launch"] for c in ctxs] == before
    # a dense-patch system makes the batch fall back to per-system graphs
    A, b, c_ = irkmg.irkmg_radau_iia(2)
    o = irkmg.irkmg_default_options()
    o.nlevels = 3
    o.patch_form = 0
    dense = irkmg.irkmg_setup(*synth.square_mesh(2), A, b, c_, 1 / 8, 1.0, o)
    try:
        mixed = irkmg.Batch(ctxs[:2] + [dense])
        assert not mixed.persistent
        mixed.close()
    finally:
        dense.close()
        for c in ctxs:
            c.close()

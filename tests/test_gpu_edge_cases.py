"""Degenerate and boundary cases of the method, against the oracle:
  * one stage (Radau IIA(1), backward Euler): the decoupled plan has a single
    real block and no complex pair (the paired kernel does not apply);
  * a zero right-hand side: FGMRES stops before its first iteration at k = 0;
  * the smallest hierarchies: one level is rejected; a 1 x 1 coarsest mesh
    (rank-deficient bordered coarse system) is reported singular; two levels
    from 2 x 2 match the oracle;
  * extreme time steps (dt = 1e-5: mass-dominated; dt = 4: stiffness-dominated);
  * the fixed-point option on 3D patches (196 DoFs per stage, above its
    63-row bound): the FP64 decoupled kernel runs instead, same results.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu


def _ctx(irkmg, s, dt, n0, nl, form=1, fixed=1, dim=2, **kw):
    A, b, c = irkmg.irkmg_radau_iia(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = nl
    o.patch_form = form
    o.patch_fixed = fixed
    o.rtol = 1e-10
    o.maxit = 200
    if dim == 3:
        o.cheb_lo, o.cheb_hi = 2.0, 17.0
    for k, v in kw.items():
        setattr(o, k, v)
    mesh = synth.square_mesh(n0) if dim == 2 else synth.cube_mesh(n0)
    return irkmg.irkmg_setup(*mesh, A, b, c, dt, 1.0, o)


def _oracle(s, dt, n0, nl, dim=2):
    from oracle import mg, tableau
    A, _, _ = tableau.radau_iia(s)
    mesh = synth.square_mesh(n0) if dim == 2 else synth.cube_mesh(n0)
    cheb = (2.0, 8.0) if dim == 2 else (2.0, 17.0)
    return mg.Hierarchy(*mesh, nl, A, dt, cheb=cheb)


@pytest.mark.parametrize("form,fixed", [(0, 0), (1, 0), (1, 1)], ids=["dense", "decoupled", "fixed"])
def test_one_stage(form, fixed):
    irkmg = need_gpu()
    n0, nl, dt = 2, 3, 1 / 16
    H = _oracle(1, dt, n0, nl)
    ctx = _ctx(irkmg, 1, dt, n0, nl, form=form, fixed=fixed)
    try:
        for l in range(1, nl):
            if fixed:
                assert ctx.levels[l]["apply_kernel"] in (8, 9)   # no complex pair: no kernel 10
            L = H.levels[l]
            r = synth.random_vector(900 + l, L.N)
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
            assert rel(host(c), L.vanka.correction(r)) < 1e-12
        r = synth.random_vector(950, H.finest.N)
        z = dev(np.zeros(H.finest.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
    finally:
        ctx.close()


def test_zero_right_hand_side():
    irkmg = need_gpu()
    ctx = _ctx(irkmg, 3, 1 / 64, 2, 3)
    try:
        N = ctx.finest["N"]
        k = dev(np.zeros(N))
        st = irkmg.irkmg_solve(ctx, dev(np.zeros(N)), k)
        assert st["status"] == 0 and st["iters"] == 0
        assert not np.any(host(k))
    finally:
        ctx.close()


def test_smallest_hierarchies():
    """One level is rejected (IRKMG_EINVAL: the V-cycle needs a relaxed
    level).  A 1 x 1 coarsest mesh has a single free velocity node and four
    pressures: its bordered coarse system is rank-deficient (the P2-P1 pair
    on one square is not inf-sup stable), which the oracle confirms, and set-up
    reports IRKMG_ESINGULAR.  The smallest stable case, two levels from 2 x 2:
    V-cycle and FGMRES solution against the oracle."""
    irkmg = need_gpu()
    import scipy.sparse as sp
    from oracle import fgmres
    with pytest.raises(irkmg.IrkmgError) as e:
        _ctx(irkmg, 2, 1 / 8, 4, 1)
    assert e.value.status == irkmg.IRKMG_EINVAL
    s, dt = 2, 1 / 8
    H1 = _oracle(s, dt, 1, 2)
    Lc = H1.levels[0]
    Nm = np.zeros((Lc.N, s))
    for t in range(s):
        Nm[t * Lc.m + 2 * Lc.mesh.nf:(t + 1) * Lc.m, t] = 1.0
    Jb = sp.bmat([[Lc.J, sp.csr_matrix(Nm)], [sp.csr_matrix(Nm.T), None]]).toarray()
    assert np.linalg.matrix_rank(Jb) < Jb.shape[0]
    with pytest.raises(irkmg.IrkmgError) as e:
        _ctx(irkmg, s, dt, 1, 2)
    assert e.value.status == irkmg.IRKMG_ESINGULAR
    n0, nl = 2, 2
    H = _oracle(s, dt, n0, nl)
    ctx = _ctx(irkmg, s, dt, n0, nl)
    try:
        r = synth.random_vector(951, H.finest.N)
        z = dev(np.zeros(H.finest.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-12
        F = H.project_pressure(synth.random_vector(955, H.finest.N))
        x_ref, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
        k = dev(np.zeros(H.finest.N))
        st = irkmg.irkmg_solve(ctx, dev(F), k)
        assert st["status"] == 0 and abs(st["iters"] - its) <= 1
        assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", [1e-5, 4.0], ids=["dt_small", "dt_large"])
def test_extreme_time_steps(dt):
    irkmg = need_gpu()
    from oracle import fgmres
    n0, nl, s = 2, 3, 3
    H = _oracle(s, dt, n0, nl)
    ctx = _ctx(irkmg, s, dt, n0, nl)
    try:
        r = synth.random_vector(952, H.finest.N)
        z = dev(np.zeros(H.finest.N))
        irkmg.irkmg_vcycle(ctx, dev(r), z)
        assert rel(host(z), H.vcycle(r)) < 1e-11
        F = synth.random_vector(953, H.finest.N)
        F = H.project_pressure(F)
        x_ref, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
        k = dev(np.zeros(H.finest.N))
        st = irkmg.irkmg_solve(ctx, dev(F), k)
        assert st["status"] == 0 and abs(st["iters"] - its) <= 1
        assert rel(H.project_pressure(host(k)), H.project_pressure(x_ref)) < 1e-8
    finally:
        ctx.close()


def test_fixed_option_on_3d_patches_falls_back_to_fp64():
    irkmg = need_gpu()
    n0, nl, s, dt = 2, 2, 2, 1 / 16
    H = _oracle(s, dt, n0, nl, dim=3)
    ctx = _ctx(irkmg, s, dt, n0, nl, fixed=1, dim=3)
    try:
        assert ctx.finest["apply_kernel"] not in (8, 9, 10)
        L = H.finest
        r = synth.random_vector(954, L.N)
        c = dev(np.zeros(L.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c)
        assert rel(host(c), L.vanka.correction(r)) < 1e-11
    finally:
        ctx.close()

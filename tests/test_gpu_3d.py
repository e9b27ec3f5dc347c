"""GPU parity in 3D (Taylor-Hood P2-P1 on Kuhn tetrahedra, Bey refinement,
s = 2, patches of up to 392 DoFs factored by blocked LU on the GPU): every step
against the oracle through the C ABI.  Smoother: Chebyshev on [2, 17] (the
3D spectrum of the Vanka-preconditioned operator reaches ~16.7)."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

CASES = [(2, 2, 2, 1 / 16), (2, 3, 2, 1 / 16)]


def _ctx(irkmg, n0, nl, s, dt, precision=64, **kw):
    A, b, c = irkmg.irkmg_radau_iia(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = nl
    o.cheb_lo, o.cheb_hi = 2.0, 17.0
    o.patch_precision = precision
    o.maxit = 400
    for k, v in kw.items():
        setattr(o, k, v)
    return irkmg.irkmg_setup(*synth.cube_mesh(n0), A, b, c, dt, 1.0, o)


_H = {}


def _oracle(n0, nl, s, dt):
    key = (n0, nl, s, dt)
    if key not in _H:
        from oracle import mg, tableau
        A, _, _ = tableau.radau_iia(s)
        _H[key] = mg.Hierarchy(*synth.cube_mesh(n0), nl, A, dt, cheb=(2.0, 17.0))
    return _H[key]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "n0=%d,L=%d" % c[:2])
def pair3(request):
    irkmg = need_gpu()
    n0, nl, s, dt = request.param
    ctx = _ctx(irkmg, n0, nl, s, dt)
    yield irkmg, ctx, _oracle(n0, nl, s, dt)
    ctx.close()


def test_3d_sizes_patches_colours(pair3):
    irkmg, ctx, H = pair3
    from oracle import vanka
    for l, L in enumerate(H.levels):
        info = ctx.levels[l]
        assert info["dim"] == 3
        assert (info["nv"], info["nf"], info["np2"], info["N"]) == (L.mesh.nv, L.mesh.nf, L.mesh.np2, L.N)
        np.testing.assert_array_equal(irkmg.irkmg_free_nodes(ctx, l), L.mesh.free_p2)
        np.testing.assert_array_equal(irkmg.irkmg_p2_coords(ctx, l), L.mesh.p2_coords)
        if l == 0:
            continue
        ptr, nodes = irkmg.irkmg_patch_map(ctx, l)
        ref = vanka.patch_nodes(L.mesh)
        assert np.array_equal(nodes, np.concatenate(ref))
        np.testing.assert_array_equal(irkmg.irkmg_colouring(ctx, l), vanka.distance2_colouring(L.mesh))
        assert info["max_patch_dofs"] == max(len(d) for d in L.dofs)
        assert info["apply_kernel"] == (3 if info["max_patch_dofs"] > 160 else info["apply_kernel"])


def test_3d_operator_transfers(pair3):
    irkmg, ctx, H = pair3
    for l, L in enumerate(H.levels):
        x = synth.random_vector(700 + l, L.N)
        y = dev(np.zeros(L.N))
        irkmg.irkmg_apply(ctx, dev(x), y, level=l)
        assert rel(host(y), L.J @ x) < 1e-13
        if l > 0:
            xc = synth.random_vector(710 + l, H.levels[l - 1].N)
            yc, yf = dev(np.zeros(H.levels[l - 1].N)), dev(np.zeros(L.N))
            irkmg.irkmg_restrict(ctx, dev(x), yc, level=l)
            irkmg.irkmg_prolong(ctx, dev(xc), yf, level=l)
            assert rel(host(yc), L.P.T @ x) < 1e-14
            assert rel(host(yf), L.P @ xc) < 1e-14


def test_3d_blocked_lu_vanka_smoother_vcycle(pair3):
    irkmg, ctx, H = pair3
    for l in range(1, len(H.levels)):
        L = H.levels[l]
        r = synth.random_vector(720 + l, L.N)
        c = dev(np.zeros(L.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
        assert rel(host(c), L.vanka.correction(r)) < 1e-11
        F = synth.random_vector(730 + l, L.N)
        x0 = 0.1 * synth.random_vector(740 + l, L.N)
        x = dev(x0)
        irkmg.irkmg_smooth(ctx, dev(F), x, 2, level=l)
        assert rel(host(x), L.vanka.chebyshev(L.J, F, x0, 2, 2.0, 17.0)) < 1e-11
    r = synth.random_vector(750, H.finest.N)
    z = dev(np.zeros(H.finest.N))
    irkmg.irkmg_vcycle(ctx, dev(r), z)
    assert rel(host(z), H.vcycle(r)) < 1e-11


def test_3d_solve_and_fp32_form(pair3):
    irkmg, ctx, H = pair3
    from oracle import fgmres, stage
    L = H.finest
    m = L.mesh
    X = m.p2_coords
    f = np.stack([np.stack(synth.mms3_forcing(*X.T))] * H.s)
    un = np.concatenate(synth.mms3_velocity(*m.p2_coords[m.free_p2].T))
    pn = synth.mms3_pressure(*m.coords.T)
    pn = pn - pn.mean()
    F_ref = stage.stage_rhs(L.ops, un, pn, f)
    F = dev(np.zeros(L.N))
    irkmg.irkmg_stage_rhs(ctx, dev(un), dev(pn), dev(f.ravel()), F)
    assert rel(host(F), F_ref) < 1e-12
    # at the benchmark tolerance 1e-10: same iteration count as the oracle +-2
    k = dev(np.zeros(L.N))
    st = irkmg.irkmg_solve(ctx, dev(F_ref), k)
    assert st["status"] == 0
    _, its_ref, _ = fgmres.fgmres(L.J, F_ref, H.vcycle, rtol=1e-10, project=H.project_pressure,
                                  maxit=400)
    assert abs(st["iters"] - its_ref) <= 2
    # solved to 1e-13 on both sides, the solutions agree to 1e-8: FP64 patches
    # and FP32 patch factors and applies inside the FP64 FGMRES, both against
    # the oracle
    x_ref, _, _ = fgmres.fgmres(L.J, F_ref, H.vcycle, rtol=1e-13, project=H.project_pressure,
                                maxit=800)
    ref = H.project_pressure(x_ref)
    nl = len(H.levels)
    for prec in (64, 32):
        c = _ctx(irkmg, 2, nl, H.s, H.dt, precision=prec, rtol=1e-13, maxit=800)
        try:
            kk = dev(np.zeros(L.N))
            stp = irkmg.irkmg_solve(c, dev(F_ref), kk)
            assert stp["status"] == 0 and stp["rfinal"] <= 1e-13 * np.linalg.norm(F_ref), (prec, stp)
            assert rel(H.project_pressure(host(kk)), ref) < 1e-8, prec
        finally:
            c.close()


def test_3d_unsupported_forms_say_so(pair3):
    irkmg, ctx, H = pair3
    G = dev(H.project_pressure(synth.random_vector(760, ctx.N())))
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_adjoint_solve(ctx, G, dev(np.zeros(ctx.N())))
    assert e.value.status == irkmg.IRKMG_ENOTIMPL


def test_3d_fp32_lu_on_tensor_cores_matches_cuda_cores():
    """FP32 patch LU with tcgen05 trailing updates (3xTF32) against the same
    LU on the CUDA cores and against the oracle's FP64 patches: one Vanka
    correction on the 4x4x4 level (patches up to 392 DoFs, 12 panels of 32).
    Both FP32 variants carry the FP32 rounding of their factors, amplified by
    the patch condition numbers; the split products keep the tensor-core
    variant as close to the oracle as the CUDA-core one."""
    irkmg = need_gpu()
    n0, nl, s, dt = 2, 2, 2, 1 / 16
    H = _oracle(n0, nl, s, dt)
    L = H.finest
    r = synth.random_vector(4242, L.N)
    ref = L.vanka.correction(r)
    out = {}
    for tc in (1, 0):
        ctx = _ctx(irkmg, n0, nl, s, dt, precision=32, patch_lu_tc=tc)
        try:
            assert ctx.finest["apply_kernel"] == 3
            c = dev(np.zeros(L.N))
            irkmg.irkmg_vanka_correction(ctx, dev(r), c)
            out[tc] = host(c)
        finally:
            ctx.close()
    e_tc, e_cc = rel(out[1], ref), rel(out[0], ref)
    assert e_cc < 1e-4
    assert e_tc < 2 * e_cc + 1e-6
    assert rel(out[1], out[0]) < 2e-4

"""GPU parity: every step of the CUDA path against the oracle on the same
seeded inputs, through the C ABI.

Bars: patch maps and colourings bit-exact; operator, transfers and stage
right-hand side to rounding (1e-13 relative); one Vanka correction, one
smoothing pass and one V-cycle to 1e-12 relative (the oracle solves each patch
by LU, the GPU applies a stored inverse, so they differ by rounding times the
patch condition number); final FGMRES solutions to 1e-8 relative in the l2
norm."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, gpu_context, host, need_gpu, oracle_hierarchy, rel

pytestmark = pytest.mark.gpu

CASES = [  # (n0, nlevels, s, dt): 8x8 from 2x2 (3 levels), 32x32 (5 levels), s = 3
    (2, 3, 2, 1 / 8),
    (2, 5, 2, 1 / 8),
    (2, 4, 3, 1 / 64),
    (3, 3, 3, 0.05),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "n0=%d,L=%d,s=%d" % c[:3])
def pair(request):
    irkmg = need_gpu()
    n0, nl, s, dt = request.param
    ctx = gpu_context(irkmg, n0, nl, s, dt)
    H = oracle_hierarchy(n0, nl, s, dt)
    yield irkmg, ctx, H
    ctx.close()


def test_sizes_numbering_patches_colours(pair):
    irkmg, ctx, H = pair
    for l, L in enumerate(H.levels):
        info = ctx.levels[l]
        assert (info["nv"], info["nf"], info["np2"], info["N"]) == (L.mesh.nv, L.mesh.nf, L.mesh.np2, L.N)
        np.testing.assert_array_equal(irkmg.irkmg_free_nodes(ctx, l), L.mesh.free_p2)
        np.testing.assert_array_equal(irkmg.irkmg_p2_coords(ctx, l), L.mesh.p2_coords)
        if l == 0:
            continue
        from oracle import vanka
        ptr, nodes = irkmg.irkmg_patch_map(ctx, l)
        ref = vanka.patch_nodes(L.mesh)
        assert np.array_equal(ptr, np.concatenate([[0], np.cumsum([len(x) for x in ref])]))
        assert np.array_equal(nodes, np.concatenate(ref))
        np.testing.assert_array_equal(irkmg.irkmg_colouring(ctx, l), vanka.distance2_colouring(L.mesh))


def test_operator_and_transpose(pair):
    irkmg, ctx, H = pair
    for l, L in enumerate(H.levels):
        x = synth.random_vector(11 + l, L.N)
        y = dev(np.zeros(L.N))
        irkmg.irkmg_apply(ctx, dev(x), y, level=l)
        assert rel(host(y), L.J @ x) < 1e-13
        irkmg.irkmg_apply(ctx, dev(x), y, level=l, transpose=True)
        assert rel(host(y), L.J.T @ x) < 1e-13


def test_transfers(pair):
    irkmg, ctx, H = pair
    for l in range(1, len(H.levels)):
        Lf, Lc = H.levels[l], H.levels[l - 1]
        xf = synth.random_vector(21 + l, Lf.N)
        xc = synth.random_vector(31 + l, Lc.N)
        yc, yf = dev(np.zeros(Lc.N)), dev(np.zeros(Lf.N))
        irkmg.irkmg_restrict(ctx, dev(xf), yc, level=l)
        irkmg.irkmg_prolong(ctx, dev(xc), yf, level=l)
        assert rel(host(yc), Lf.P.T @ xf) < 1e-14
        assert rel(host(yf), Lf.P @ xc) < 1e-14


def test_vanka_correction_and_smoother(pair):
    irkmg, ctx, H = pair
    for l in range(1, len(H.levels)):
        L = H.levels[l]
        r = synth.random_vector(41 + l, L.N)
        c = dev(np.zeros(L.N))
        irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l)
        assert rel(host(c), L.vanka.correction(r)) < 1e-12
        # transposed patches: (R J R^T)^{-T} = R J^T R^T inverted
        irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=l, transpose=True)
        ref_t = np.zeros(L.N)
        for idx, (lu, piv) in zip(L.vanka.dofs, L.vanka.lu):
            import scipy.linalg as sla
            ref_t[idx] += sla.lu_solve((lu, piv), r[idx], trans=1)
        assert rel(host(c), ref_t) < 1e-12
        F = synth.random_vector(51 + l, L.N)
        x0 = 0.1 * synth.random_vector(61 + l, L.N)
        x = dev(x0)
        irkmg.irkmg_smooth(ctx, dev(F), x, 2, level=l)
        assert rel(host(x), L.vanka.chebyshev(L.J, F, x0, 2, 2.0, 8.0)) < 1e-12


def test_coarse_solve(pair):
    irkmg, ctx, H = pair
    L = H.levels[0]
    r = H.project_pressure(synth.random_vector(71, L.N), level=0)
    x = dev(np.zeros(L.N))
    irkmg.irkmg_coarse_solve(ctx, dev(r), x)
    assert rel(host(x), H.coarse_solve(r)) < 1e-11


def test_vcycle(pair):
    irkmg, ctx, H = pair
    r = synth.random_vector(81, H.finest.N)
    z = dev(np.zeros(H.finest.N))
    irkmg.irkmg_vcycle(ctx, dev(r), z)
    assert rel(host(z), H.vcycle(r)) < 1e-12


def test_stage_rhs_solve_advance(pair):
    irkmg, ctx, H = pair
    from oracle import fgmres, problem, stage, tableau
    _, bw, c = tableau.radau_iia(H.s)
    F_ref, un, pn = problem.mms_rhs(H, c)
    f = problem.forcing(H.finest.mesh, c, 0.0, H.dt)
    F = dev(np.zeros(H.finest.N))
    irkmg.irkmg_stage_rhs(ctx, dev(un), dev(pn), dev(f.ravel()), F)
    # for a steady manufactured solution M f - K u^n - B p^n cancels down to the
    # discretisation residual, so rounding is bounded componentwise by the
    # absolute terms |M||f| + |K||u| + |B||p| (times a small multiple of eps)
    ops = H.finest.ops
    nf = H.finest.mesh.nf
    a = lambda S: abs(S)
    bound_p = a(ops["B"]).T @ abs(un)
    bound = np.concatenate([
        np.concatenate([np.concatenate([a(ops["Mall"]) @ abs(f[t, d]) + a(ops["K"]) @ abs(un[d * nf:(d + 1) * nf])
                                        for d in range(2)]) + a(ops["B"]) @ abs(pn), bound_p])
        for t in range(H.s)])
    assert np.all(np.abs(host(F) - F_ref) <= 64 * np.finfo(float).eps * bound)
    k = dev(np.zeros(H.finest.N))
    st = irkmg.irkmg_solve(ctx, F, k)
    assert st["status"] == 0 and st["rfinal"] <= 1e-10 * np.linalg.norm(F_ref)
    x_ref, its_ref, _ = fgmres.fgmres(H.finest.J, F_ref, H.vcycle, rtol=1e-10,
                                      project=H.project_pressure)
    kk = host(k)
    assert rel(H.project_pressure(kk), H.project_pressure(x_ref)) < 1e-8
    assert abs(st["iters"] - its_ref) <= 1
    u, p = dev(un), dev(pn)
    irkmg.irkmg_advance(ctx, k, u, p)
    u_ref, p_ref = stage.advance(kk, un, pn, bw, H.dt)
    assert rel(host(u), u_ref) < 1e-14 and rel(host(p), p_ref) < 1e-14


def test_adjoint_solve(pair):
    irkmg, ctx, H = pair
    L = H.finest
    G = H.project_pressure(synth.random_vector(91, L.N))
    lam = dev(np.zeros(L.N))
    st = irkmg.irkmg_adjoint_solve(ctx, dev(G), lam)
    assert st["status"] == 0
    res = G - L.J.T @ host(lam)
    assert np.linalg.norm(res) <= 1.01e-10 * np.linalg.norm(G)

"""Parity at the benchmarked 3D size: Stokes on 32³ cubes × 6 Kuhn tetrahedra
from 4³ (4 levels, Bey refinement), Radau IIA(2), dt = 1/16, N = 1,572,156,
with bench.py's 3D options (Chebyshev [2, 17] V(2,2), FGMRES(30), rtol 1e-10,
decoupled complex-layout FP32 patches of up to 392 DoFs factored by the
blocked LU with tensor-core trailing updates) and its autotuned launch
configuration.  As in tests/test_gpu_fullsize.py, the integer work is checked
in full against oracle.mesh / oracle.vanka and the floating-point outputs on
samples against oracle/local.py:
  * numbering, P2 coordinates, every patch map and the colouring, bit-exact;
  * J x and J^T x at sampled rows (FP64 operator);
  * the finest-level Vanka correction at sampled DoFs: FP32 patch inverses,
    so the bar is an FP32 one, 1e-6 entry-wise (measured 6.2e-8, about the
    FP32 unit roundoff);
  * a full FGMRES solve (FP64 outer iteration): sampled rows of F - J k
    within the solver's bound.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

N0, NL, S, DT = 4, 4, 2, 1 / 16


@pytest.fixture(scope="module")
def full3():
    irkmg = need_gpu()
    from oracle import local, mesh, tableau
    A, b, c = irkmg.irkmg_radau_iia(S)
    o = irkmg.irkmg_default_options()
    o.nlevels = NL
    o.patch_form = 1
    o.patch_precision = 32
    o.cheb_lo, o.cheb_hi = 2.0, 17.0
    o.rtol = 1e-10
    o.maxit = 300
    ctx = irkmg.irkmg_setup(*synth.cube_mesh(N0), A, b, c, DT, 1.0, o)
    H = mesh.hierarchy(*synth.cube_mesh(N0), NL)
    Ao, _, _ = tableau.radau_iia(S)
    yield irkmg, ctx, H[-1], local.LocalStage(H[-1], Ao, DT), local.LocalStage(H[-1], Ao.T, DT)
    ctx.close()


def _samples(L, count, seed, pressure_only=False):
    """Random DoFs, the corner pressures and velocity DoFs next to the
    boundary, every stage (pressure DoFs only: each sits in one patch)."""
    rng = np.random.default_rng(seed)
    m, nf, nv, d = L.m, L.nf, L.nv, L.d
    msh = L.mesh
    cv = msh.coords[:nv]
    corners = np.nonzero(np.all(np.isclose(cv, 0.0) | np.isclose(cv, 1.0), axis=1))[0]
    assert corners.size == 8
    picks = []
    for t in range(L.s):
        picks += [t * m + d * nf + int(v) for v in corners]
        picks += [t * m + d * nf + int(v) for v in rng.choice(nv, count // (2 * L.s), replace=False)]
    if not pressure_only:
        xy = msh.p2_coords[msh.free_p2]
        near = np.nonzero((np.minimum(xy, 1.0 - xy) < 1.5 / 32).any(axis=1))[0]
        picks += [int(i) for i in rng.choice(L.N, count, replace=False)]
        for t in range(L.s):
            picks += [t * m + c * nf + int(f) for c in range(d) for f in rng.choice(near, 3, replace=False)]
    return np.array(sorted(set(picks)))


def test_3d_numbering_patch_maps_and_colouring_bit_exact(full3):
    irkmg, ctx, msh, L, _ = full3
    from oracle import vanka
    fin = ctx.nlevels - 1
    info = ctx.levels[fin]
    assert (info["nv"], info["nf"], info["np2"], info["N"]) == (msh.nv, msh.nf, msh.np2, L.N)
    assert L.N == 1572156
    np.testing.assert_array_equal(irkmg.irkmg_free_nodes(ctx, fin), msh.free_p2)
    np.testing.assert_array_equal(irkmg.irkmg_p2_coords(ctx, fin), msh.p2_coords)
    ptr, nodes = irkmg.irkmg_patch_map(ctx, fin)
    ref = vanka.patch_nodes(msh)
    assert np.array_equal(ptr, np.concatenate([[0], np.cumsum([len(x) for x in ref])]))
    assert np.array_equal(nodes, np.concatenate(ref))
    np.testing.assert_array_equal(irkmg.irkmg_colouring(ctx, fin), vanka.distance2_colouring(msh))


def test_3d_operator_rows_at_full_size(full3):
    irkmg, ctx, msh, L, LT = full3
    x = synth.random_vector(601, L.N)
    rows = _samples(L, 400, 21)
    y = dev(np.zeros(L.N))
    for tr, Lx in ((False, L), (True, LT)):
        irkmg.irkmg_apply(ctx, dev(x), y, transpose=tr)
        got = host(y)[rows]
        ref, mag = Lx.apply_rows(rows, x)
        assert np.all(np.abs(got - ref) <= 1e-13 * mag + 1e-300), (tr, np.max(np.abs(got - ref) / mag))


def test_3d_vanka_correction_at_full_size(full3):
    irkmg, ctx, msh, L, _ = full3
    fin = ctx.nlevels - 1
    r = synth.random_vector(602, L.N)
    c = dev(np.zeros(L.N))
    irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=fin)
    got_all = host(c)
    rows = _samples(L, 24, 22, pressure_only=True)
    # plus a few velocity DoFs (each in up to 15 patches of 392 DoFs)
    rng = np.random.default_rng(24)
    vel = rng.choice(L.d * L.nf, 4, replace=False)
    rows = np.array(sorted(set(rows.tolist()) | {int(t * L.m + i) for t in range(L.s) for i in vel[:2]}))
    ref = L.vanka_entries(rows, r)
    got = got_all[rows]
    scale = np.abs(ref).max()
    err = np.abs(got - ref) / (np.abs(ref) + scale)
    print("3D FP32-patch Vanka correction, max entry-wise error %.3g over %d DoFs" % (err.max(), rows.size))
    assert np.all(err <= 1e-6), err.max()


def test_3d_solve_residual_rows_at_full_size(full3):
    irkmg, ctx, msh, L, _ = full3
    F = synth.random_vector(603, L.N)
    for t in range(L.s):   # compatible: zero pressure mean per stage
        p = slice(t * L.m + L.d * L.nf, (t + 1) * L.m)
        F[p] -= F[p].mean()
    k = dev(np.zeros(L.N))
    st = irkmg.irkmg_solve(ctx, dev(F), k)
    assert st["status"] == 0
    kh = host(k)
    rows = _samples(L, 400, 25)
    Jk, mag = L.apply_rows(rows, kh)
    res = F[rows] - Jk
    bound = 1e-10 * np.linalg.norm(F) + 1e-13 * mag
    assert np.all(np.abs(res) <= bound), np.max(np.abs(res) / bound)

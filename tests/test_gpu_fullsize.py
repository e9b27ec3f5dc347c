"""Parity at the benchmarked size: 2D Stokes, Radau IIA(3), dt = 1/64, 512 x 512
from 8 x 8 (7 levels, N = 7,068,681), with bench.py's options (Chebyshev
[2, 8] V(2,2), FGMRES(30), rtol 1e-10, decoupled complex-layout patches with
fixed-point mat-vecs) and its launch configuration on the finest level (the
paired fixed-point kernel, shape 7, one launch per sweep).

The oracle cannot assemble J at this size, so outputs are checked one by one
on samples against oracle/local.py (rows of J and single-patch systems from
the element matrices around the sampled nodes), and the integer work
(numbering, patch maps, colouring) in full against oracle.mesh / oracle.vanka:
  * numbering, P2 coordinates, every patch map and the colouring, bit-exact;
  * J x and J^T x at 600 sampled rows (both velocity components, the
    pressure, every stage, the corner vertices and nodes next to the boundary);
  * the finest-level Vanka correction with J and J^T patches at sampled DoFs;
  * a full FGMRES solve: sampled rows of F - J k within the solver's bound.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

N0, NL, S, DT = 8, 7, 3, 1 / 64


@pytest.fixture(scope="module")
def full():
    irkmg = need_gpu()
    from oracle import local, mesh, tableau
    A, b, c = irkmg.irkmg_radau_iia(S)
    o = irkmg.irkmg_default_options()
    o.nlevels = NL
    o.patch_form = 1
    o.patch_fixed = 1
    o.rtol = 1e-10
    o.maxit = 300
    ctx = irkmg.irkmg_setup(*synth.square_mesh(N0), A, b, c, DT, 1.0, o)
    H = mesh.hierarchy(*synth.square_mesh(N0), NL)
    Ao, _, _ = tableau.radau_iia(S)
    L = local.LocalStage(H[-1], Ao, DT)
    LT = local.LocalStage(H[-1], Ao.T, DT)   # J^T: M and St symmetric for Stokes
    yield irkmg, ctx, H[-1], L, LT
    ctx.close()


def _samples(L, count, seed):
    """Random DoFs of every kind plus the corner pressures and velocity DoFs
    of nodes next to the boundary (ragged patches), every stage."""
    rng = np.random.default_rng(seed)
    m, nf, nv = L.m, L.nf, L.nv
    msh = L.mesh
    xy = msh.p2_coords[msh.free_p2]
    h = 1.0 / 512
    near = np.nonzero((np.minimum(xy, 1.0 - xy) < 1.5 * h).any(axis=1))[0]
    cv = msh.coords[:nv]
    corners = np.nonzero(np.all(np.isclose(cv, 0.0) | np.isclose(cv, 1.0), axis=1))[0]
    assert corners.size == 4
    picks = list(rng.choice(L.N, size=count, replace=False))
    for t in range(L.s):
        picks += [t * m + 2 * nf + v for v in corners]
        picks += [t * m + c * nf + f for c in range(2) for f in rng.choice(near, 4, replace=False)]
    return np.array(sorted(set(int(i) for i in picks)))


def test_numbering_patch_maps_and_colouring_bit_exact(full):
    irkmg, ctx, msh, L, _ = full
    from oracle import vanka
    fin = ctx.nlevels - 1
    info = ctx.levels[fin]
    assert (info["nv"], info["nf"], info["np2"], info["N"]) == (msh.nv, msh.nf, msh.np2, L.N)
    assert L.N == 7068681
    np.testing.assert_array_equal(irkmg.irkmg_free_nodes(ctx, fin), msh.free_p2)
    np.testing.assert_array_equal(irkmg.irkmg_p2_coords(ctx, fin), msh.p2_coords)
    ptr, nodes = irkmg.irkmg_patch_map(ctx, fin)
    ref = vanka.patch_nodes(msh)
    assert np.array_equal(ptr, np.concatenate([[0], np.cumsum([len(x) for x in ref])]))
    assert np.array_equal(nodes, np.concatenate(ref))
    np.testing.assert_array_equal(irkmg.irkmg_colouring(ctx, fin), vanka.distance2_colouring(msh))


def test_operator_rows_at_full_size(full):
    irkmg, ctx, msh, L, LT = full
    x = synth.random_vector(501, L.N)
    rows = _samples(L, 600, 11)
    y = dev(np.zeros(L.N))
    for tr, Lx in ((False, L), (True, LT)):
        irkmg.irkmg_apply(ctx, dev(x), y, transpose=tr)
        got = host(y)[rows]
        ref, mag = Lx.apply_rows(rows, x)
        # entry by entry: both sides sum the same products in FP64
        assert np.all(np.abs(got - ref) <= 1e-13 * mag + 1e-300), (tr, np.max(np.abs(got - ref) / mag))


@pytest.mark.parametrize("transpose", [False, True], ids=["J", "JT"])
def test_vanka_correction_at_full_size(full, transpose):
    irkmg, ctx, msh, L, _ = full
    fin = ctx.nlevels - 1
    # the benchmarked launch on the finest level: paired fixed-point kernel,
    # shape 7, one launch over all patches plus the per-DoF sum
    irkmg.irkmg_level_set_apply(ctx, fin, 7, 1)
    assert ctx.levels[fin]["apply_kernel"] == 10
    r = synth.random_vector(502, L.N)
    c = dev(np.zeros(L.N))
    irkmg.irkmg_vanka_correction(ctx, dev(r), c, level=fin, transpose=transpose)
    got_all = host(c)
    rows = _samples(L, 40, 12)
    ref = L.vanka_entries(rows, r, transpose=transpose)
    got = got_all[rows]
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 1e-11 * (np.abs(ref) + scale)), \
        np.max(np.abs(got - ref) / (np.abs(ref) + scale))


def test_solve_residual_rows_at_full_size(full):
    irkmg, ctx, msh, L, _ = full
    F = synth.random_vector(503, L.N)
    for t in range(L.s):   # compatible: zero pressure mean per stage (the null space of J^T)
        p = slice(t * L.m + 2 * L.nf, (t + 1) * L.m)
        F[p] -= F[p].mean()
    k = dev(np.zeros(L.N))
    st = irkmg.irkmg_solve(ctx, dev(F), k)
    assert st["status"] == 0
    kh = host(k)
    rows = _samples(L, 400, 13)
    Jk, mag = L.apply_rows(rows, kh)
    res = F[rows] - Jk
    # every entry of r = F - J k is bounded by ||r|| <= 1e-10 ||F|| (the solver's
    # stopping rule), up to the rounding of the oracle's own row sums
    bound = 1e-10 * np.linalg.norm(F) + 1e-13 * mag
    assert np.all(np.abs(res) <= bound), np.max(np.abs(res) / bound)

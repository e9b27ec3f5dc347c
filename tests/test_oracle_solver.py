"""Pins for the oracle's V-cycle + FGMRES stage solve (Section 4): it must
reach the solution of a sparse direct solve of the bordered stage system, and
its iteration counts must stay flat under refinement (Section 5.1, Table 1)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fgmres, mg, problem, tableau


def _direct(H, F):
    L = H.finest
    Nm = np.zeros((L.N, H.s))
    for t in range(H.s):
        Nm[t * L.m + 2 * L.mesh.nf:(t + 1) * L.m, t] = 1.0
    Jb = sp.bmat([[L.J, sp.csr_matrix(Nm)], [sp.csr_matrix(Nm.T), None]], format="csc")
    return spla.spsolve(Jb, np.concatenate([F, np.zeros(H.s)]))[: L.N]


@pytest.mark.parametrize("s,dt", [(2, 1 / 8), (3, 1 / 64)])
def test_fgmres_vcycle_matches_direct_solve(s, dt):
    """cfg-1 shape: 8x8 finest mesh from a 2x2 coarsest, 3 levels."""
    A, b, c = tableau.radau_iia(s)
    H = mg.Hierarchy(*synth.square_mesh(2), 3, A, dt)
    F, _, _ = problem.mms_rhs(H, c)
    x, its, hist = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
    ref = H.project_pressure(_direct(H, F))
    assert hist[-1] <= 1e-10 * np.linalg.norm(F)
    assert np.linalg.norm(H.project_pressure(x) - ref) <= 1e-8 * np.linalg.norm(ref)
    assert its < 30


def test_richardson_omega_half_is_not_contractive():
    """The plain additive step damped by 0.5 amplifies the top of the spectrum
    (largest eigenvalue near 8, Section 5.1), so as a stationary iteration it
    diverges; the Chebyshev smoother on [2, 8] does not."""
    A, b, c = tableau.radau_iia(2)
    F = None
    for smoother, grows in (("richardson", True), ("chebyshev", False)):
        H = mg.Hierarchy(*synth.square_mesh(2), 2, A, 1 / 8, smoother=smoother)
        L = H.finest
        if F is None:
            F = H.project_pressure(synth.random_vector(1, L.N))
        k = np.zeros(L.N)
        for _ in range(6):
            k = k + H.vcycle(F - L.J @ k)
        ratio = np.linalg.norm(F - L.J @ k) / np.linalg.norm(F)
        assert (ratio > 1.0) == grows, (smoother, ratio)


@pytest.mark.slow
@pytest.mark.parametrize("s,dt", [(2, 1 / 8), (3, 1 / 64)])
def test_iterations_flat_under_refinement(s, dt):
    """FGMRES iterations for 4x4 ... 32x32 finest meshes (2 .. 5 levels from
    2x2) stay within 2 of the middle of their range (max - min <= 4), and one
    refinement adds at most 2 (Section 5.1, Table 1: nearly constant counts;
    the paper's own fixed-dt Radau IIA rows grow by 5 to 8 over two
    refinements, so this bar is stricter than the paper's behaviour)."""
    A, b, c = tableau.radau_iia(s)
    its = []
    for nl in (2, 3, 4, 5):
        H = mg.Hierarchy(*synth.square_mesh(2), nl, A, dt)
        F, _, _ = problem.mms_rhs(H, c)
        _, k, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
        its.append(k)
    assert max(its) - min(its) <= 4, its
    assert all(b_ - a_ <= 2 for a_, b_ in zip(its, its[1:])), its

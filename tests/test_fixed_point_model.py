"""Model check of the fixed-point patch apply on real patch matrices (CPU).

The library can store the decoupled FP64 patch inverses row by row as 57-bit
fixed point and apply them by exact integer dot products against sources
scaled to 58-bit integers, with one rounding to FP64 (`patch_fixed`).  This
test restates that arithmetic with Python integers (independently of the CUDA
code) and applies it to the stored matrices of an 8x8 level: for Radau IIA(3),
the real-eigenvalue inverse (M̃ + Δtλ K̃)⁻¹ and X, Y, X + Y of the complex
pair's inverse X + iY (Section 3's Kronecker form on the patches of Section
4.2).  Against the exact product (rational arithmetic) it checks, for every
row, the error bound of the representation,
    |y_fx − y| ≤ 2^-57 max_j|M_ij| Σ_j|x_j| + 2^-58 max_j|x_j| Σ_j|M_ij| + 2^-53 |y|,
and that over the level the fixed-point products are at least as accurate
as FP64 mat-vecs of the same matrices."""
import math

import numpy as np
import scipy.linalg as sla  # noqa: F401  (LAPACK through numpy.linalg)

import synth
from oracle import mg, stage, tableau


def exact(M, x):
    """Exact products y_i = Σ_j M_ij x_j as (integer, exponent) pairs."""
    def split(d):
        f, e = math.frexp(d)
        return int(f * 2 ** 53), e - 53
    xs = [split(v) for v in x]
    out = []
    for row in M:
        terms = []
        for a, (mx, ex) in zip(row, xs):
            ma, ea = split(a)
            terms.append((ma * mx, ea + ex))
        e0 = min(e for _, e in terms)
        out.append((sum(m << (e - e0) for m, e in terms), e0))
    return out


def fixed_product(M, x):
    """The fixed-point apply: rows to 57-bit integers with their own power of
    two, the source to 58-bit integers with one power of two, exact integer
    dot products, one correctly rounded conversion to FP64."""
    F = math.frexp(float(np.max(np.abs(x))))[1]
    v = [round(math.ldexp(float(t), 58 - F)) for t in x]          # exact scaling, ties to even
    y = []
    for row in M:
        E = math.frexp(float(np.max(np.abs(row))))[1]
        q = [round(math.ldexp(float(a), 57 - E)) for a in row]
        assert max(map(abs, q)) <= 2 ** 57 and max(map(abs, v)) <= 2 ** 58
        t = sum(qi * vi for qi, vi in zip(q, v))
        assert abs(t) < 2 ** 121
        y.append(math.ldexp(float(t), E + F - 115))              # float(int) rounds to nearest even
    return np.array(y)


def err(y, ex):
    """|y_i − exact_i| as floats (exact rational difference, then rounded)."""
    out = []
    for yi, (m, e) in zip(y, ex):
        f, fe = math.frexp(yi)
        my, ey = int(f * 2 ** 53), fe - 53
        e0 = min(e, ey)
        d = (my << (ey - e0)) - (m << (e - e0))
        out.append(abs(math.ldexp(float(d), e0)))
    return np.array(out)


def test_fixed_point_products_meet_the_bound_and_beat_fp64():
    A = tableau.radau_iia(3)[0]
    dt = 1 / 64
    H = mg.Hierarchy(*synth.square_mesh(2), 3, A, dt)
    L = H.levels[-1]
    Mt, St = stage.single_stage_blocks(L.ops)
    lam = np.linalg.eigvals(A)
    lr = float(lam[np.argmin(np.abs(lam.imag))].real)
    lc = lam[np.argmax(lam.imag)]
    rng = np.random.default_rng(3)
    s, worst_ratio = 3, 0.0
    num_fx = num_64 = den = 0.0
    for idx in L.dofs:
        n = len(idx) // s
        one = idx[:n]
        Mv = Mt[one][:, one].toarray()
        Kv = St[one][:, one].toarray()
        Z = np.linalg.inv(Mv + dt * lc * Kv)
        mats = [np.linalg.inv(Mv + dt * lr * Kv), Z.real + Z.imag, Z.real, Z.imag]
        for Mat in mats:
            # a source with entries spread over three decades, as a smoothed
            # residual may have
            x = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 0, n)
            ex = exact(Mat, x)
            y_fx = fixed_product(Mat, x)
            y_64 = Mat @ x
            e_fx, e_64 = err(y_fx, ex), err(y_64, ex)
            ymag = np.array([abs(math.ldexp(float(m), e)) for m, e in ex])
            bound = (2.0 ** -57 * np.abs(Mat).max(axis=1) * np.abs(x).sum()
                     + 2.0 ** -58 * np.abs(x).max() * np.abs(Mat).sum(axis=1)
                     + 2.0 ** -53 * ymag)
            worst_ratio = max(worst_ratio, float(np.max(e_fx / bound)))
            num_fx += float(e_fx @ e_fx)
            num_64 += float(e_64 @ e_64)
            den += float(ymag @ ymag)
    assert worst_ratio <= 1.0
    rel_fx, rel_64 = math.sqrt(num_fx / den), math.sqrt(num_64 / den)
    assert rel_fx <= rel_64, (rel_fx, rel_64)
    assert rel_fx < 2.0 ** -52

"""CPU checks of the C ABI: the library loads, exports every function that
include/irkmg.h declares, and its host-only entry points behave (no GPU
needed: nothing here launches a kernel or allocates device memory)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def irkmg():
    from paper_2202_07381_gb300 import build, irkmg as m
    if not os.path.exists(build.LIB):
        build.build()
    m.lib()
    return m


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(irkmg_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(irkmg):
    names = declared_functions()
    assert len(names) >= 25
    lib = ct.CDLL(irkmg.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(names) <= set(irkmg._SIGS), set(names) - set(irkmg._SIGS)


@pytest.mark.parametrize("s", [1, 2, 3])
def test_radau_closed_forms_match_oracle(irkmg, s):
    from oracle import tableau
    A, b, c = irkmg.irkmg_radau_iia(s)
    Ao, bo, co = tableau.radau_iia(s)
    np.testing.assert_allclose(A, Ao, atol=2e-15)
    np.testing.assert_allclose(b, bo, atol=2e-15)
    np.testing.assert_allclose(c, co, atol=2e-15)


@pytest.mark.parametrize("fam,s", [("gauss", 2), ("gauss", 3), ("lobatto_iiic", 2), ("lobatto_iiic", 3)])
def test_gauss_lobatto_closed_forms_match_oracle(irkmg, fam, s):
    from oracle import tableau
    A, b, c = getattr(irkmg, "irkmg_" + fam)(s)
    Ao, bo, co = getattr(tableau, fam)(s)
    np.testing.assert_allclose(A, Ao, atol=3e-15)
    np.testing.assert_allclose(b, bo, atol=3e-15)
    np.testing.assert_allclose(c, co, atol=3e-15)


def test_radau_rejects_unsupported_stage_count(irkmg):
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_radau_iia(4)
    assert e.value.status == irkmg.IRKMG_EINVAL


def test_defaults_and_strerror(irkmg):
    o = irkmg.irkmg_default_options()
    assert (o.nu_pre, o.nu_post, o.smoother, o.cheb_lo, o.cheb_hi) == (2, 2, 1, 2.0, 8.0)
    assert (o.restart, o.rtol, o.patch_precision) == (30, 1e-10, 64)
    assert irkmg.irkmg_strerror(irkmg.IRKMG_ESINGULAR).startswith("singular")
    assert irkmg.irkmg_strerror(99) == "unknown status"


@pytest.mark.parametrize("bad", ["tableau", "dt", "levels", "precision", "smoother", "dim",
                                 "fixed"])
def test_setup_rejects_bad_arguments_before_touching_the_gpu(irkmg, bad):
    """Validation failures are reported as EINVAL/ENOTIMPL with a message and a
    NULL context; they happen before any CUDA call, so this runs on the CPU."""
    A, b, c = irkmg.irkmg_radau_iia(2)
    o = irkmg.irkmg_default_options()
    dt = 0.1
    if bad == "tableau":
        A = A.copy()
        A[0, 0] += 1e-6            # row sum no longer equals c_1 (Section 2 consistency)
    elif bad == "dt":
        dt = -1.0
    elif bad == "levels":
        o.nlevels = 1
    elif bad == "precision":
        o.patch_precision = 16
    elif bad == "fixed":
        o.patch_form = 1
        o.patch_fixed = 2
    elif bad == "smoother":
        o.smoother = 1
        o.cheb_lo, o.cheb_hi = 8.0, 2.0
    coords, cells, bnd = synth.square_mesh(2)
    if bad == "dim":
        xy, pxy = irkmg._hptr(coords, np.float64)
        cl, pcl = irkmg._hptr(cells, np.int64)
        bd, pbd = irkmg._hptr(bnd, np.uint8)
        Aa, pA = irkmg._hptr(A, np.float64)
        ba, pb = irkmg._hptr(b, np.float64)
        ca, pc = irkmg._hptr(c, np.float64)
        mesh = irkmg.Mesh(4, xy.shape[0], cl.shape[0], pxy, pcl, pbd)
        tab = irkmg.Tableau(2, pA, pb, pc)
        h = ct.c_void_p()
        rc = irkmg.lib().irkmg_setup(ct.byref(mesh), ct.byref(tab), 0.1, 1.0, ct.byref(o), ct.byref(h))
        assert rc == irkmg.IRKMG_ENOTIMPL and not h.value
        return
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_setup(coords, cells, bnd, A, b, c, dt, 1.0, o)
    assert e.value.status == irkmg.IRKMG_EINVAL
    assert irkmg.lib().irkmg_last_error().decode()


def test_3d_wind_is_rejected_before_touching_the_gpu(irkmg):
    """The Oseen wind is built for 2D meshes only: a 3D set-up with a wind
    returns ENOTIMPL from validation, before any CUDA call."""
    A, b, c = irkmg.irkmg_radau_iia(2)
    coords, cells, bnd = synth.cube_mesh(1)
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_setup(coords, cells, bnd, A, b, c, 0.1, 1.0, irkmg.irkmg_default_options(),
                          wind=np.zeros((27, 2)))
    assert e.value.status == irkmg.IRKMG_ENOTIMPL


def _tableaux():
    from oracle import tableau
    out = [("radau_iia", s, tableau.radau_iia(s)[0]) for s in (1, 2, 3)]
    out += [(f, s, getattr(tableau, f)(s)[0]) for f in ("gauss", "lobatto_iiic") for s in (2, 3)]
    return out


@pytest.mark.parametrize("name,s,A", _tableaux(), ids=lambda x: str(x) if not hasattr(x, "shape") else "")
def test_kron_split_block_diagonalises_the_butcher_matrix(irkmg, name, s, A):
    """The decoupled patch solves rest on A = T D T⁻¹ (the Kronecker form of
    the stage system, Section 3): T D T⁻¹ gives back A, T⁻¹ inverts T, D is
    block diagonal with [[α, β], [−β, α]] (β > 0) for each complex pair and its
    eigenvalues are those of A (LAPACK on the oracle's tableau)."""
    T, Ti, D = irkmg.irkmg_kron_split(A)
    np.testing.assert_allclose(T @ D @ Ti, A, atol=1e-14)
    np.testing.assert_allclose(T @ Ti, np.eye(s), atol=1e-14)
    lam = np.linalg.eigvals(A)
    i = 0
    while i < s:
        if i + 1 < s and D[i, i + 1] != 0.0:
            al, be = D[i, i], D[i, i + 1]
            assert be > 0 and D[i + 1, i] == -be and D[i + 1, i + 1] == al
            assert np.min(np.abs(lam - complex(al, be))) < 1e-13
            assert abs(T[:, i] @ T[:, i + 1]) < 1e-13   # Re v and Im v rotated orthogonal
            assert abs(T[:, i] @ T[:, i] + T[:, i + 1] @ T[:, i + 1] - 1.0) < 1e-14
            i += 2
        else:
            assert np.min(np.abs(lam - D[i, i])) < 1e-13
            assert abs(np.linalg.norm(T[:, i]) - 1.0) < 1e-14
            i += 1
    off = D.copy()
    for k in range(s):
        off[k, k] = 0.0
        if k + 1 < s:
            off[k, k + 1] = off[k + 1, k] = 0.0 if D[k, k + 1] != 0.0 else off[k, k + 1]
    assert np.all(off == 0.0)


def test_decoupled_form_needs_distinct_eigenvalues(irkmg):
    """Two copies of the implicit midpoint rule (a valid tableau whose Butcher
    matrix is 0.5 I) cannot be split into distinct eigen-blocks: the split and
    a set-up asking for decoupled patches report ENOTIMPL before any CUDA call;
    patch_form outside 0..3 is EINVAL."""
    A = 0.5 * np.eye(2)
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_kron_split(A)
    assert e.value.status == irkmg.IRKMG_ENOTIMPL
    coords, cells, bnd = synth.square_mesh(2)
    o = irkmg.irkmg_default_options()
    o.patch_form = 1
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_setup(coords, cells, bnd, A, np.array([0.5, 0.5]), np.array([0.5, 0.5]),
                          0.1, 1.0, o)
    assert e.value.status == irkmg.IRKMG_ENOTIMPL
    A, b, c = irkmg.irkmg_radau_iia(2)
    o.patch_form = 4
    with pytest.raises(irkmg.IrkmgError) as e:
        irkmg.irkmg_setup(coords, cells, bnd, A, b, c, 0.1, 1.0, o)
    assert e.value.status == irkmg.IRKMG_EINVAL


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (12, 3), (30, 4)])
def test_hessenberg_eigenvalues_match_lapack(irkmg, n, seed):
    """The Ritz-value solver (shifted QR in complex arithmetic) on seeded
    upper Hessenberg matrices, which have real and complex-pair eigenvalues,
    against LAPACK's eigenvalues."""
    rng = np.random.default_rng(seed)
    H = np.triu(rng.standard_normal((n, n)), -1)
    ev = irkmg.irkmg_hessenberg_eigvals(H)
    ref = np.linalg.eigvals(H)
    for z in ref:
        assert np.min(np.abs(ev - z)) <= 1e-10 * max(1.0, np.abs(ref).max())
    assert ev.imag.sum() == pytest.approx(0.0, abs=1e-9)


def test_hessenberg_eigenvalues_special_cases(irkmg):
    """A rotation (eigenvalues ±i), a split matrix (zero subdiagonal) and a
    Jordan-like block with a tiny perturbation."""
    ev = irkmg.irkmg_hessenberg_eigvals(np.array([[0.0, -1.0], [1.0, 0.0]]))
    np.testing.assert_allclose(np.sort_complex(ev), [-1j, 1j], atol=1e-14)
    H = np.array([[2.0, 1.0, 3.0], [0.0, 5.0, 1.0], [0.0, 4.0, 1.0]])
    ev = irkmg.irkmg_hessenberg_eigvals(H)
    np.testing.assert_allclose(np.sort(ev.real), np.sort(np.linalg.eigvals(H).real), atol=1e-12)
    H = np.array([[1.0, 1.0], [1e-12, 1.0]])
    ev = irkmg.irkmg_hessenberg_eigvals(H)
    np.testing.assert_allclose(np.sort(ev.real), np.sort(np.linalg.eigvals(H).real), atol=1e-9)


def test_binding_structs_match_the_header_layout(irkmg, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the same struct from include/irkmg.h (a field
    added on one side only would shift every later field)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = [(irkmg.Mesh, "irkmg_mesh"), (irkmg.Tableau, "irkmg_tableau"),
             (irkmg.Options, "irkmg_options"), (irkmg.Stats, "irkmg_stats"),
             (irkmg.LevelInfo, "irkmg_level_info"), (irkmg.NSStats, "irkmg_ns_stats"),
             (irkmg.Trace, "irkmg_trace")]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "irkmg.h"', "int main(void) {"]
    expect = []
    for cls, cname in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(ct.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {name}));')
            expect.append(getattr(cls, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect

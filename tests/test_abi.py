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


@pytest.mark.parametrize("bad", ["tableau", "dt", "levels", "precision", "smoother", "dim"])
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

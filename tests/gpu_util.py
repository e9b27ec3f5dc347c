"""Shared helpers for the GPU parity tests: set up the same seeded problem on
the CUDA library (through the C ABI) and on the oracle."""
import functools

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07381_gb300 import irkmg
    irkmg.lib()   # raises if the library is missing: no silent fallback
    return irkmg


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    """Error of a against the reference b, as the larger of two measures so
    that an assertion rel(a, b) < tol checks both: the relative l2 error
    ||a - b|| / ||b||, and entry by entry max_i |a_i - b_i| / (|b_i| + ||b||_inf)
    (a few wrong entries of a long vector hide in the l2 norm, not here)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    d = np.abs(a - b)
    l2 = np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300)
    if b.size == 0:
        return l2
    ent = np.max(d / np.maximum(np.abs(b) + np.max(np.abs(b)), 1e-300))
    return max(l2, float(ent))


@functools.lru_cache(maxsize=None)
def oracle_hierarchy(n0, nlevels, s, dt, nu=1.0, smoother="chebyshev", wind_key=None):
    from oracle import mg, tableau
    A, b, c = tableau.radau_iia(s)
    wind = WINDS[wind_key] if wind_key else None
    return mg.Hierarchy(*synth.square_mesh(n0), nlevels, A, dt, nu=nu, wind_finest=wind,
                        smoother=smoother)


WINDS = {}


def gpu_context(irkmg, n0, nlevels, s, dt, nu=1.0, smoother=1, precision=64, wind=None,
                **kw):
    A, b, c = irkmg.irkmg_radau_iia(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = nlevels
    o.smoother = smoother
    o.patch_precision = precision
    for k, v in kw.items():
        setattr(o, k, v)
    coords, cells, bnd = synth.square_mesh(n0)
    return irkmg.irkmg_setup(coords, cells, bnd, A, b, c, dt, nu, o, wind=wind)

"""The threaded host assembly sums every stored entry in one fixed order
(ascending cell index), so a context built on one host thread and one built
on seven give bitwise-identical operators (J x and J^T x on every level) and,
with the same launch shapes pinned, bitwise-identical V-cycles."""
import os

import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


def _ctx(irkmg, threads):
    old = os.environ.get("IRKMG_HOST_THREADS")
    os.environ["IRKMG_HOST_THREADS"] = str(threads)
    try:
        A, b, c = irkmg.irkmg_radau_iia(3)
        o = irkmg.irkmg_default_options()
        o.nlevels = 5
        o.patch_form = 1
        o.patch_fixed = 1
        return irkmg.irkmg_setup(*synth.square_mesh(4), A, b, c, 1 / 64, 1.0, o)
    finally:
        if old is None:
            del os.environ["IRKMG_HOST_THREADS"]
        else:
            os.environ["IRKMG_HOST_THREADS"] = old


def test_assembly_does_not_depend_on_the_host_thread_count():
    irkmg = need_gpu()
    c1, c7 = _ctx(irkmg, 1), _ctx(irkmg, 7)
    try:
        for l in range(c1.nlevels):
            N = c1.levels[l]["N"]
            assert c7.levels[l]["N"] == N
            x = dev(synth.random_vector(70 + l, N))
            for tr in (False, True):
                y1, y7 = dev(np.zeros(N)), dev(np.zeros(N))
                irkmg.irkmg_apply(c1, x, y1, level=l, transpose=tr)
                irkmg.irkmg_apply(c7, x, y7, level=l, transpose=tr)
                assert np.array_equal(host(y1), host(y7))
        for l in range(1, c1.nlevels):
            for ctx in (c1, c7):
                irkmg.irkmg_level_set_apply(ctx, l, 3, 1)
        N = c1.finest["N"]
        r = dev(synth.random_vector(79, N))
        z1, z7 = dev(np.zeros(N)), dev(np.zeros(N))
        irkmg.irkmg_vcycle(c1, r, z1)
        irkmg.irkmg_vcycle(c7, r, z7)
        assert np.array_equal(host(z1), host(z7))
    finally:
        c1.close()
        c7.close()

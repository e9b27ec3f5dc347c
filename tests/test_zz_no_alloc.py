"""GPU test of irkmg_smooth_noalloc, the relaxation entry point that allocates
no device memory (for callers that cannot call cudaMalloc when they relax a
vector: their device memory belongs to another allocator, or their loop must
not pay an allocation's implicit synchronisation).  It must give what
irkmg_smooth gives, call after call, although its work vectors live in one
static device array shared by every call.  This file is collected last so a
failure here never hides the other tests."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, gpu_context, host, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("smoother", [1, 0], ids=["chebyshev", "damped"])
def test_noalloc_smooth_matches_smooth_on_consecutive_calls(smoother):
    irkmg = need_gpu()
    ctx = gpu_context(irkmg, 2, 4, 3, 1 / 64, smoother=smoother, omega=0.125)
    try:
        for call in range(2):               # two calls in a row share the static array
            for level in (ctx.nlevels - 1, 1):
                N = ctx.N(level)
                F = dev(synth.random_vector(100 + 10 * call + level, N))
                x0 = 0.1 * synth.random_vector(200 + 10 * call + level, N)
                xa, xb = dev(x0), dev(x0)
                irkmg.irkmg_smooth(ctx, F, xa, 2, level=level)
                irkmg.irkmg_smooth_noalloc(ctx, F, xb, 2, level=level)
                assert rel(host(xb), host(xa)) <= 1e-12
                irkmg.irkmg_smooth(ctx, F, xa, 3, level=level, transpose=True)
                irkmg.irkmg_smooth_noalloc(ctx, F, xb, 3, level=level, transpose=True)
                assert rel(host(xb), host(xa)) <= 1e-12
    finally:
        ctx.close()


def test_noalloc_smooth_rejects_levels_beyond_the_static_array():
    irkmg = need_gpu()
    ctx = gpu_context(irkmg, 8, 5, 2, 1 / 64)        # finest 128x128, s = 2: N = 293,378
    big = gpu_context(irkmg, 8, 6, 3, 1 / 64)        # finest 256x256, s = 3: N = 1,765,641
    try:
        N = big.N()
        assert N > 524288
        F, x = dev(np.zeros(N)), dev(np.ones(N))
        with pytest.raises(irkmg.IrkmgError) as e:
            irkmg.irkmg_smooth_noalloc(big, F, x, 1)
        assert e.value.status == irkmg.IRKMG_EINVAL and "at most 524288" in str(e.value)
        assert np.all(host(x) == 1.0)                 # nothing was done
        n = ctx.N()
        xa, xb = dev(np.zeros(n)), dev(np.zeros(n))
        F = dev(synth.random_vector(7, n))
        irkmg.irkmg_smooth(ctx, F, xa, 2)
        irkmg.irkmg_smooth_noalloc(ctx, F, xb, 2)
        assert rel(host(xb), host(xa)) <= 1e-12
    finally:
        ctx.close()
        big.close()

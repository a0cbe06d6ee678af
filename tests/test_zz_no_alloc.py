"""The sums entry point that allocates nothing.

Callers that may not allocate device memory while they run (a host framework
that gives the whole GPU to its own pool at start-up, a service that must not
stall on an allocation) use icarus_conservation_sums_static, whose scratch is a
fixed array inside the library.  Its result must equal the ordinary
icarus_conservation_sums on the same state, call after call, even though every
call reuses (and leaves behind) the same scratch.  This file is collected last
on purpose and also passes when it runs alone in a fresh process."""
import numpy as np
import pytest

from gpu_common import make_pair, wind_setup
from paper_2211_12867_gb300.icarus import conservation_sums_static

pytestmark = pytest.mark.gpu
TOL = 1e-13   # the bound the conservation tests use for FP64 sums


def _close(a, b):
    return np.all(np.abs(a - b) <= TOL * (np.abs(b) + 1e-300))


def test_static_scratch_sums_match_the_allocating_entry_point():
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    wind_setup(g, o)
    ref1 = g.sums(0)
    got1 = conservation_sums_static(g, 0)
    assert _close(got1, ref1), (got1, ref1)
    # second call in a row after the state changed: the scratch left by the
    # first call must not leak into the result
    g.step(3)
    ref2 = g.sums(0)
    got2 = conservation_sums_static(g, 0)
    assert _close(got2, ref2), (got2, ref2)
    assert not np.allclose(ref1, ref2)


def test_static_scratch_sums_allocate_no_device_memory():
    """What the entry point is for: once a context exists, calls leave the
    device's free memory unchanged (read with cudaMemGetInfo), the first call
    included (the scratch and the kernels are put in place when the context
    is created)."""
    import torch
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    wind_setup(g, o)
    ref = g.sums(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert _close(conservation_sums_static(g, 0), ref)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_sums_on_a_refined_member_and_fp32():
    import math
    g, o = make_pair(n=(24, 16, 32), nb=(8, 8, 8), max_level=2, stretch=True, max_blocks=400,
                     x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi))
    wind_setup(g, o)
    f = np.zeros(g.n_leaves(0), dtype=np.int8)
    f[[1, 4, 9]] = 1
    g.set_flags(f)
    g.regrid()
    for _ in range(2):
        assert _close(conservation_sums_static(g, 0), g.sums(0))
    g32, o32 = make_pair(n=(60, 16, 32), nb=(12, 8, 8), precision=1)
    wind_setup(g32, o32)
    for _ in range(2):
        assert _close(conservation_sums_static(g32, 0), g32.sums(0))

"""Parity at the shapes the product runs, not only at test sizes.

* The 512 x 60 x 180 wedge that bench.py times: blocks of 64 x 60 x 180
  cells, the stage tile 12 x 20 with 32-plane radial segments (the
  autotuner's choice on GB300), the shared-memory geometry staging and the
  184-wide padded phi rows of that shape, with the cone CME being injected.
  FP64 against the oracle within 1e-10; FP32 error per variable reported
  and bounded.
* The stretched 264 x 36 x 96 grid with 12^3 blocks of the AMR workloads:
  cycles of GPU flags -> regrid -> 10 steps with the cone CME.  Flags are
  compared bit for bit on the same stored state, ghost layers included (the
  oracle's estimator runs on the padded blocks the device filled), in FP64
  and in FP32 mode; trees bit for bit; FP64 state within 1e-10."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, rel_linf, wind_setup
from paper_2211_12867_gb300 import inputs as I
from paper_2211_12867_gb300.icarus import FP32_MIXED, FP64

pytestmark = pytest.mark.gpu
WEDGE = dict(n=(512, 60, 180), nb=(64, 60, 180), x_min=(0.1, math.pi / 6, 0.0),
             x_max=(2.0, 5 * math.pi / 6, 2 * math.pi))
CFG3 = dict(n=(264, 36, 96), nb=(12, 12, 12), stretch=True, x_min=(0.1, math.pi / 6, 0.0),
            x_max=(2.0, 5 * math.pi / 6, 2 * math.pi))
CRIT = dict(e_refine=0.1, e_coarsen=0.0125, eps=0.01, dv=I.kms(50.0))


def _wedge(precision):
    g, o = make_pair(precision=precision, **WEDGE)
    wind_setup(g, o)
    cme = dict(I.cme_config2(seed=0), t_start=0.0)
    g.inject_cone_cme(0, **cme)
    o.set_cme(**cme)
    o.snapshot_vbg()
    g.set_tile(12, 20, 32)
    return g, o


def test_bench_wedge_fp64_at_the_bench_launch_shape():
    g, o = _wedge(FP64)
    t = g.step(5)
    o.advance(5)
    assert abs(t[0] - o.t) / o.t < 1e-12
    err = rel_linf(g.get_state(0), o.get_state())
    assert err.max() < 1e-10, err


def test_bench_wedge_fp32_error_against_the_fp64_oracle():
    g, o = _wedge(FP32_MIXED)
    g.step(5)
    o.advance(5)
    err = rel_linf(g.get_state(0), o.get_state())
    print("FP32 - FP64 oracle after 5 steps, per variable:", err)
    assert err.max() < 2e-5, err


def _flags_on_the_device_data(g, o, member=0):
    """GPU flags, and the oracle's estimator on the padded blocks (ghost
    layers included) that the GPU estimator read"""
    fg = g.flag_refine(**CRIT)
    o.set_state(g.get_state(member))
    for n in range(o.nleaves):
        o.set_padded(n, g.get_padded(member, n))
    return fg, o.flag(**CRIT)


@pytest.mark.parametrize("precision", [FP64, FP32_MIXED])
def test_config3_grid_flag_regrid_cycles(precision):
    g, o = make_pair(max_level=3, max_blocks=20000, precision=precision, **CFG3)
    wind_setup(g, o)
    cme = dict(I.cme_config2(seed=0), t_start=0.0)
    g.inject_cone_cme(0, **cme)
    o.set_cme(**cme)
    o.snapshot_vbg()
    t = g.step(20)
    o.advance(20)
    refined = 0
    for cycle in range(3):
        if precision == FP64:
            err = rel_linf(g.get_state(0), o.get_state())
            assert err.max() < 1e-10, (cycle, err)
        fg, fo = _flags_on_the_device_data(g, o)
        assert np.array_equal(fg, fo), (cycle, np.flatnonzero(fg != fo)[:10])
        refined += int((fg == 1).sum())
        g.regrid()
        o.regrid(fg)
        assert np.array_equal(g.tree(0), o.tree()), cycle
        assert o.balance_violations() == 0
        # the oracle continues from the device's regridded state and time
        o.set_state(g.get_state(0))
        o.t = t[0]
        t = g.step(10)
        o.advance(10)
        if precision == FP64:
            assert abs(t[0] - o.t) <= 1e-12 * o.t
        else:
            print("cycle", cycle, "FP32 - FP64 oracle after 10 steps:", rel_linf(g.get_state(0), o.get_state()))
    assert refined > 0 and g.tree(0)[:, 0].max() >= 2, "the cycles must refine"
    if precision == FP64:
        err = rel_linf(g.get_state(0), o.get_state())
        assert err.max() < 1e-10, err

"""The paper's shock criterion (Sect. 3.2) on the GPU against the oracle.

Flags must agree bit for bit on the same stored state: the oracle's
estimator runs on the padded blocks (ghost layers included) that the GPU
estimator read.  Covered: a converging analytic flow whose windows cross the
periodic seam, a cone-CME run in FP64 and FP32 mode, and flag -> regrid
cycles whose trees must match."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, wind_setup
from paper_2211_12867_gb300 import inputs as I
from paper_2211_12867_gb300.icarus import FLAG_SHOCK, FP32_MIXED, FP64, SHOCK_WINDOWS

pytestmark = pytest.mark.gpu
STR = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi), stretch=True)


def _both(g, o, div_thr=0.0, windows=SHOCK_WINDOWS):
    fg = g.flag_refine(mode=FLAG_SHOCK, div_thr=div_thr, windows=windows)
    o.set_state(g.get_state(0))
    o.t = g.step(0)[0]
    for n in range(o.nleaves):
        o.set_padded(n, g.get_padded(0, n))
    return fg, o.flag_shock(div_thr, *windows)


def test_converging_flow_windows_across_the_seam():
    g, o = make_pair(n=(16, 36, 48), nb=(8, 6, 8), omega=0.0, bc_lo=(1, 1, 0), bc_hi=(1, 1, 0))
    W = np.zeros((g.n_leaves(0), 8) + g.block)
    W[:, 0], W[:, 4], W[:, 1] = 1.0, 1.0, -1.0
    g.set_state(0, W, prim=True)
    for lon_e, lon_c in ((math.radians(350.0), math.radians(10.0)), (math.radians(100.0), math.radians(200.0))):
        g.set_earth(0, math.radians(93.0), lon_e)
        o.set_earth(math.radians(93.0), lon_e)
        cme = dict(t_start=0.0, t_max=1.0, colat=math.pi / 2, lon=lon_c, half_width=0.3, v=5.0, rho=10.0, p=1.0)
        g.inject_cone_cme(0, **cme)
        o.set_cme(**cme)
        fg, fo = _both(g, o)
        assert np.array_equal(fg, fo)
        assert 0 < (fg == 1).sum() < len(fg)
        # the windows switched off: every converging block refines
        fg, fo = _both(g, o, windows=(0.0, 0.0, 0.0))
        assert np.array_equal(fg, fo) and np.all(fg == 1)


@pytest.mark.parametrize("precision", [FP64, FP32_MIXED])
def test_cone_cme_run_flags_bit_exact(precision):
    g, o = make_pair(n=(48, 24, 48), nb=(12, 12, 12), max_level=3, max_blocks=4000, precision=precision, **STR)
    wind_setup(g, o)
    cme = dict(I.cme_config2(seed=0), t_start=0.0)
    g.inject_cone_cme(0, **cme)
    o.set_cme(**cme)
    g.set_earth(0, math.pi / 2, math.pi, 0.0, I.OMEGA_SYN)
    o.set_earth(math.pi / 2, math.pi, 0.0, I.OMEGA_SYN)
    g.step(40)
    fg, fo = _both(g, o)
    assert np.array_equal(fg, fo)
    assert (fg == 1).sum() > 0 and (fg == -1).sum() > 0
    # a threshold: fewer blocks, still the same on both sides
    thr = 2.0
    fg2, fo2 = _both(g, o, div_thr=thr)
    assert np.array_equal(fg2, fo2)
    assert (fg2 == 1).sum() <= (fg == 1).sum()


def test_shock_flags_drive_regrids():
    g, o = make_pair(n=(48, 24, 48), nb=(12, 12, 12), max_level=3, max_blocks=4000, **STR)
    wind_setup(g, o)
    cme = dict(I.cme_config2(seed=0), t_start=0.0)
    g.inject_cone_cme(0, **cme)
    o.set_cme(**cme)
    o.snapshot_vbg()
    g.set_earth(0, math.pi / 2, math.pi, 0.0, I.OMEGA_SYN)
    o.set_earth(math.pi / 2, math.pi, 0.0, I.OMEGA_SYN)
    g.step(30)
    for cycle in range(3):
        fg, fo = _both(g, o)
        assert np.array_equal(fg, fo), cycle
        g.regrid()
        o.regrid(fg)
        assert np.array_equal(g.tree(0), o.tree()), cycle
        assert o.balance_violations() == 0
        g.step(10)
    assert g.tree(0)[:, 0].max() >= 2

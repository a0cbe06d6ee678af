"""CME density tracer (Sect. 3.1) and the tracer and combined refinement
criteria (Sects. 3.1, 3.3) on the GPU against the oracle: transport of
rho X with the cone CME (FP64 within 1e-10, FP32 error reported), X = 1
staying rho X = rho, tracer data through regrids, and flags bit for bit on
the same stored state."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, rel_linf, wind_setup
from paper_2211_12867_gb300 import inputs as I
from paper_2211_12867_gb300.icarus import FLAG_COMBINED, FLAG_TRACER, FP32_MIXED, FP64, SHOCK_WINDOWS

pytestmark = pytest.mark.gpu
STR = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi), stretch=True)


def _cme_pair(precision=FP64, **kw):
    args = dict(n=(48, 24, 48), nb=(12, 12, 12), tracer=True, precision=precision, **STR)
    args.update(kw)
    g, o = make_pair(**args)
    wind_setup(g, o)
    cme = dict(I.cme_config2(seed=0), t_start=0.0)
    g.inject_cone_cme(0, **cme)
    o.set_cme(**cme)
    o.snapshot_vbg()
    return g, o


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_tracer_transport_matches_oracle_fp64():
    g, o = _cme_pair()
    assert np.all(g.get_tracer(0) == 0)
    g.step(30)
    o.advance(30)
    T, To = g.get_tracer(0), o.get_tracer()
    assert To.max() > 0, "the CME must have brought tracer in"
    assert _rel(T, To) < 1e-10, _rel(T, To)
    assert rel_linf(g.get_state(0), o.get_state()).max() < 1e-10


def test_tracer_fp32_error_against_the_fp64_oracle():
    g, o = _cme_pair(precision=FP32_MIXED)
    g.step(30)
    o.advance(30)
    err = _rel(g.get_tracer(0), o.get_tracer())
    print("FP32 tracer - FP64 oracle after 30 steps (relative to max):", err)
    assert err < 1e-4, err


def test_unit_fraction_follows_the_mass():
    g, o = make_pair(n=(16, 16, 16), nb=(8, 8, 8), geometry=1, x_min=(0, 0, 0), x_max=(1, 1, 1), omega=0.0,
                     divb_cd=0.0, gamma=5 / 3, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), tracer=True)
    W = np.zeros((g.n_leaves(0), 8) + g.block)
    for n in range(g.n_leaves(0)):
        W[n] = I.random_state(g.block, 100 + n, 5 / 3, v=0.3, b=0.3)
    g.set_state(0, W, prim=True)
    g.set_tracer(0, g.get_state(0)[:, 0])
    g.step(8)
    assert np.allclose(g.get_tracer(0), g.get_state(0)[:, 0], rtol=1e-13, atol=0)


def _flags_same_state(g, o, mode, **kw):
    fg = g.flag_refine(mode=mode, **kw)
    o.set_state(g.get_state(0))
    o.set_tracer(g.get_tracer(0))
    o.t = g.step(0)[0]
    for n in range(o.nleaves):
        o.set_padded(n, g.get_padded(0, n))
    w = kw.get("windows", SHOCK_WINDOWS)
    fo = o.flag_tracer(kw.get("x_thr", 0.0), kw.get("div_thr", 0.0), *w, combined=(mode == FLAG_COMBINED))
    return fg, fo


@pytest.mark.parametrize("precision", [FP64, FP32_MIXED])
def test_tracer_and_combined_flags_bit_exact(precision):
    g, o = _cme_pair(precision=precision, max_level=3, max_blocks=4000)
    g.set_earth(0, math.pi / 2, math.pi, 0.0, I.OMEGA_SYN)
    o.set_earth(math.pi / 2, math.pi, 0.0, I.OMEGA_SYN)
    g.step(12)
    for mode, kw in ((FLAG_TRACER, dict(windows=(0.0, 0.0, 0.0))), (FLAG_TRACER, dict(x_thr=0.1)),
                     (FLAG_COMBINED, dict()), (FLAG_COMBINED, dict(x_thr=0.5, div_thr=1.0))):
        fg, fo = _flags_same_state(g, o, mode, **kw)
        assert np.array_equal(fg, fo), (mode, kw)
    # the CME plasma (X near 1) fills only part of the grid after 12 steps
    fg, _ = _flags_same_state(g, o, FLAG_TRACER, windows=(0.0, 0.0, 0.0), x_thr=0.1)
    assert (fg == 1).sum() > 0 and (fg == -1).sum() > 0


def test_tracer_through_regrids():
    g, o = _cme_pair(max_level=3, max_blocks=4000)
    g.step(30)
    o.advance(30)
    for cycle in range(2):
        fg, fo = _flags_same_state(g, o, FLAG_TRACER, windows=(0.0, 0.0, 0.0))
        assert np.array_equal(fg, fo)
        g.regrid()
        o.regrid(fg)
        assert np.array_equal(g.tree(0), o.tree())
        assert _rel(g.get_tracer(0), o.get_tracer()) < 1e-12
        g.step(5)
        o.advance(5)
        assert _rel(g.get_tracer(0), o.get_tracer()) < 1e-10
    assert g.tree(0)[:, 0].max() >= 2

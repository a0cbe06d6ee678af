"""Oracle of the shock criterion (Sect. 3.2) against closed forms.

The paper refines where the velocity divergence is negative, limited to
windows around the Sun-Earth line (Earth longitude +-30 deg, Earth
colatitude +-10 deg) and to the CME's hemisphere (CME longitude +-90 deg),
and coarsens once the criterion no longer holds.  The divergence is taken by
central differences at cell centres in the spherical form; each of its three
terms has a closed form for a suitable field, and the windows are checked by
brute force over the cell centres.  Slips these pins catch: a dropped r^2 or
sin(theta) weight, face instead of centre coordinates, a sign, a window on
the wrong coordinate or without the periodic wrap."""
import math

import numpy as np
import pytest

import oracle as O

XMIN = (0.1, math.pi / 6, 0.0)
XMAX = (1.1, 5 * math.pi / 6, 2 * math.pi)
N = (24, 12, 16)
NB = (8, 6, 8)
OUT = (O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC)


def _grid(n=N, nb=NB, stretch=0, geometry=0, xmin=XMIN, xmax=XMAX):
    return O.Grid(n=n, nb=nb, stretch=stretch, geometry=geometry, xmin=xmin, xmax=xmax, gamma=1.5, omega=0.0,
                  divb_cd=0.0, bc_lo=OUT, bc_hi=OUT)


def _centres(n=N, xmin=XMIN, xmax=XMAX, stretch=0):
    c = []
    for d in range(3):
        f = np.linspace(0.0, 1.0, n[d] + 1)
        if d == 0 and stretch:
            f = xmin[0] * (xmax[0] / xmin[0]) ** f
        else:
            f = xmin[d] + (xmax[d] - xmin[d]) * f
        c.append(0.5 * (f[1:] + f[:-1]))
    return c


def _set_velocity(g, field, n=N, stretch=0, xmin=XMIN, xmax=XMAX):
    """primitive state rho = 1, p = 1, B = 0, v = field(r, th, ph) at centres"""
    rc, tc, pc = _centres(n, xmin, xmax, stretch)
    R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
    vr, vt, vp = field(R, T, P)
    W = np.zeros((g.nleaves, 8) + g.nb)
    for m, (_, bi, bj, bk) in enumerate(g.tree()):
        sl = (slice(bi * g.nb[0], (bi + 1) * g.nb[0]), slice(bj * g.nb[1], (bj + 1) * g.nb[1]),
              slice(bk * g.nb[2], (bk + 1) * g.nb[2]))
        W[m, 0], W[m, 4] = 1.0, 1.0
        W[m, 1], W[m, 2], W[m, 3] = vr[sl], vt[sl], vp[sl]
    g.set_state(W, prim=True)
    g.ghost_fill()
    return R, T, P


def _global_divv(g, n=N):
    out = np.zeros(n)
    for m, (_, bi, bj, bk) in enumerate(g.tree()):
        out[bi * g.nb[0]:(bi + 1) * g.nb[0], bj * g.nb[1]:(bj + 1) * g.nb[1],
            bk * g.nb[2]:(bk + 1) * g.nb[2]] = g.divv(m)
    return out


INNER = (slice(1, -1), slice(1, -1), slice(None))   # cells whose neighbours are all interior


def test_radial_term_linear_field_equidistant():
    """v_r = r: div = 3 continuously; the centred difference on an
    equidistant grid gives exactly 3 + (dr / r)^2."""
    g = _grid()
    R, T, P = _set_velocity(g, lambda r, t, p: (r, 0 * r, 0 * r))
    dr = (XMAX[0] - XMIN[0]) / N[0]
    want = 3.0 + (dr / R) ** 2
    assert np.allclose(_global_divv(g)[INNER], want[INNER], rtol=1e-12, atol=0)


def test_radial_term_second_order_on_the_stretched_grid():
    errs = []
    for k in (1, 2, 4):
        n = (24 * k, 12, 16)
        g = _grid(n=n, nb=(8, 6, 8), stretch=1)
        _set_velocity(g, lambda r, t, p: (r, 0 * r, 0 * r), n=n, stretch=1)
        errs.append(np.abs(_global_divv(g, n)[INNER] - 3.0).max())
    assert errs[0] > 3.5 * errs[1] > 3.5 * 3.5 * errs[2] > 0, errs


def test_theta_term_uniform_field():
    """v_theta = 1: div = cot(theta) / r; the centred difference of
    sin(theta) v_theta gives exactly cot(theta) sin(dth) / (r dth)."""
    g = _grid()
    R, T, P = _set_velocity(g, lambda r, t, p: (0 * r, 1.0 + 0 * r, 0 * r))
    dth = (XMAX[1] - XMIN[1]) / N[1]
    want = np.cos(T) / np.sin(T) * math.sin(dth) / (R * dth)
    assert np.allclose(_global_divv(g)[INNER], want[INNER], rtol=1e-11, atol=1e-13)


def test_phi_term_sine_field():
    """v_phi = sin(phi): div = cos(phi) / (r sin(theta)); centred:
    cos(phi) sin(dph) / (dph r sin(theta))."""
    g = _grid()
    R, T, P = _set_velocity(g, lambda r, t, p: (0 * r, 0 * r, np.sin(p)))
    dph = (XMAX[2] - XMIN[2]) / N[2]
    want = np.cos(P) * math.sin(dph) / (dph * R * np.sin(T))
    assert np.allclose(_global_divv(g)[INNER], want[INNER], rtol=1e-11, atol=1e-12)


def test_cartesian_linear_field():
    g = _grid(geometry=1, xmin=(0, 0, 0), xmax=(2.0, 1.5, 1.0))
    _set_velocity(g, lambda x, y, z: (0.5 * x, -2.0 * y, 0.25 * z), xmin=(0, 0, 0), xmax=(2.0, 1.5, 1.0))
    d = _global_divv(g)
    assert np.allclose(d[1:-1, 1:-1, 1:-1], 0.5 - 2.0 + 0.25, rtol=0, atol=1e-12)


def test_rigid_rotation_and_outflow_refine_nothing():
    """div(Omega x r) = 0 exactly; a uniform radial outflow v0 r_hat has
    div = 2 v0 / r > 0 (exact on the equidistant grid): neither is a shock."""
    g = _grid()
    _set_velocity(g, lambda r, t, p: (0 * r, 0 * r, 0.7 * r * np.sin(t)))
    assert np.abs(_global_divv(g)).max() == 0.0
    g.set_earth(math.pi / 2, 0.0)
    g.set_cme(0.0, 1.0, math.pi / 2, 0.0, 0.3, 5.0, 10.0, 1.0)
    assert np.all(g.flag_shock(dlon_earth=0, dcolat_earth=0, dlon_cme=0) == -1)
    R, T, P = _set_velocity(g, lambda r, t, p: (2.0 + 0 * r, 0 * r, 0 * r))
    assert np.allclose(_global_divv(g)[INNER], (4.0 / R)[INNER], rtol=1e-12)
    assert np.all(g.flag_shock(dlon_earth=0, dcolat_earth=0, dlon_cme=0) == -1)


def _brute_force(g, R, T, P, div, thr, lon_e, colat_e, lon_c, w):
    """+1 where some interior cell of the block has div < -thr inside all
    windows (half widths w = (lon_earth, colat_earth, lon_cme))"""
    def wrap(a):
        return (a + math.pi) % (2 * math.pi) - math.pi
    ok = div < -thr
    if w[0] > 0:
        ok &= np.abs(wrap(P - lon_e)) <= w[0]
    if w[1] > 0:
        ok &= np.abs(T - colat_e) <= w[1]
    if w[2] > 0:
        ok &= np.abs(wrap(P - lon_c)) <= w[2]
    out = []
    for (_, bi, bj, bk) in g.tree():
        blk = ok[bi * g.nb[0]:(bi + 1) * g.nb[0], bj * g.nb[1]:(bj + 1) * g.nb[1], bk * g.nb[2]:(bk + 1) * g.nb[2]]
        out.append(1 if blk.any() else -1)
    return np.array(out, dtype=np.int8)


@pytest.mark.parametrize("lon_e,lon_c", [(math.radians(350.0), math.radians(10.0)),
                                         (math.radians(100.0), math.radians(200.0)),
                                         (math.radians(3.0), math.radians(300.0))])
def test_windows_on_a_converging_flow(lon_e, lon_c):
    """v_r = -1 converges everywhere; the windows (Earth +-30 deg in
    longitude, +-10 deg in colatitude, CME +-90 deg in longitude, across the
    periodic seam) decide which blocks refine."""
    n, nb = (16, 36, 48), (8, 6, 8)
    g = _grid(n=n, nb=nb)
    R, T, P = _set_velocity(g, lambda r, t, p: (-1.0 + 0 * r, 0 * r, 0 * r), n=n)
    div = _global_divv(g, n)
    colat_e = math.radians(93.0)
    g.set_earth(colat_e, lon_e)
    g.set_cme(0.0, 1.0, math.pi / 2, lon_c, 0.3, 5.0, 10.0, 1.0)
    w = (math.radians(30.0), math.radians(10.0), math.radians(90.0))
    got = g.flag_shock(0.0, *w)
    want = _brute_force(g, R, T, P, div, 0.0, lon_e, colat_e, lon_c, w)
    assert np.array_equal(got, want)
    assert 0 < (got == 1).sum() < len(got)


def test_threshold_and_earth_drift():
    n, nb = (16, 36, 48), (8, 6, 8)
    g = _grid(n=n, nb=nb)
    R, T, P = _set_velocity(g, lambda r, t, p: (-1.0 + 0 * r, 0 * r, 0 * r), n=n)
    div = _global_divv(g, n)
    rate, t0, lon0 = 0.4, 1.0, math.radians(40.0)
    g.set_earth(math.pi / 2, lon0, t0, rate)
    g.set_cme(0.0, 1.0, math.pi / 2, math.radians(60.0), 0.3, 5.0, 10.0, 1.0)
    w = (math.radians(30.0), math.radians(10.0), math.radians(90.0))
    for t, thr in ((1.0, 0.0), (1.0, 5.0), (2.5, 0.0), (2.5, 8.0)):
        g.t = t
        got = g.flag_shock(thr, *w)
        want = _brute_force(g, R, T, P, div, thr, lon0 - rate * (t - t0), math.pi / 2, math.radians(60.0), w)
        assert np.array_equal(got, want), (t, thr)
        assert (got == 1).sum() > 0
    # a threshold above every |div| refines nothing
    assert np.all(g.flag_shock(2.0 / 0.1 + 1.0, *w) == -1)


def test_windows_need_earth_and_cme():
    g = _grid()
    _set_velocity(g, lambda r, t, p: (-1.0 + 0 * r, 0 * r, 0 * r))
    assert np.all(g.flag_shock(0.0, 0.5, 0.0, 0.0) == -1)        # Earth window, no Earth set
    assert np.all(g.flag_shock(0.0, 0.0, 0.0, 0.0) == 1)         # no window: every block converges
    g.set_earth(math.pi / 2, 0.0)
    assert np.all(g.flag_shock(0.0, 0.0, 0.0, 1.0) == -1)        # CME window, no CME

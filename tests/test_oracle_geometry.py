"""Oracle geometry pins: Eq. 5, the stretched radial grid of Sect. 2.2 /
Tables 1 and 3, exact cell volumes, and the prolongation offsets."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from golden_io import load
from paper_2211_12867_gb300 import inputs as I

P = load("paper_numbers.txt")
AU_RSUN = I.AU_M / I.R_SUN_M


def test_eq5_gives_46_cells():
    # Sect. 2.2, Eq. 5 with dtheta = 3.75 deg: 45.76 -> 46
    N = I.eq5_cells(P["eq5_r_in_au"], P["eq5_r_out_au"], math.radians(P["eq5_low_dtheta_deg"]))
    assert 45.5 < N < 46.0
    assert round(N) == P["eq5_low_cells"]


def test_inner_boundary_in_solar_radii():
    assert abs(0.1 * AU_RSUN - P["inner_boundary_rsun"]) < 0.05


def test_equidistant_dr_matches_paper():
    for key_n, key_dr, nr in (("equidistant_low_nr", "equidistant_low_dr_rsun", 300),
                              (None, "equidistant_middle_dr_rsun", 600),
                              (None, "equidistant_high_dr_rsun", 1200)):
        g = O.Grid(n=(nr, 4, 4), nb=(nr // 4 if nr % 4 == 0 else nr, 4, 4), stretch=0,
                   xmin=(0.1, math.pi / 6, 0), xmax=(2.0, 5 * math.pi / 6, 2 * math.pi))
        f = g.faces(1, 0)
        dr = np.diff(f) * AU_RSUN
        assert np.allclose(dr, dr[0], rtol=1e-12)
        assert abs(dr[0] - P[key_dr]) / P[key_dr] < 0.01


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5])
def test_stretched_dr_at_1au_matches_table3(level):
    """Table 3: radial resolution at L1 (1 AU) of the stretched Low grid and
    its AMR levels; every level halves the local spacing r ln(q)."""
    keys = ["dr_L1_noamr_rsun", "dr_L1_amr2_rsun", "dr_L1_amr3_rsun", "dr_L1_amr4_rsun",
            "dr_L1_amr5_rsun"]
    g = O.Grid(n=(60, 8, 8), nb=(12, 8, 8), stretch=1, max_level=level,
               xmin=(0.1, math.pi / 6, 0), xmax=(2.0, 5 * math.pi / 6, 2 * math.pi))
    f = g.faces(level, 0)
    q = f[1:] / f[:-1]
    assert np.allclose(q, q[0], rtol=1e-12)          # geometric faces
    assert abs(f[0] - 0.1) < 1e-15 and abs(f[-1] - 2.0) < 1e-14
    dr_1au = 1.0 * (q[0] - 1.0) / math.sqrt(q[0]) * AU_RSUN
    assert abs(dr_1au - P[keys[level - 1]]) / P[keys[level - 1]] < 0.005


def test_coarse_faces_are_fine_faces():
    g = O.Grid(n=(24, 8, 8), nb=(12, 8, 8), stretch=1, max_level=4,
               xmin=(0.1, math.pi / 6, 0), xmax=(2.0, 5 * math.pi / 6, 2 * math.pi))
    for L in range(1, 4):
        for d in range(3):
            c, f = g.faces(L, d), g.faces(L + 1, d)
            assert np.array_equal(c, f[::2])


@pytest.mark.parametrize("stretch", [0, 1])
def test_wedge_volume_closed_form(stretch):
    xmin, xmax = (0.1, math.pi / 6, 0.3), (2.0, 5 * math.pi / 6, 1.9)
    g = O.Grid(n=(24, 8, 16), nb=(12, 8, 8), stretch=stretch, xmin=xmin, xmax=xmax,
               bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_OUTFLOW),
               bc_hi=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_OUTFLOW))
    exact = (xmax[0] ** 3 - xmin[0] ** 3) / 3 * (math.cos(xmin[1]) - math.cos(xmax[1])) * (xmax[2] - xmin[2])
    assert abs(g.total_volume() - exact) / exact < 1e-13


def _mean_index(lo, hi, weight, frac):
    num = integrate.quad(lambda x: frac(x) * weight(x), lo, hi, epsabs=0, epsrel=1e-12)[0]
    den = integrate.quad(weight, lo, hi, epsabs=0, epsrel=1e-12)[0]
    return num / den, den


@pytest.mark.parametrize("stretch", [0, 1])
def test_prolongation_offsets_by_quadrature(stretch):
    """delta_child = volume-weighted mean index coordinate of the child minus
    that of the parent (index coordinate in parent-cell units; linear in
    log r on the stretched grid, in r otherwise, in theta, in phi)."""
    g = O.Grid(n=(12, 8, 8), nb=(12, 8, 8), stretch=stretch, max_level=2,
               xmin=(0.1, math.pi / 6, 0), xmax=(2.0, 5 * math.pi / 6, 2 * math.pi))
    for d, weight in ((0, lambda r: r * r), (1, math.sin), (2, lambda p: 1.0)):
        fc = g.faces(1, d)
        off = g.offsets(1, d)
        for Ic in (0, 3, 7):
            a, b = fc[Ic], fc[Ic + 1]
            if d == 0 and stretch:
                frac = lambda x, a=a, b=b: math.log(x / a) / math.log(b / a) - 0.5
            else:
                frac = lambda x, a=a, b=b: (x - a) / (b - a) - 0.5
            m = np.sqrt(a * b) if (d == 0 and stretch) else 0.5 * (a + b)
            xp, _ = _mean_index(a, b, weight, frac)
            x0, _ = _mean_index(a, m, weight, frac)
            x1, _ = _mean_index(m, b, weight, frac)
            assert abs(off[Ic, 0] - (x0 - xp)) < 1e-11
            assert abs(off[Ic, 1] - (x1 - xp)) < 1e-11


def test_cartesian_offsets_are_quarters():
    g = O.Grid(geometry=1, n=(8, 8, 8), nb=(8, 8, 8), max_level=2, xmin=(0, 0, 0),
               xmax=(1, 1, 1), bc_lo=(0, 0, 0), bc_hi=(0, 0, 0))
    for d in range(3):
        off = g.offsets(1, d)
        assert np.all(off[:, 0] == -0.25) and np.all(off[:, 1] == 0.25)

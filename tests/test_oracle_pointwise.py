"""Oracle pointwise pins: state conversion, fast speed limits, limiter,
flux consistency, Loehner estimator special cases, cone-CME geometry."""
import math

import numpy as np
import pytest

import oracle as O
from golden_io import load
from paper_2211_12867_gb300 import inputs as I

P = load("paper_numbers.txt")


def test_prim_cons_roundtrip():
    rng = np.random.default_rng(1)
    for _ in range(50):
        W = np.concatenate([[rng.uniform(0.1, 3)], rng.normal(size=3), [rng.uniform(0.1, 3)],
                            rng.normal(size=3)])
        U = O.prim2cons(W, 1.5)
        assert np.allclose(O.cons2prim(U, 1.5), W, rtol=1e-13, atol=1e-13)
        # e = p/(g-1) + rho v^2/2 + B^2/2 for a state at rest without field
    U = O.prim2cons([2.0, 0, 0, 0, 3.0, 0, 0, 0], 1.5)
    assert U[4] == 6.0


def test_fast_speed_limits():
    g = 5.0 / 3.0
    # B = 0: sound speed
    W = np.array([2.0, 0, 0, 0, 3.0, 0, 0, 0])
    assert abs(O.fast_speed(W, 0, g) - math.sqrt(g * 3.0 / 2.0)) < 1e-15
    # B perpendicular to the direction: sqrt(a^2 + b^2)
    W = np.array([2.0, 0, 0, 0, 3.0, 0, 4.0, 0])
    assert abs(O.fast_speed(W, 0, g) - math.sqrt(g * 1.5 + 16.0 / 2.0)) < 1e-14
    # B along the direction: max(a, b_n)
    W = np.array([2.0, 0, 0, 0, 3.0, 4.0, 0, 0])
    assert abs(O.fast_speed(W, 0, g) - max(math.sqrt(g * 1.5), math.sqrt(8.0))) < 1e-14
    W = np.array([2.0, 0, 0, 0, 30.0, 0.5, 0, 0])
    assert abs(O.fast_speed(W, 0, g) - math.sqrt(g * 15.0)) < 1e-14


def test_mc_limiter_cases():
    assert O.mc_slope(1.0, 2.0, 3.0) == 1.0          # linear data: exact slope
    assert O.mc_slope(1.0, 2.0, 1.5) == 0.0          # extremum
    assert O.mc_slope(0.0, 0.1, 3.0) == 0.2          # 2 x the small side
    assert O.mc_slope(0.0, 1.0, 1.5) == 0.75         # central difference
    assert O.mc_slope(3.0, 2.0, 1.0) == -1.0         # sign
    assert O.mc_slope(1.0, 1.0, 5.0) == 0.0          # flat side


def test_tvdlf_consistency_and_symmetry():
    rng = np.random.default_rng(2)
    for d in range(3):
        W = np.array([1.3, 0.2, -0.4, 0.7, 0.9, 0.5, -0.3, 0.8])
        F = O.tvdlf(W, W, d, 1.5)
        # equal states: mass flux rho v_n, normal induction flux zero
        assert abs(F[0] - W[0] * W[1 + d]) < 1e-15
        assert F[5 + d] == 0.0
        # static field-free state: flux is the pressure in the normal momentum
        S = np.array([1.0, 0, 0, 0, 0.7, 0, 0, 0])
        Fs = O.tvdlf(S, S, d, 1.5)
        e = np.zeros(8)
        e[1 + d] = 0.7
        assert np.allclose(Fs, e, atol=1e-16)
        # mirror symmetry: reflecting v_n and B_n negates the mass flux
        WL = np.array([1.0, *rng.normal(size=3), 1.1, *rng.normal(size=3)])
        WR = np.array([0.8, *rng.normal(size=3), 0.7, *rng.normal(size=3)])
        mir = lambda w: np.array([w[k] * (-1 if k in (1 + d, 5 + d) else 1) for k in range(8)])
        F1 = O.tvdlf(WL, WR, d, 1.5)
        F2 = O.tvdlf(mir(WR), mir(WL), d, 1.5)
        assert abs(F1[0] + F2[0]) < 1e-14
        assert abs(F1[4] + F2[4]) < 1e-14


def test_loehner_special_cases():
    eps = 0.01
    # linear field: E = 0
    assert O.loehner([1.0, 2.0, 3.0], 2.0 + 0.0, [3.0, 2.0, 1.0], eps) >= 0.0
    assert O.loehner([1.0, 1.0, 1.0], 2.0, [3.0, 3.0, 3.0], eps) == 0.0
    # unit step next to the cell, flat elsewhere: E = 1/(1+eps)
    assert O.loehner([0.0, 0.0, 0.0], 0.0, [1.0, 0.0, 0.0], eps) == pytest.approx(1.0 / 1.01, rel=1e-15)
    rng = np.random.default_rng(3)
    for _ in range(200):
        um, up = rng.uniform(0.1, 5, 3), rng.uniform(0.1, 5, 3)
        E = O.loehner(um, rng.uniform(0.1, 5), up, eps)
        assert 0.0 <= E <= 1.0


def _cme(hw_deg, v_kms):
    return dict(t_start=0.0, t_max=1e9, colat=math.pi / 2, lon=1.0,
                half_width=math.radians(hw_deg), v=I.kms(v_kms))


@pytest.mark.parametrize("hw,v,hours", [(P["cme_half_width_deg"], P["cme_speed_kms"], 4.04),
                                        (30.0, 1000.0, 4.16)])
def test_cone_cme_opening_angle(hw, v, hours):
    """Eqs. 1-3: theta(0) = 0; max theta = omega/2 at R_c = sqrt(R^2 - r_half^2);
    theta returns to 0 at t = 2 r_half / v (Table 2: 4.04 h; 30 deg, 1000 km/s: 4.16 h)."""
    c = _cme(hw, v)
    R = 0.1
    rh = R * math.sin(c["half_width"])
    # at t = 0 the argument of arccos is 1 up to rounding: zero opening, or none
    th0, _ = O.cme_eval(**c, R=R, t=0.0, pcolat=0, plon=0)
    assert th0 < 1e-7
    th1, _ = O.cme_eval(**c, R=R, t=1e-6 * rh / c["v"], pcolat=0, plon=0)
    assert 0.0 < th1 < 0.05 * c["half_width"]
    t_end = 2 * rh / c["v"]
    assert abs(t_end / I.hours(1.0) - hours) < 0.01
    # just before the end the sphere still intersects; just after it does not
    assert O.cme_eval(**c, R=R, t=t_end * (1 - 1e-6), pcolat=0, plon=0)[0] >= 0
    assert O.cme_eval(**c, R=R, t=t_end * (1 + 1e-6), pcolat=0, plon=0)[0] < 0
    t_max = (math.sqrt(R * R - rh * rh) - (R - rh)) / c["v"]
    th, _ = O.cme_eval(**c, R=R, t=t_max, pcolat=0, plon=0)
    assert abs(th - c["half_width"]) < 1e-7
    ts = np.linspace(0, t_end * 0.999, 400)
    ths = np.array([O.cme_eval(**c, R=R, t=t, pcolat=0, plon=0)[0] for t in ts])
    assert ths.max() <= c["half_width"] + 1e-12


def test_cone_cme_mask_matches_sphere_intersection():
    """A boundary point at angular distance d from the axis lies inside the
    CME sphere (centre at R_c on the axis, radius r_half) iff d <= theta(t)."""
    rng = np.random.default_rng(4)
    R = 0.1
    for _ in range(20):
        c = dict(t_start=0.0, t_max=1e9, colat=rng.uniform(0.5, 2.5), lon=rng.uniform(0, 6),
                 half_width=math.radians(rng.uniform(15, 45)), v=I.kms(rng.uniform(600, 1800)))
        rh = R * math.sin(c["half_width"])
        t = rng.uniform(0, 2 * rh / c["v"])
        Rc = t * c["v"] + R - rh
        axis = np.array([math.sin(c["colat"]) * math.cos(c["lon"]),
                         math.sin(c["colat"]) * math.sin(c["lon"]), math.cos(c["colat"])])
        for _ in range(50):
            th, ph = rng.uniform(0.3, 2.8), rng.uniform(0, 2 * math.pi)
            p = R * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            inside = np.sum((p - Rc * axis) ** 2) <= rh * rh
            op, d = O.cme_eval(**c, R=R, t=t, pcolat=th, plon=ph)
            if abs(np.sum((p - Rc * axis) ** 2) - rh * rh) > 1e-12:
                assert inside == (d <= op)


def test_cme_window():
    c = _cme(30, 1000)
    c["t_start"], c["t_max"] = 1.0, I.hours(6.0)
    assert O.cme_eval(**c, R=0.1, t=0.99, pcolat=0, plon=0)[0] < 0
    assert O.cme_eval(**c, R=0.1, t=1.0 + I.hours(1.0), pcolat=0, plon=0)[0] > 0

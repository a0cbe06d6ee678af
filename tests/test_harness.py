"""Arrival-time analysis on synthetic series with a known crossing."""
import math

import numpy as np

from paper_2211_12867_gb300 import harness as H
from paper_2211_12867_gb300 import inputs as I


def test_arrival_of_a_tanh_shock():
    # background 4.0 (400 km/s), shock of 3.0 (300 km/s) centred at t0 with
    # width w: v - v_bg crosses 0.5 (50 km/s) where tanh((t-t0)/w) = -2/3
    t0, w = I.hours(50.0), I.hours(0.5)
    t = np.arange(0.0, I.hours(100.0), I.hours(1 / 6))
    vbg = np.full_like(t, 4.0)
    v = vbg + 1.5 * (1 + np.tanh((t - t0) / w))
    exact = t0 + w * math.atanh(0.5 / 1.5 - 1)
    got = H.arrival_time(t, v, vbg)
    # linear interpolation of a tanh over 10-min samples: error << 10 min
    assert abs(got - exact) < I.hours(0.05)


def test_no_arrival_and_first_sample():
    t = np.linspace(0, 1, 11)
    assert H.arrival_time(t, np.zeros(11), np.zeros(11)) is None
    assert H.arrival_time(t, np.ones(11), np.zeros(11)) == 0.0


def test_width_and_peak():
    t = np.arange(0, 48) * I.hours(1.0)
    v = np.full(48, 4.0)
    v[10:] = 6.0
    v[14] = 7.5
    vbg = np.full(48, 4.0)
    a = H.arrival_time(t, v, vbg)
    assert abs(a - I.hours(9.25)) < 1e-12        # crossing 0.5 of a 2.0 jump from 9 h to 10 h
    assert abs(H.shock_width(t, v, a) - (I.hours(14) - a)) < 1e-12
    assert H.peak_speed(t, v, a) == 7.5


def test_earth_moves_at_the_synodic_rate():
    p0 = I.earth_position(0.0, 0.0)
    p1 = I.earth_position(I.days(27.2753), 0.0)
    assert abs(p0[0] - 1.0) < 1e-15 and abs(p0[1] - math.pi / 2) < 1e-15
    # one synodic rotation later the longitude is back (27.2753 d)
    assert abs(((p1[2] - p0[2] + math.pi) % (2 * math.pi)) - math.pi) < 1e-3

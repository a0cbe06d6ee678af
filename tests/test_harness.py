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


# ---------------------------------------------------------------- pre-flag bookkeeping
def _tree(rows):
    return np.array(rows, dtype=np.int32).reshape(-1, 4)


def test_labels_follow_the_region_across_a_regrid():
    # regrid k: two base leaves; between k and k+1 leaf 0 was refined
    tk = _tree([[1, 0, 0, 0], [1, 1, 0, 0]])
    children = [[2, (c >> 2) & 1, (c >> 1) & 1, c & 1] for c in range(8)]
    tk1 = _tree(children + [[1, 1, 0, 0]])
    # one child flagged at k+1 -> the parent region at k is labelled 1
    f = np.zeros(9, dtype=np.int8)
    f[3] = 1
    assert H.next_regrid_labels(tk, tk1, f).tolist() == [1.0, 0.0]
    # the unchanged leaf flagged at k+1 -> itself labelled
    f = np.zeros(9, dtype=np.int8)
    f[8] = 1
    assert H.next_regrid_labels(tk, tk1, f).tolist() == [0.0, 1.0]
    # coarsening flags (-1) are not refinements
    assert H.next_regrid_labels(tk, tk1, -np.ones(9, dtype=np.int8)).tolist() == [0.0, 0.0]
    # k+1 leaf coarser than the k leaves (8 children merged): all 8 labelled
    assert H.next_regrid_labels(tk1, tk, np.array([1, 0], dtype=np.int8)).tolist() == [1.0] * 8 + [0.0]


def test_missed_flag_rate_counts_unmarked_regions():
    tk = _tree([[1, 0, 0, 0], [1, 1, 0, 0], [1, 2, 0, 0]])
    tk1 = tk.copy()
    f1 = np.array([1, 1, 0], dtype=np.int8)
    assert H.missed_flag_rate(tk, np.array([True, False, False]), tk1, f1) == 0.5
    assert H.missed_flag_rate(tk, np.array([True, True, True]), tk1, f1) == 0.0
    assert H.missed_flag_rate(tk, np.array([False, False, True]), tk1, f1) == 1.0
    assert H.missed_flag_rate(tk, np.zeros(3, bool), tk1, np.zeros(3, np.int8)) is None
    # at the finest level a flag cannot act: excluded when max_level is given
    tk2 = _tree([[2, 0, 0, 0], [1, 1, 0, 0]])
    f2 = np.array([1, 1], dtype=np.int8)
    assert H.missed_flag_rate(tk2, np.zeros(2, bool), tk2, f2) == 1.0
    assert H.missed_flag_rate(tk2, np.array([False, True]), tk2, f2, max_level=2) == 0.0


def test_training_pairs_skip_the_finest_level():
    tk = _tree([[2, 0, 0, 0], [1, 1, 0, 0]])
    f1 = np.array([1, 1], dtype=np.int8)
    recs = [{"tree": tk, "feat": np.arange(128, dtype=np.float32).reshape(2, 64), "flags": f1},
            {"tree": tk, "feat": np.zeros((2, 64), np.float32), "flags": f1}]
    X, T = H.training_pairs(recs)
    assert T.tolist() == [1.0, 1.0] and X.shape == (2, 64)
    X, T = H.training_pairs(recs, max_level=2)
    # the level-2 leaf is dropped; the level-1 leaf keeps its refinable label
    assert T.tolist() == [1.0] and X[0, 0] == 64.0


def test_rebalance_repeats_rare_positives():
    X = np.arange(1000, dtype=np.float32).reshape(1000, 1)
    T = np.zeros(1000, np.float32)
    T[[3, 500, 900]] = 1.0
    Xb, Tb = H.rebalance(X, T, cap=600)
    assert len(Tb) == 600 and Tb.sum() == 300
    # every sample is an original pair, positives stay positive
    assert np.all(T[Xb[:, 0].astype(int)] == Tb)
    assert set(Xb[Tb > 0, 0].astype(int)) == {3, 500, 900}


def test_threshold_calibration_and_bias_shift():
    rng = np.random.default_rng(0)
    T = (rng.uniform(size=5000) < 0.02).astype(np.float32)
    # scores: positives mostly above 0.8, negatives spread below 0.9
    prob = np.where(T > 0, rng.uniform(0.75, 1.0, 5000), rng.uniform(0.0, 0.9, 5000))
    t, f = H.calibrate_threshold(prob, T)
    assert 0.8 < t < 0.95 and f > 0.5
    theta = np.zeros(10, np.float32)
    th = H.shift_output_bias(theta, 0.8)
    # sigmoid(z + b') = 1/2 exactly where sigmoid(z + b) = 0.8
    z = math.log(0.8 / 0.2)
    assert abs(z + th[-1]) < 1e-6


def test_missed_refinements_by_level():
    """per level: the share of next-regrid refinements (below the finest
    level) whose region the pre-flags did not mark"""
    tk = _tree([[1, 0, 0, 0], [2, 2, 0, 0], [2, 3, 0, 0], [1, 2, 0, 0]])
    recs = [{"tree": tk, "applied": np.array([1, 0, 1, 0], np.int8), "plain": np.zeros(4, np.int8)},
            {"tree": tk, "applied": np.zeros(4, np.int8), "plain": np.array([1, 1, 1, 1], np.int8)}]
    got = H.missed_by_level(recs, 3, "applied")
    assert got == {1: 0.5, 2: 0.5}
    # at the finest level flags cannot act: that level is not judged
    assert H.missed_by_level(recs, 2, "applied") == {1: 0.5}
    none = [dict(recs[0]), dict(recs[1], plain=np.zeros(4, np.int8))]
    assert H.missed_by_level(none, 3, "applied") == {1: None, 2: None}

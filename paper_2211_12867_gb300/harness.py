"""Run driver: relaxation, cone-CME injection, propagation with regrids and
probes at Earth, and the arrival-time analysis.

The paper relaxes the wind until the slow stream has crossed the domain,
injects the cone CME through the inner boundary (Sect. 2.1, Eqs. 1-4) and
reads time series at Earth (Figs. 1, 3, 6, 9); it reports the shock arrival
time and the shock width, the time from arrival to the peak speed
(Sect. 3.1).  Arrival is read here as the first sample where the radial speed
exceeds the background at the same point by 50 km/s, linearly interpolated to
the crossing; the background is the relaxed state sampled along Earth's path
(steady in the co-rotating frame).  All device work goes through the C ABI
(``icarus.Icarus``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I
from .icarus import IcarusError

CAPACITY = 7   # ICARUS_ERR_CAPACITY


# ---------------------------------------------------------------- analysis
def arrival_time(t, vr, vbg, dv=I.kms(50.0)):
    """First crossing of vr - vbg above dv (linear interpolation between
    samples); None if the series never crosses."""
    t, vr, vbg = (np.asarray(x, dtype=np.float64) for x in (t, vr, vbg))
    ex = vr - vbg - dv
    above = np.nonzero(ex > 0.0)[0]
    if len(above) == 0:
        return None
    k = above[0]
    if k == 0:
        return float(t[0])
    a, b = ex[k - 1], ex[k]
    return float(t[k - 1] + (t[k] - t[k - 1]) * (-a) / (b - a))


def shock_width(t, vr, t_arr, window=None):
    """Time from arrival to the peak radial speed within `window` after it
    (default 24 h)."""
    if t_arr is None:
        return None
    window = I.hours(24.0) if window is None else window
    t, vr = np.asarray(t), np.asarray(vr)
    sel = (t >= t_arr) & (t <= t_arr + window)
    if not np.any(sel):
        return None
    k = np.argmax(np.where(sel, vr, -np.inf))
    return float(t[k] - t_arr)


def peak_speed(t, vr, t_arr, window=None):
    if t_arr is None:
        return None
    window = I.hours(24.0) if window is None else window
    t, vr = np.asarray(t), np.asarray(vr)
    sel = (t >= t_arr) & (t <= t_arr + window)
    return float(np.max(vr[sel])) if np.any(sel) else None


# ---------------------------------------------------------------- learned pre-flagger
def _related(tree_a, tree_b):
    """For each leaf of tree_b, the indices of tree_a leaves overlapping it
    (a regrid changes a region by at most one level: self, parent or the 8
    children)."""
    index = {(int(l), int(i), int(j), int(k)): n for n, (l, i, j, k) in enumerate(tree_a)}
    out = []
    for (l, i, j, k) in tree_b:
        l, i, j, k = int(l), int(i), int(j), int(k)
        hit = []
        if (l, i, j, k) in index:
            hit.append(index[(l, i, j, k)])
        if (l - 1, i >> 1, j >> 1, k >> 1) in index:
            hit.append(index[(l - 1, i >> 1, j >> 1, k >> 1)])
        for c in range(8):
            key = (l + 1, 2 * i + (c >> 2 & 1), 2 * j + (c >> 1 & 1), 2 * k + (c & 1))
            if key in index:
                hit.append(index[key])
        out.append(hit)
    return out


def next_regrid_labels(tree_k, tree_k1, flags_k1, max_level=None):
    """Label of each leaf at regrid k: 1 if the plain estimator flags any
    overlapping leaf for refinement at regrid k+1 (with `max_level`, only
    flagged leaves that can still refine count)."""
    lab = np.zeros(len(tree_k), dtype=np.float32)
    for (l, _, _, _), hits, f in zip(tree_k1, _related(tree_k, tree_k1), flags_k1):
        if f > 0 and (max_level is None or l < max_level):
            lab[hits] = 1.0
    return lab


def missed_flag_rate(tree_k, preflag_k, tree_k1, flags_k1, max_level=None):
    """Fraction of leaves flagged +1 by the plain estimator at regrid k+1 whose
    region was not pre-flagged at regrid k (None if nothing was flagged).
    With `max_level`, only flagged leaves that can still refine count."""
    need = missed = 0
    for (l, _, _, _), hits, f in zip(tree_k1, _related(tree_k, tree_k1), flags_k1):
        if max_level is not None and l >= max_level:
            continue
        if f > 0:
            need += 1
            if not any(preflag_k[h] for h in hits):
                missed += 1
    return (missed / need) if need else None


def missed_by_level(recs, max_level, key):
    """Missed-refinement rate per level over consecutive regrid records
    (tree, pre-flags under `key`, plain flags): the share of the leaves the
    plain estimator flags +1 at regrid k+1 (and that can still refine) whose
    region the pre-flags of regrid k did not flag; {level: rate or None}."""
    need, missed = {}, {}
    for a, b in zip(recs[:-1], recs[1:]):
        pre = a[key] > 0
        for (l, _, _, _), hits, f in zip(b["tree"], _related(a["tree"], b["tree"]), b["plain"]):
            l = int(l)
            if l >= max_level or f <= 0:
                continue
            need[l] = need.get(l, 0) + 1
            if not any(pre[h] for h in hits):
                missed[l] = missed.get(l, 0) + 1
    return {L: (missed.get(L, 0) / need[L] if need.get(L) else None) for L in range(1, max_level)}


def collect_regrids(g, n_regrids, regrid_every, t_stop=np.inf, crit=None):
    """Advance with plain regrids and record, at every regrid, the tree of
    member 0, the features of its leaves and the plain flags."""
    recs = []
    for _ in range(n_regrids):
        g.step(regrid_every, t_stop=t_stop)
        feats = g.mlp_features()
        flags = g.flag_refine(**(crit or {}))
        n0 = g.n_leaves(0)
        recs.append({"tree": g.tree(0), "feat": feats[:n0].copy(), "flags": flags[:n0].copy()})
        g.regrid()
    return recs


def training_pairs(recs, max_level=None):
    """(features at regrid k, label from the plain flags at regrid k+1).
    With `max_level`, leaves already at the finest level (whose flags a
    regrid ignores) are left out and only refinable flags make labels."""
    X, T = [], []
    for a, b in zip(recs[:-1], recs[1:]):
        lab = next_regrid_labels(a["tree"], b["tree"], b["flags"], max_level)
        keep = np.ones(len(lab), bool) if max_level is None else np.asarray(a["tree"])[:, 0] < max_level
        X.append(a["feat"][keep])
        T.append(lab[keep])
    return np.concatenate(X), np.concatenate(T)


def rebalance(X, T, cap=65536, seed=0):
    """Training set with the positives repeated until they are about as many
    as the negatives (refinement labels are rare, and a network trained on
    the raw prior never reaches probability 1/2); at most `cap` samples, a
    seeded subsample of the negatives if needed."""
    rng = np.random.default_rng(seed)
    pos, neg = np.nonzero(T > 0.5)[0], np.nonzero(T <= 0.5)[0]
    if len(pos) == 0 or len(neg) == 0:
        sel = np.arange(len(T))
    else:
        n_neg = min(len(neg), cap // 2)
        neg = np.sort(rng.choice(neg, n_neg, replace=False))
        pos = np.resize(pos, min(n_neg, cap - n_neg))   # repeated in order
        sel = np.concatenate([neg, pos])
        sel = sel[rng.permutation(len(sel))]
    sel = sel[:cap]
    return X[sel], T[sel]


def calibrate_threshold(prob, T):
    """Probability threshold with the best F1 score on (unbalanced) labelled
    pairs: a network trained on a rebalanced set over-predicts the rare
    class at 1/2."""
    prob, T = np.asarray(prob, np.float64), np.asarray(T) > 0.5
    best_t, best_f = 0.5, -1.0
    for t in np.unique(np.quantile(prob, np.linspace(0.5, 0.9999, 400))):
        pred = prob > t
        tp = np.sum(pred & T)
        f = 2.0 * tp / max(1, pred.sum() + T.sum())
        if f > best_f:
            best_t, best_f = float(t), f
    return best_t, best_f


def shift_output_bias(theta, threshold):
    """Parameters whose sigmoid output crosses 1/2 where the original one
    crosses `threshold` (the output bias is the last parameter)."""
    th = np.array(theta, dtype=np.float32, copy=True)
    th[-1] -= np.float32(math.log(threshold / (1.0 - threshold)))
    return th


# ---------------------------------------------------------------- driver
@dataclass
class RunResult:
    times: np.ndarray
    series: np.ndarray          # [member][sample][8] primitives at Earth
    background: np.ndarray      # [member][sample][8]
    arrival: list
    width: list
    peak: list
    steps: int = 0
    regrids: int = 0
    leaves: list = field(default_factory=list)   # leaves per regrid (all members)
    wall_s: float = 0.0
    wall_at: np.ndarray = None  # wall clock [s] since injection at each sample
    capacity_skips: int = 0     # regrids refused for want of blocks

    def wall_to(self, t):
        """Wall clock from injection until simulated time t (interpolated
        between samples); None if t is None."""
        return None if t is None else float(np.interp(t, self.times, self.wall_at))


def advance_to(g, t_target, max_steps=1_000_000, regrid_every=0, crit=None, counters=None,
               on_regrid=None):
    """Step every member until it reaches t_target (scalar or per member;
    regridding every `regrid_every` steps when > 0)."""
    counters = counters if counters is not None else {"steps": 0, "regrids": 0, "leaves": []}
    counters.setdefault("since", 0)
    cells_per_block = int(np.prod(g.block))
    n = 0
    while True:
        k = max(1, regrid_every - counters["since"]) if regrid_every > 0 else 500
        u0 = g.cell_updates()
        t = g.step(k, t_stop=t_target)
        du = g.cell_updates() - u0
        # steps actually taken (a member stops at t_target): from the exact
        # per-member cell-update counters, no regrid in between
        taken = max(int(round(du[m] / (g.n_leaves(m) * cells_per_block))) for m in range(g.n_members))
        n += taken
        counters["steps"] += taken
        counters["since"] += taken
        if regrid_every > 0 and counters["since"] >= regrid_every:
            flags = g.flag_refine(**(crit or {}))
            if on_regrid is not None:
                flags = on_regrid(g, flags)
                g.set_flags(flags)
            try:
                g.regrid()
            except IcarusError as e:
                # the block pool cannot hold the refined tree: the tree (and
                # the state) stay as they are until a later regrid fits
                if e.code != CAPACITY:
                    raise
                counters["capacity_skips"] = counters.get("capacity_skips", 0) + 1
            counters["since"] = 0
            counters["regrids"] += 1
            counters["leaves"].append(g.n_leaves(-1))
        if np.all(t >= np.asarray(t_target)) or n >= max_steps or taken == 0:
            return t


def propagate(g, cmes, *, t_inj, duration, sample=None, earth_lon0=math.pi, regrid_every=0, crit=None,
              on_regrid=None, stop_after_arrival=None, progress=None, max_wall_s=None):
    """Inject one cone CME per member at t_inj and record Earth time series
    every `sample` (default 10 min) for `duration`; returns RunResult.  With
    `stop_after_arrival` (code time), a member stops advancing once its shock
    has arrived and that much time has passed (its later samples repeat the
    last state).  `progress` (a file) receives one line per simulated hour.
    With `max_wall_s`, the run ends early once that much wall clock has
    passed, or once every member has stopped (the series are cut there)."""
    import time as _time
    sample = I.hours(1.0 / 6.0) if sample is None else sample
    nm = g.n_members
    times = t_inj + sample * np.arange(int(round(duration / sample)) + 1)
    pts = np.stack([I.earth_position(t, t_inj, earth_lon0) for t in times])
    bg = np.stack([g.probe(m, pts) for m in range(nm)])
    for m, c in enumerate(cmes):
        g.inject_cone_cme(m, t_start=t_inj, **{k: v for k, v in c.items() if k in
                                               ("t_max", "colat", "lon", "half_width", "v", "rho", "p")})
    series = np.zeros((nm, len(times), 8))
    for m in range(nm):
        series[m, 0] = g.probe(m, pts[:1])[0]
    counters = {"steps": 0, "regrids": 0, "leaves": []}
    wall_at = np.zeros(len(times))
    w0 = _time.perf_counter()
    t_hold = np.full(nm, np.inf)   # time a member stopped at
    for k in range(1, len(times)):
        target = np.minimum(times[k], t_hold)
        advance_to(g, target, regrid_every=regrid_every, crit=crit, counters=counters, on_regrid=on_regrid)
        for m in range(nm):
            series[m, k] = g.probe(m, pts[k:k + 1])[0]
            if stop_after_arrival is not None and not np.isfinite(t_hold[m]):
                a = arrival_time(times[:k + 1], series[m, :k + 1, 1], bg[m, :k + 1, 1])
                if a is not None and times[k] >= a + stop_after_arrival:
                    t_hold[m] = times[k]
        wall_at[k] = _time.perf_counter() - w0
        if progress is not None and int((times[k] - t_inj) / I.hours(1.0)) > int((times[k - 1] - t_inj) / I.hours(1.0)):
            print(f"t = {(times[k] - t_inj) / I.hours(1.0):.1f} h  wall {wall_at[k]:.1f} s  leaves {g.n_leaves(-1)}  "
                  f"held {int(np.sum(np.isfinite(t_hold)))}/{nm}", file=progress, flush=True)
        all_held = stop_after_arrival is not None and bool(np.all(np.isfinite(t_hold)))
        if (max_wall_s is not None and wall_at[k] > max_wall_s) or all_held:
            times, series, bg, wall_at = times[:k + 1], series[:, :k + 1], bg[:, :k + 1], wall_at[:k + 1]
            break
    wall = wall_at[-1]
    arr = [arrival_time(times, series[m, :, 1], bg[m, :, 1]) for m in range(nm)]
    wid = [shock_width(times, series[m, :, 1], a) for m, a in zip(range(nm), arr)]
    pk = [peak_speed(times, series[m, :, 1], a) for m, a in zip(range(nm), arr)]
    return RunResult(times, series, bg, arr, wid, pk, counters["steps"], counters["regrids"],
                     counters["leaves"], wall, wall_at, counters.get("capacity_skips", 0))

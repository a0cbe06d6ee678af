"""The synthetic workloads: grids, relaxation and CME runs.

* wedge   — 512 x 60 x 180 equidistant single-level wedge, 0.1-2 AU.
* amr     — radially stretched 264 x 36 x 96 base grid (q = 20^(1/264),
            12^3 blocks, 528 base blocks; 256 x 30 x 90 as printed does
            not divide into 12^3 blocks), solution AMR up to level 4 with the
            Loehner + speed-gate criterion, regrid every 10 steps.
* ensemble — 32 cone-CME draws on the amr grid, levels 3 or 4 per member.
* learned — the amr grid at level 5 with the learned pre-flagger.
* ladder  — the resolution ladder of the paper's comparison (Sects. 3.1-3.3,
            Tables 1, 4-6): the Low and Middle stretched grids, the Middle
            equidistant grid, and AMR levels 2-5 on the Low stretched base
            grid with the tracer, shock and combined criteria.

Relaxation: the wind runs from the spherical start state until the slow
stream has crossed the domain (reading R14: 10 days for 0.1-2 AU; the paper
used 14 days, Table 2), then the CME is injected (Eqs. 1-4).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import harness as H
from . import inputs as I
from .icarus import FP32_MIXED, FP64, Icarus, IcarusError

X_MIN = (0.1, math.pi / 6, 0.0)
X_MAX = (2.0, 5 * math.pi / 6, 2 * math.pi)
AMR_CELLS = (264, 36, 96)
AMR_BLOCK = (12, 12, 12)
CRIT = dict(e_refine=0.1, e_coarsen=0.0125, eps=0.01, dv=I.kms(50.0))


def amr_grid(n_members=1, max_level=4, precision=FP32_MIXED, max_blocks=60000, cells=AMR_CELLS):
    return Icarus(n_cells=cells, block=AMR_BLOCK, max_level=max_level, stretch=True, x_min=X_MIN, x_max=X_MAX,
                  omega=I.OMEGA, cfl=0.8, divb_cd=0.8, precision=precision, n_members=n_members,
                  max_blocks=max_blocks)


def start_wind(g, seed=0):
    n = g.n_cells
    for m in range(g.n_members):
        wm = I.wind_map(n[1], n[2], X_MIN[1], X_MAX[1], seed=seed, r_in=X_MIN[0])
        g.set_inner_boundary(m, wm)
        rc = I.radial_centres(n[0], X_MIN[0], X_MAX[0], g.desc.radial_stretch)
        G = I.initial_prim(wm, rc, X_MIN[0], 1.5, colat_min=X_MIN[1], colat_max=X_MAX[1])
        g.set_state(m, I.global_to_blocks(G, g.tree(m), g.block), prim=True)


def relax(g, days=10.0):
    """Advance every member to t = `days` (base grid only)."""
    t_end = I.days(days)
    w0 = time.perf_counter()
    while True:
        t = g.step(500, t_stop=t_end)
        if np.all(t >= t_end):
            break
    return t_end, time.perf_counter() - w0


def amr_report(g, res, wall_relax, t_inj, ups0=0.0):
    """Summary of one propagation (JSON-ready); ups0: cell updates before it."""
    ups = float(np.sum(g.cell_updates())) - ups0
    to_h = lambda x: None if x is None else (x - t_inj) / I.hours(1.0)
    return {
        "cell_updates": ups, "wall_s": res.wall_s, "cell_updates_per_s": ups / max(res.wall_s, 1e-9),
        "steps": res.steps, "regrids": res.regrids,
        "leaves_max": int(max(res.leaves)) if res.leaves else g.n_leaves(-1),
        "leaves_mean": float(np.mean(res.leaves)) if res.leaves else float(g.n_leaves(-1)),
        "arrival_h": [to_h(a) for a in res.arrival],
        "shock_width_h": [None if w is None else w / I.hours(1.0) for w in res.width],
        "peak_speed_kms": [None if p is None else p * 100.0 for p in res.peak],
        "relax_wall_s": wall_relax, "status": g.status()[0], "floor_hits": int(g.status()[1]),
        "capacity_skips": res.capacity_skips,
    }


def run_cme(g, cmes, *, t_inj, hours_after=72.0, regrid_every=10, max_levels=None, learned=False,
            sample_min=10.0, stop_hours_after_arrival=None, progress=None, max_wall_s=None, records=None):
    """Inject one CME per member at t_inj and propagate for `hours_after`
    with regrids every `regrid_every` steps and Earth probes every
    `sample_min` minutes (a member stops `stop_hours_after_arrival` after its
    shock arrival when given).  With a list `records`, every regrid appends
    member 0's tree with the plain flags and the flags applied (the plain
    estimator is evaluated on the same state as the learned pre-flags).
    Returns the harness RunResult."""
    from .icarus import FLAG_LEARNED, FLAG_PLAIN
    if max_levels is not None:
        for m, L in enumerate(max_levels):
            g.set_member_max_level(m, int(L))
    crit = dict(CRIT)
    if learned:
        crit["mode"] = FLAG_LEARNED
    hook = None
    if records is not None:
        def hook(gg, flags):
            n0 = gg.n_leaves(0)
            applied = np.array(flags, copy=True)
            plain = gg.flag_refine(**dict(CRIT, mode=FLAG_PLAIN)) if learned else applied
            records.append({"tree": gg.tree(0), "plain": np.array(plain[:n0]), "applied": applied[:n0]})
            return applied
    stop = None if stop_hours_after_arrival is None else I.hours(stop_hours_after_arrival)
    return H.propagate(g, cmes, t_inj=t_inj, duration=I.hours(hours_after), sample=I.hours(sample_min / 60.0),
                       regrid_every=regrid_every, crit=crit, stop_after_arrival=stop, progress=progress,
                       max_wall_s=max_wall_s, on_regrid=hook)


def step_profile(g, n_steps=20, crit=None, repeats=3):
    """Where the time of an AMR step goes: per kernel kind of the step (CUDA
    events, graph replay off while profiling), the host-timed cost of a flag
    and a regrid, and the device time of the first flag + regrid per kernel
    kind (the rest of its wall time is host work and synchronisation);
    returns a JSON-ready dict (per step / per regrid)."""
    from .icarus import PROFILE_KINDS, STEP_KINDS
    g.profile(True)
    g.profile_read()
    g.step(n_steps)
    ms, cnt = g.profile_read()
    tot = float(ms[:STEP_KINDS].sum())
    kinds = {k: {"ms_per_step": float(ms[i]) / n_steps, "launches_per_step": int(cnt[i]) / n_steps,
                 "share": float(ms[i]) / tot if tot > 0 else None} for i, k in enumerate(PROFILE_KINDS[:STEP_KINDS])}
    t_flag = t_regrid = 0.0
    done = 0
    regrid_device = None
    for _ in range(repeats):
        w0 = time.perf_counter()
        g.flag_refine(**(crit or CRIT))
        w1 = time.perf_counter()
        try:
            g.regrid()
        except IcarusError as e:   # block pool full: the regrid changed nothing
            if e.code != H.CAPACITY:
                raise
        w2 = time.perf_counter()
        if regrid_device is None:
            fms, fcnt = g.profile_read()
            regrid_device = {k: float(fms[i]) for i, k in enumerate(PROFILE_KINDS) if fcnt[i] > 0}
            g.profile(False)
        t_flag += w1 - w0
        t_regrid += w2 - w1
        done += 1
    g.profile(False)
    return {"kernels_ms_per_step": tot / n_steps, "kernels": kinds, "leaves": g.n_leaves(-1),
            "flag_ms": 1e3 * t_flag / done, "regrid_ms": 1e3 * t_regrid / done,
            "flag_regrid_device_ms": regrid_device}


def run_learned_window(g, *, n_regrids, regrid_every, max_level, crit=None, t_stop=np.inf):
    """Advance with the learned pre-flags applied at every regrid and, for the
    same states, record the plain estimator's flags; returns per-regrid
    records and the missed-flag rates of the learned and of the plain
    pre-flags against the next regrid's plain refinements (refinable leaves
    only: below `max_level`)."""
    from .icarus import FLAG_LEARNED, FLAG_PLAIN
    crit = dict(crit or CRIT)
    recs, steps = [], 0
    w0 = time.perf_counter()
    for _ in range(n_regrids):
        u0 = g.cell_updates()
        g.step(regrid_every, t_stop=t_stop)
        steps += regrid_every
        n0 = g.n_leaves(0)
        plain = g.flag_refine(**crit, mode=FLAG_PLAIN)[:n0].copy()
        learned = g.flag_refine(**crit, mode=FLAG_LEARNED)[:n0].copy()   # stays set for the regrid
        recs.append({"tree": g.tree(0), "plain": plain, "learned": learned, "leaves": g.n_leaves(-1)})
        g.regrid()
    wall = time.perf_counter() - w0
    mp, ml = [], []
    for a, b in zip(recs[:-1], recs[1:]):
        x = H.missed_flag_rate(a["tree"], a["plain"] > 0, b["tree"], b["plain"], max_level)
        y = H.missed_flag_rate(a["tree"], a["learned"] > 0, b["tree"], b["plain"], max_level)
        if x is not None:
            mp.append(x)
            ml.append(y)
    return {"regrids": n_regrids, "regrid_every": regrid_every, "wall_s": wall,
            "leaves": [r["leaves"] for r in recs],
            "extra_preflags": int(sum(int((r["learned"] > 0).sum() - (r["plain"] > 0).sum()) for r in recs)),
            "missed_refinable_plain": float(np.mean(mp)) if mp else None,
            "missed_refinable_learned": float(np.mean(ml)) if ml else None, "judged_regrids": len(mp)}


# ---- resolution ladder (Table 1 grids; Sects. 3.1-3.3) ----
LADDER_GRIDS = {
    # name: (cells r, theta, phi), radially stretched, block
    "low_str": ((60, 32, 96), True, (12, 8, 12)),
    "middle_str": ((120, 64, 192), True, (12, 8, 12)),
    "middle_eq": ((600, 64, 192), False, (24, 16, 48)),
}


def ladder_grid(name, max_level=1, precision=FP32_MIXED, tracer=False, max_blocks=60000):
    cells, stretch, block = LADDER_GRIDS[name]
    return Icarus(n_cells=cells, block=block, max_level=max_level, stretch=stretch, x_min=X_MIN, x_max=X_MAX,
                  omega=I.OMEGA, cfl=0.8, divb_cd=0.8, precision=precision, max_blocks=max_blocks,
                  tracer=tracer)


def ladder_crit(kind):
    """refinement criterion of a ladder run: 'shock' (Sect. 3.2: div v < 0 in
    the Earth and CME windows), 'tracer' (Sect. 3.1: X > 0, no windows) or
    'combined' (Sect. 3.3: either, in the windows)"""
    from .icarus import FLAG_COMBINED, FLAG_SHOCK, FLAG_TRACER, SHOCK_WINDOWS
    if kind == "shock":
        return dict(mode=FLAG_SHOCK, div_thr=0.0, windows=SHOCK_WINDOWS)
    if kind == "tracer":
        return dict(mode=FLAG_TRACER, x_thr=0.0, windows=(0.0, 0.0, 0.0))
    if kind == "combined":
        return dict(mode=FLAG_COMBINED, x_thr=0.0, div_thr=0.0, windows=SHOCK_WINDOWS)
    raise ValueError(kind)


def run_ladder_case(grid, kind=None, max_level=1, *, relax_days=10.0, hours_after=60.0, regrid_every=10,
                    precision=FP32_MIXED, earth_lon0=math.pi, max_blocks=60000):
    """One rung: relax the seeded wind on the base grid, inject the cone CME
    of the 512 x 60 x 180 workload, propagate with Earth probes every 10
    minutes (regridding with criterion `kind` when max_level > 1); returns a
    JSON-ready report with the wall clock from injection to the end and to
    the shock's arrival."""
    tracer = kind in ("tracer", "combined")
    g = ladder_grid(grid, max_level=max_level, precision=precision, tracer=tracer, max_blocks=max_blocks)
    # the floors of the CME's trailing near-vacuum are counted, not budgeted:
    # on a small refined region they can be a large share of a step's cells
    g.set_floor_budget(0.0)
    start_wind(g)
    t_inj, wall_relax = relax(g, relax_days)
    g.set_earth(0, 0.5 * math.pi, earth_lon0, t_inj, I.OMEGA_SYN)
    ups0 = float(np.sum(g.cell_updates()))
    crit = ladder_crit(kind) if max_level > 1 else None
    try:
        res = H.propagate(g, [I.cme_config2(seed=0, earth_lon=earth_lon0)], t_inj=t_inj,
                          duration=I.hours(hours_after), regrid_every=regrid_every if max_level > 1 else 0,
                          crit=crit, earth_lon0=earth_lon0)
    except IcarusError as e:
        word, hits = g.status()
        out = {"grid": grid, "max_level": max_level, "criterion": kind, "error": str(e), "status_word": word,
               "floor_hits": int(hits), "leaves": g.n_leaves(-1)}
        del g
        return out
    rep = amr_report(g, res, wall_relax, t_inj, ups0)
    rep.update({"grid": grid, "cells": list(LADDER_GRIDS[grid][0]), "stretched": LADDER_GRIDS[grid][1],
                "max_level": max_level, "criterion": kind, "time_to_arrival_s": res.wall_to(res.arrival[0]),
                "relax_days": relax_days, "hours_after_injection": hours_after})
    del g
    return rep

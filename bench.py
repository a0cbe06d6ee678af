"""Benchmark of the Icarus MHD update on GB300.

Workload (N = 1): the 512 x 60 x 180 single-level spherical wedge over
0.1-2 AU, +-60 deg, 360 deg, with the seeded inner-boundary wind and a cone
CME (30 deg half width, 1000 km/s) being injected, in the FP32 mode with FP64
pressure islands (or FP64 with --precision fp64).  A step is one full
midpoint predictor-corrector step of every cell (ghost fills, two stage
sweeps with cleaning, CFL reduction); the metric is cell-updates per second.

Timed region: K steps replayed from the CUDA graph, bracketed by CUDA events
on the library's stream (inputs resident in HBM; the state, 0.2-0.35 GB, is
larger than L2).  A second pass of K steps with per-launch events gives the
average duration of each kernel for the roofline of the dominant kernel.  The
end-to-end figure drives the same K steps through the public API from pinned
host buffers: the initial state uploaded, every step's stop times sent and
member times read back, the Earth probe read back every step, the final state
downloaded.

--impl reference times the FP64 CPU oracle (test infrastructure, not the
product) on a bounded sample of the same workload on the host cores.

Multi-GPU (torchrun, N > 1): every rank runs an independent replica of the
workload (weak scaling); ranks meet at barriers and the slowest rank's time
is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2211_12867_gb300 import inputs as I  # noqa: E402

N_CELLS = (512, 60, 180)
BLOCK = (64, 60, 180)
X_MIN = (0.1, math.pi / 6, 0.0)
X_MAX = (2.0, 5 * math.pi / 6, 2 * math.pi)
WORKLOAD = "wedge512x60x180_cme"
BYTES_PER_CELL_STEP = {"f32": 160, "f64": 320}          # read U, write U*, read U*, read U, write U
BYTES_PER_CELL_CORRECTOR = {"f32": 96, "f64": 192}       # read U*, read U, write U^{n+1}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="icarus", choices=["icarus", "reference"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--skip-cpu-baseline", action="store_true")
    p.add_argument("--islands", default="0.002,0.1",
                   help="FP32 mode: FP64 pressure where p < a*e or p < b*B^2/2 ('a,b')")
    p.add_argument("--tile", default="", help="force the stage tile 'tile_theta,tile_phi,r_segment'")
    p.add_argument("--workload", default="wedge",
                   choices=["wedge", "amr", "ensemble", "tt1au", "learned5", "series", "ladder"],
                   help="amr / ensemble / tt1au: stretched AMR CME runs (one JSON line of their own)")
    p.add_argument("--members", type=int, default=32)
    p.add_argument("--max-blocks", type=int, default=60000)
    p.add_argument("--train-regrids", type=int, default=60)
    p.add_argument("--train-draws", type=int, default=3, help="tt1au: CME draws the pre-flagger is trained on")
    p.add_argument("--batch", type=int, default=8, help="tt1au: members of the batched learned arm")
    p.add_argument("--window-regrids", type=int, default=60, help="learned5: regrids after injection")
    p.add_argument("--arms", default="fp32_learned,fp32_plain,fp64_plain,learned,plain",
                   help="tt1au arms (fp32_learned, fp32_learned_batch, fp32_plain, fp64_plain); learned5 arms "
                        "(learned, plain)")
    p.add_argument("--max-level", type=int, default=4)
    p.add_argument("--hours", type=float, default=72.0)
    p.add_argument("--relax-days", type=float, default=10.0)
    p.add_argument("--profile-range", action="store_true",
                   help="amr: end with one step between cudaProfilerStart and cudaProfilerStop")
    p.add_argument("--regrid-every", type=int, default=10)
    p.add_argument("--max-wall", type=float, default=None,
                   help="ensemble / tt1au FP64 arm: end the propagation after this many wall-clock seconds "
                        "(reported with the simulated hours reached)")
    p.add_argument("--rungs", default="low_str,middle_str,middle_eq,shock2,shock3,shock4,shock5,tracer2,tracer3,"
                   "combined2,combined3,combined4,combined5",
                   help="ladder: the single-level grids and <criterion><level> AMR runs on the Low stretched grid")
    p.add_argument("--mode", default="full", choices=["full", "kernel"],
                   help="kernel: set up and run warmup + steps only (for profiler captures)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def setup_grid(precision, seed=0):
    from paper_2211_12867_gb300.icarus import FP32_MIXED, FP64, Icarus
    g = Icarus(n_cells=N_CELLS, block=BLOCK, x_min=X_MIN, x_max=X_MAX, omega=I.OMEGA, cfl=0.8, divb_cd=0.8,
               precision=FP32_MIXED if precision == "fp32" else FP64)
    wm = I.wind_map(N_CELLS[1], N_CELLS[2], X_MIN[1], X_MAX[1], seed=seed, r_in=X_MIN[0])
    g.set_inner_boundary(0, wm)
    rc = I.radial_centres(N_CELLS[0], X_MIN[0], X_MAX[0], 0)
    G = I.initial_prim(wm, rc, X_MIN[0], 1.5, colat_min=X_MIN[1], colat_max=X_MAX[1])
    W = I.global_to_blocks(G, g.tree(0), BLOCK)
    g.set_state(0, W, prim=True)
    cme = dict(I.cme_config2(seed=seed), t_start=0.0)
    g.inject_cone_cme(0, **cme)
    return g, W, wm, cme


def profile_figure(prec_tag, key):
    """A per-launch figure of the corrector (`traffic_bytes_per_launch`:
    dram__bytes_read + write; `warp_inst_per_launch`: inst_executed;
    `fp64_flop_per_launch`: 2 x DFMA + DADD + DMUL thread instructions) from
    the committed ncu summary, if it was taken on the current stage-kernel
    source and precision; None otherwise."""
    path = os.path.join(ROOT, "profiles", f"k_stage_corrector_wedge512_{'fp32' if prec_tag == 'f32' else 'fp64'}.md")
    src = os.path.join(ROOT, "paper_2211_12867_gb300", "csrc", "k_stage.cu")
    try:
        text = open(path).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m = re.search(r"sha256\[:16\] = `([0-9a-f]{16})`", text)
        t = re.search(key + r" = (\d+)", text)
        if not m or not t or m.group(1) != h:
            return None
        return float(t.group(1))
    except OSError:
        return None


def roofline_traffic(prec_tag):
    return profile_figure(prec_tag, "traffic_bytes_per_launch")


def alu_peaks():
    """measured FMA throughput of this GPU (TFLOP/s): FP64, FP32 (the better
    of scalar and packed pairs)"""
    from paper_2211_12867_gb300.icarus import alu_peak
    return {"fp64_tflops": alu_peak(0) / 1e12, "fp32_tflops": max(alu_peak(1), alu_peak(2)) / 1e12,
            "fp32_scalar_tflops": alu_peak(1) / 1e12, "how": "eight independent FMA chains per thread, "
            "8 CTAs of 256 threads per SM, best of 5 (icarus_alu_peak)"}


def _oracle_sample():
    """The bounded CPU sample of the headline workload: the inner 64 radial
    cells of the same wedge (64 x 60 x 180), same wind, start state and CME,
    on the FP64 oracle (all host cores)."""
    import oracle as O
    n = (64, 60, 180)
    r_out = X_MIN[0] + (X_MAX[0] - X_MIN[0]) * 64 / N_CELLS[0]
    g = O.Grid(n=n, nb=(16, 12, 12), xmin=X_MIN, xmax=(r_out, X_MAX[1], X_MAX[2]), omega=I.OMEGA, cfl=0.8,
               divb_cd=0.8)
    wm = I.wind_map(n[1], n[2], X_MIN[1], X_MAX[1], seed=0)
    g.set_boundary_map(wm)
    rc = I.radial_centres(N_CELLS[0], X_MIN[0], X_MAX[0], 0)[:64]
    G = I.initial_prim(wm, rc, X_MIN[0], 1.5, colat_min=X_MIN[1], colat_max=X_MAX[1])
    g.set_state(I.global_to_blocks(G, g.tree(), (16, 12, 12)), prim=True)
    g.set_cme(t_start=0.0, **I.cme_config2(seed=0))
    return g, 64 * 60 * 180, O.max_threads()


def cpu_baseline(seconds, precision_tag):
    """Oracle rate on the bounded sample, stepped for about `seconds`."""
    g, cells, cores = _oracle_sample()
    t0 = time.perf_counter()
    steps = 0
    while True:
        g.advance(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": cells * steps / el, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} step(s) of the inner 64x60x180 cells of the 512x60x180 wedge (FP64 oracle, "
                      f"{el:.1f} s)"}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each step is one oracle step of the bounded sample; W untimed steps, then
    K timed ones (at most as many as fit in about 120 s; the count is in
    `sample`)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, cells, cores = _oracle_sample()
    for _ in range(args.warmup):
        g.advance(1)
    t0 = time.perf_counter()
    steps = 0
    while steps < max(1, args.steps):
        g.advance(1)
        steps += 1
        if time.perf_counter() - t0 > 120.0:
            break
    el = time.perf_counter() - t0
    value = cells * steps / el
    sample = (f"{steps} timed step(s) after {args.warmup} warm-up step(s) of the inner 64x60x180 cells of the "
              f"512x60x180 wedge (FP64 oracle, {el:.1f} s)")
    cb = {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle", "sample": sample}
    line = {"metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / steps,                      # measured: one step of the sample
            "ms_per_step_full_grid_extrapolated": 1e3 * int(np.prod(N_CELLS)) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": int(np.prod(N_CELLS)), "sample_cells": cells,
                       "sample": sample},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_amr_workload(args):
    """Stretched 264x36x96 grid with AMR (levels <= 4): relax 10 days, inject
    the 512x60x180 workload's cone CME, propagate with regrids every 10 steps
    and Earth probes every 10 minutes.  Prints one JSON line (not the
    headline metric line)."""
    import torch
    from paper_2211_12867_gb300 import workloads as WL
    from paper_2211_12867_gb300.icarus import FP32_MIXED, FP64, set_fp64_islands
    torch.cuda.set_device(0)
    prec = FP32_MIXED if args.precision == "fp32" else FP64
    g = WL.amr_grid(n_members=1, max_level=args.max_level, precision=prec, max_blocks=args.max_blocks)
    if prec == FP32_MIXED:
        set_fp64_islands(g, *(float(x) for x in args.islands.split(",")))
    WL.start_wind(g)
    t_inj, wall_relax = WL.relax(g, args.relax_days)
    cme = I.cme_config2(seed=0)
    ups0 = float(np.sum(g.cell_updates()))
    res = WL.run_cme(g, [cme], t_inj=t_inj, hours_after=args.hours, regrid_every=args.regrid_every)
    rep = WL.amr_report(g, res, wall_relax, t_inj, ups0)
    line = {"workload": "amr264x36x96_L%d" % args.max_level, "precision": args.precision, **rep}
    print(json.dumps(line), flush=True)
    lv = g.tree(0)[:, 0]
    print(json.dumps({"workload": line["workload"], "profile_at_end": WL.step_profile(g),
                      "leaves_by_level": [int((lv == q).sum()) for q in range(1, args.max_level + 1)]}), flush=True)
    if args.profile_range:
        # one more step inside cudaProfilerStart / Stop (ncu --profile-from-start off)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        g.step(1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    return 0


def run_ensemble_workload(args):
    """Ensemble of cone-CME draws on the stretched AMR grid, all members in
    the same launches; members' finest levels 3 or 4 from the draws."""
    import torch
    from paper_2211_12867_gb300 import workloads as WL
    from paper_2211_12867_gb300.icarus import FP32_MIXED
    torch.cuda.set_device(0)
    draws = I.cme_ensemble(args.members)
    g = WL.amr_grid(n_members=args.members, max_level=4, precision=FP32_MIXED, max_blocks=args.max_blocks)
    WL.start_wind(g)
    t_inj, wall_relax = WL.relax(g, args.relax_days)
    ups0 = float(np.sum(g.cell_updates()))
    res = WL.run_cme(g, draws, t_inj=t_inj, hours_after=args.hours, regrid_every=args.regrid_every,
                     max_levels=[d["max_level"] for d in draws], stop_hours_after_arrival=6.0,
                     progress=sys.stderr, max_wall_s=args.max_wall)
    rep = WL.amr_report(g, res, wall_relax, t_inj, ups0)
    name = f"ensemble{args.members}_amr264x36x96"
    rep["simulated_hours"] = float((res.times[-1] - t_inj) / I.hours(1.0))
    rep["arrived"] = int(sum(a is not None for a in res.arrival))
    print(json.dumps({"workload": name, "precision": "fp32", "hours_after_injection": args.hours,
                      "max_levels": [d["max_level"] for d in draws],
                      "speeds_kms": [d["v"] * 100.0 for d in draws], **rep}), flush=True)
    print(json.dumps({"workload": name, "profile_at_end": WL.step_profile(g)}), flush=True)
    return 0


class _Lines:
    """A file-like sink that keeps the last line written (hourly progress)."""

    def __init__(self):
        self.last = None

    def write(self, text):
        if text.strip():
            self.last = text.strip()

    def flush(self):
        pass


def run_tt1au_workload(args):
    """Time to 1 AU: the plain FP64 single instance against the FP32 path with
    the learned pre-flagger (trained on a separate run's regrids) at a doubled
    regrid interval; wall clock from injection to the simulated arrival."""
    import torch
    from paper_2211_12867_gb300 import harness as H
    from paper_2211_12867_gb300 import workloads as WL
    from paper_2211_12867_gb300.icarus import FP32_MIXED, FP64, IcarusError
    torch.cuda.set_device(0)
    L = args.max_level
    # training data: FP32 runs of other CME draws (seeds 7, 8, ...), labels
    # one regrid ahead at the interval the learned run uses
    Xs, Ts = [], []
    for seed in range(7, 7 + args.train_draws):
        g = WL.amr_grid(max_level=L, precision=FP32_MIXED, max_blocks=args.max_blocks)
        WL.start_wind(g)
        t_inj, _ = WL.relax(g, args.relax_days)
        g.inject_cone_cme(0, t_start=t_inj, **I.cme_config2(seed=seed))
        recs = H.collect_regrids(g, n_regrids=args.train_regrids, regrid_every=2 * args.regrid_every,
                                 crit=WL.CRIT)
        x, t = H.training_pairs(recs, max_level=L)
        Xs.append(x)
        Ts.append(t)
        if seed < 6 + args.train_draws:
            del g
    X0, T0 = np.concatenate(Xs), np.concatenate(Ts)
    pos_frac = float(T0.mean())
    X, T = H.rebalance(X0, T0, seed=2)
    g.mlp_set_params(I.mlp_init(5).astype(np.float32))
    g.mlp_dataset_clear()
    g.mlp_dataset_add(X, T)
    w0 = time.perf_counter()
    losses = g.mlp_train(len(T), epochs=100, batch=1024, lr=1e-3, seed=1)
    train_s = time.perf_counter() - w0
    # decision threshold with the best F1 on the unbalanced training pairs,
    # folded into the output bias (the library decides at probability 1/2)
    thr, f1 = H.calibrate_threshold(g.mlp_predict(X0), T0)
    theta = H.shift_output_bias(g.mlp_get_params(), thr)
    del g
    out = {}
    B = args.batch
    for name, prec, learned, every, nm in (("fp32_learned", FP32_MIXED, True, 2 * args.regrid_every, 1),
                                           (f"fp32_learned_batch{B}", FP32_MIXED, True, 2 * args.regrid_every, B),
                                           ("fp32_plain", FP32_MIXED, False, args.regrid_every, 1),
                                           ("fp64_plain", FP64, False, args.regrid_every, 1)):
        if (nm < 2 and name.startswith("fp32_learned_batch")) or name.split("_batch")[0] not in args.arms.split(","):
            continue
        # a level-4 member peaks near 47k leaves: the pool holds that per member
        per_member = 50000 if L >= 4 else 15000
        g = WL.amr_grid(n_members=nm, max_level=L, precision=prec, max_blocks=max(args.max_blocks, per_member * nm))
        if learned:
            g.mlp_set_params(theta)
        WL.start_wind(g)
        t_inj, wall_relax = WL.relax(g, args.relax_days)
        ups0 = float(np.sum(g.cell_updates()))
        # a batch holds nm copies of the same CME run (the time per instance
        # is the batch's wall clock / nm)
        recs = [] if nm == 1 and prec == FP32_MIXED else None
        hourly = _Lines()
        try:
            res = WL.run_cme(g, [I.cme_config2(seed=0)] * nm, t_inj=t_inj, hours_after=args.hours,
                             regrid_every=every, learned=learned, records=recs, progress=hourly,
                             max_wall_s=args.max_wall if prec == FP64 else None)
        except IcarusError as e:
            word, hits = g.status()
            out[name] = {"error": str(e), "status_word": word, "floor_hits": int(hits), "members": nm,
                         "last_progress": hourly.last}
            print(json.dumps({"arm": name, **out[name]}), flush=True)
            del g
            continue
        rep = WL.amr_report(g, res, wall_relax, t_inj, ups0)
        rep["simulated_hours"] = float((res.times[-1] - t_inj) / I.hours(1.0))
        if recs:
            rep["missed_refinable_by_level"] = H.missed_by_level(recs, L, "applied")
            rep["regrid_every"] = every
        rep["members"] = nm
        rep["time_to_arrival_s"] = res.wall_to(res.arrival[0])
        if rep["time_to_arrival_s"] is not None:
            rep["time_to_arrival_per_instance_s"] = rep["time_to_arrival_s"] / nm
        rep["series_at_earth"] = {"t_h": ((res.times - t_inj) / I.hours(1.0)).tolist(),
                                  "vr_kms": (res.series[0, :, 1] * 100.0).tolist(),
                                  "n": res.series[0, :, 0].tolist()}
        out[name] = rep
        print(json.dumps({"arm": name, **{k: v for k, v in rep.items() if k != "series_at_earth"}}), flush=True)
        del g
    arr = lambda k: out[k].get("arrival_h", [None])[0] if k in out else None
    a32, a64 = arr("fp32_learned"), arr("fp64_plain")
    # FP32 against FP64 along the Earth probe series (both plain flags)
    serr = {}
    if all("series_at_earth" in out.get(k, {}) for k in ("fp32_plain", "fp64_plain")):
        s32, s64 = out["fp32_plain"]["series_at_earth"], out["fp64_plain"]["series_at_earth"]
        # both series sample every 10 minutes from the injection; an FP64 run
        # cut by its wall-clock limit is compared over the hours it covers
        nc = min(len(s32["t_h"]), len(s64["t_h"]))
        serr["hours_compared"] = float(s64["t_h"][nc - 1])
        for key in ("vr_kms", "n"):
            x, y = np.asarray(s32[key][:nc]), np.asarray(s64[key][:nc])
            serr[key + "_max_abs_diff"] = float(np.max(np.abs(x - y)))
            serr[key + "_max_rel_diff"] = float(np.max(np.abs(x - y)) / np.max(np.abs(y)))
    print(json.dumps({"workload": f"tt1au_amr264x36x96_L{L}", "train_pairs": int(len(T)),
                      "train_draws": args.train_draws,
                      "label_positive_fraction": pos_frac, "threshold": thr, "train_f1": f1,
                      "train_loss": [float(losses[0]), float(losses[-1])], "train_s": train_s, **out,
                      "fp32_vs_fp64_series": serr,
                      "arrival_diff_h": None if (a32 is None or a64 is None) else abs(a32 - a64)}), flush=True)
    return 0


def run_learned5_workload(args):
    """AMR level 5 with the learned pre-flagger (the level-5 configuration):
    trained on the GPU from the regrids of level-4 runs of other CME draws
    (labels: refinable flags one regrid ahead), then applied at every regrid
    (at twice the plain interval) of a level-5 run of the headline CME; with
    --hours > 0 the run goes on to the shock's arrival at Earth (or
    --max-wall) and a plain level-5 run with regrids every --regrid-every
    steps is the reference.  Reports block counts, the missed refinements per
    level of the learned and of the plain pre-flags, arrival, shock width and
    peak speed of both, and the throughput."""
    import torch
    from paper_2211_12867_gb300 import harness as H
    from paper_2211_12867_gb300 import workloads as WL
    from paper_2211_12867_gb300.icarus import FP32_MIXED
    torch.cuda.set_device(0)
    every = 2 * args.regrid_every
    Xs, Ts = [], []
    for seed in range(7, 7 + args.train_draws):
        g = WL.amr_grid(max_level=4, precision=FP32_MIXED, max_blocks=args.max_blocks)
        WL.start_wind(g)
        t_inj, _ = WL.relax(g, args.relax_days)
        g.inject_cone_cme(0, t_start=t_inj, **I.cme_config2(seed=seed))
        recs = H.collect_regrids(g, n_regrids=args.train_regrids, regrid_every=every, crit=WL.CRIT)
        x, t = H.training_pairs(recs, max_level=4)
        Xs.append(x)
        Ts.append(t)
        if seed < 6 + args.train_draws:
            del g
    X0, T0 = np.concatenate(Xs), np.concatenate(Ts)
    X, T = H.rebalance(X0, T0, seed=2)
    g.mlp_set_params(I.mlp_init(5).astype(np.float32))
    g.mlp_dataset_clear()
    g.mlp_dataset_add(X, T)
    losses = g.mlp_train(len(T), epochs=100, batch=1024, lr=1e-3, seed=1)
    thr, f1 = H.calibrate_threshold(g.mlp_predict(X0), T0)
    theta = H.shift_output_bias(g.mlp_get_params(), thr)
    del g
    head = {"workload": "learned_amr264x36x96_L5", "train_pairs": int(len(T0)), "train_draws": args.train_draws,
            "label_positive_fraction": float(T0.mean()), "threshold": thr, "train_f1": f1,
            "train_loss": [float(losses[0]), float(losses[-1])]}
    if args.hours <= 0:
        g = WL.amr_grid(max_level=5, precision=FP32_MIXED, max_blocks=args.max_blocks)
        g.mlp_set_params(theta)
        WL.start_wind(g)
        t_inj, wall_relax = WL.relax(g, args.relax_days)
        g.inject_cone_cme(0, t_start=t_inj, **I.cme_config2(seed=0))
        ups0 = float(np.sum(g.cell_updates()))
        rep = WL.run_learned_window(g, n_regrids=args.window_regrids, regrid_every=every, max_level=5)
        ups = float(np.sum(g.cell_updates())) - ups0
        t_end = g.step(0)[0]
        print(json.dumps({**head, "hours_after_injection": (t_end - t_inj) / I.hours(1.0), "cell_updates": ups,
                          "cell_updates_per_s": ups / rep["wall_s"], "relax_wall_s": wall_relax,
                          "status": g.status()[0], **rep}), flush=True)
        return 0
    out = {}
    for name, learned, ev in (("learned", True, every), ("plain", False, args.regrid_every)):
        if name not in args.arms.split(","):
            continue
        g = WL.amr_grid(max_level=5, precision=FP32_MIXED, max_blocks=args.max_blocks)
        if learned:
            g.mlp_set_params(theta)
        WL.start_wind(g)
        t_inj, wall_relax = WL.relax(g, args.relax_days)
        ups0 = float(np.sum(g.cell_updates()))
        recs = []
        res = WL.run_cme(g, [I.cme_config2(seed=0)], t_inj=t_inj, hours_after=args.hours, regrid_every=ev,
                         learned=learned, records=recs, max_wall_s=args.max_wall, stop_hours_after_arrival=3.0)
        rep = WL.amr_report(g, res, wall_relax, t_inj, ups0)
        rep.update({"regrid_every": ev, "simulated_hours": float((res.times[-1] - t_inj) / I.hours(1.0)),
                    "time_to_arrival_s": res.wall_to(res.arrival[0]),
                    "missed_refinable_by_level": H.missed_by_level(recs, 5, "applied")})
        out[name] = rep
        print(json.dumps({"arm": name, **rep}), flush=True)
        del g
    diff = {}
    if "learned" in out and "plain" in out:
        for k in ("arrival_h", "peak_speed_kms", "shock_width_h"):
            a, b = out["learned"][k][0], out["plain"][k][0]
            diff[k] = None if (a is None or b is None) else a - b
    print(json.dumps({**head, **out, "learned_minus_plain": diff}), flush=True)
    return 0


def run_series_workload(args):
    """The 512x60x180 wedge in FP64 and in FP32: relax the wind, inject the
    cone CME, probe at Earth every 10 minutes for `--hours`; reports both
    runs' arrival, shock width and peak speed, their wall clocks and the
    FP32 - FP64 difference per probed variable (the FP64 path is the oracle's
    arithmetic on the GPU: it matches the CPU oracle to 1e-10, which is too
    slow for this size)."""
    import torch
    from paper_2211_12867_gb300 import harness as H
    from paper_2211_12867_gb300.icarus import FP32_MIXED, FP64, Icarus
    torch.cuda.set_device(0)
    names = ["rho", "v_r", "v_theta", "v_phi", "p", "B_r", "B_theta", "B_phi"]
    out, series = {}, {}
    for tag, prec in (("fp32", FP32_MIXED), ("fp64", FP64)):
        g = Icarus(n_cells=N_CELLS, block=BLOCK, x_min=X_MIN, x_max=X_MAX, omega=I.OMEGA, cfl=0.8, divb_cd=0.8,
                   precision=prec)
        wm = I.wind_map(N_CELLS[1], N_CELLS[2], X_MIN[1], X_MAX[1], seed=0, r_in=X_MIN[0])
        g.set_inner_boundary(0, wm)
        rc = I.radial_centres(N_CELLS[0], X_MIN[0], X_MAX[0], 0)
        G = I.initial_prim(wm, rc, X_MIN[0], 1.5, colat_min=X_MIN[1], colat_max=X_MAX[1])
        g.set_state(0, I.global_to_blocks(G, g.tree(0), BLOCK), prim=True)
        t_end = I.days(args.relax_days)
        w0 = time.perf_counter()
        while g.step(2000, t_stop=t_end)[0] < t_end:
            pass
        wall_relax = time.perf_counter() - w0
        ups0 = float(np.sum(g.cell_updates()))
        res = H.propagate(g, [I.cme_config2(seed=0)], t_inj=t_end, duration=I.hours(args.hours))
        ups = float(np.sum(g.cell_updates())) - ups0
        to_h = lambda x: None if x is None else x / I.hours(1.0)
        out[tag] = {"arrival_h": to_h(None if res.arrival[0] is None else res.arrival[0] - t_end),
                    "shock_width_h": to_h(res.width[0]), "peak_speed_kms": None if res.peak[0] is None else
                    res.peak[0] * 100.0, "wall_s": res.wall_s, "relax_wall_s": wall_relax, "steps": res.steps,
                    "cell_updates_per_s": ups / res.wall_s, "time_to_arrival_s": res.wall_to(res.arrival[0])}
        series[tag] = res.series[0]
        del g
    a, b = series["fp32"], series["fp64"]
    diff = {n: {"max_abs": float(np.max(np.abs(a[:, v] - b[:, v]))),
                "max_rel_to_range": float(np.max(np.abs(a[:, v] - b[:, v])) / max(np.ptp(b[:, v]), 1e-300))}
            for v, n in enumerate(names)}
    a32, a64 = out["fp32"]["arrival_h"], out["fp64"]["arrival_h"]
    print(json.dumps({"workload": WORKLOAD + "_series", "hours_after_injection": args.hours,
                      "relax_days": args.relax_days, **out, "fp32_minus_fp64_at_earth": diff,
                      "arrival_diff_h": None if a32 is None or a64 is None else abs(a32 - a64)}), flush=True)
    return 0


def run_ladder_workload(args):
    """The resolution ladder of the paper's comparison on the synthetic wind
    and cone CME: single-level Low/Middle stretched and Middle equidistant
    grids (Table 1), then AMR levels 2-5 on the Low stretched base grid with
    the tracer (Sect. 3.1), shock (Sect. 3.2) and combined (Sect. 3.3)
    criteria.  One JSON line per rung, then a summary line with speed-ups
    against the Middle grids (the shape of Tables 4-6)."""
    import torch
    from paper_2211_12867_gb300 import workloads as WL
    from paper_2211_12867_gb300.icarus import FP32_MIXED, FP64
    torch.cuda.set_device(0)
    prec = FP32_MIXED if args.precision == "fp32" else FP64
    out = {}
    for rung in args.rungs.split(","):
        if rung in WL.LADDER_GRIDS:
            rep = WL.run_ladder_case(rung, None, 1, relax_days=args.relax_days, hours_after=args.hours,
                                     precision=prec)
        else:
            kind, level = rung.rstrip("0123456789"), int(rung[len(rung.rstrip("0123456789")):])
            rep = WL.run_ladder_case("low_str", kind, level, relax_days=args.relax_days, hours_after=args.hours,
                                     regrid_every=args.regrid_every, precision=prec, max_blocks=args.max_blocks)
        out[rung] = rep
        print(json.dumps({"rung": rung, **rep}), flush=True)
    summ = {}
    for rung, rep in out.items():
        if "error" in rep:
            summ[rung] = {"error": rep["error"], "status_word": rep["status_word"]}
            continue
        row = {"wall_s": rep["wall_s"], "time_to_arrival_s": rep["time_to_arrival_s"],
               "arrival_h": rep["arrival_h"][0], "shock_width_h": rep["shock_width_h"][0],
               "peak_speed_kms": rep["peak_speed_kms"][0], "leaves_max": rep["leaves_max"],
               "cell_updates_per_s": rep["cell_updates_per_s"]}
        for ref in ("middle_eq", "middle_str"):
            if ref in out and "wall_s" in out[ref] and rep["wall_s"] > 0:
                row[f"speedup_vs_{ref}"] = out[ref]["wall_s"] / rep["wall_s"]
        summ[rung] = row
    print(json.dumps({"workload": "ladder", "precision": args.precision, "hours_after_injection": args.hours,
                      "rungs": summ}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "amr":
        return run_amr_workload(args)
    if args.workload == "ensemble":
        return run_ensemble_workload(args)
    if args.workload == "tt1au":
        return run_tt1au_workload(args)
    if args.workload == "learned5":
        return run_learned5_workload(args)
    if args.workload == "series":
        return run_series_workload(args)
    if args.workload == "ladder":
        return run_ladder_workload(args)
    import torch
    from paper_2211_12867_gb300.replicas import ReplicaGroup
    grp = ReplicaGroup("nccl")
    world, rank, local = grp.world, grp.rank, grp.local
    if world == 1:
        torch.cuda.set_device(0)
    prec_tag = "f32" if args.precision == "fp32" else "f64"
    g, W0, wm, cme = setup_grid(args.precision, seed=grp.seed)
    from paper_2211_12867_gb300.icarus import set_fp64_islands
    isl = tuple(float(x) for x in args.islands.split(","))
    set_fp64_islands(g, *isl)
    tuned = None
    if args.tile:
        tj, tk, seg = (int(x) for x in args.tile.split(","))
        g.set_tile(tj, tk, seg)
        tuned = {"tile": [tj, tk], "r_segment": seg, "ms": None, "forced": True}
    elif not args.no_tune:
        from paper_2211_12867_gb300.autotune import tune
        best, best_ms, _ = tune(g, steps=3)
        tuned = {"tile": [best[0], best[1]], "r_segment": best[2], "ms": round(best_ms, 4)}
    cells = int(np.prod(N_CELLS))
    peaks_alu = alu_peaks() if args.mode != "kernel" else None
    g.step(args.warmup, want_time=False)
    g.stream.synchronize()
    if args.mode == "kernel":
        g.step(args.steps, want_time=False)
        g.stream.synchronize()
        print(json.dumps({"mode": "kernel", "steps": args.steps, "status": g.status()[0]}), flush=True)
        return 0

    def barrier():
        grp.barrier()
        torch.cuda.synchronize()

    # ---- timed region: graph replay ----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        e0.record(g.stream)
        g.step(args.steps, want_time=False)
        e1.record(g.stream)
        e1.synchronize()
    barrier()
    ms = grp.max_over_ranks(e0.elapsed_time(e1))
    value = grp.job_rate(cells * args.steps, ms / 1e3)
    kps = g.kernels_per_step()

    # ---- per-kernel durations (direct launches with event pairs) ----
    g.profile(True)
    g.profile_read()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(g.stream)
    g.step(args.steps, want_time=False)
    p1.record(g.stream)
    kms, kcnt = g.profile_read()
    prof_step_ms = p0.elapsed_time(p1) / args.steps
    g.profile(False)
    from paper_2211_12867_gb300.icarus import PROFILE_KINDS, STEP_KINDS
    kinds = PROFILE_KINDS[:STEP_KINDS]
    per_kernel = {k: {"launches": int(c), "avg_ms": (float(m) / c if c else None), "share": None}
                  for k, m, c in zip(kinds, kms, kcnt)}
    tot = float(kms[:STEP_KINDS].sum())
    for k, m in zip(kinds, kms):
        per_kernel[k]["share"] = float(m) / tot if tot > 0 else None
    hbm, peak_kind = peaks()
    corr_ms = per_kernel["stage_corrector"]["avg_ms"]
    achieved = BYTES_PER_CELL_CORRECTOR[prec_tag] * cells / (corr_ms / 1e3) / 1e9
    traffic = roofline_traffic(prec_tag)
    clocks = clk.summary()
    hbm_roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "k_stage (corrector)", "peak_source": peak_kind,
                "algorithmic_bytes_per_cell": BYTES_PER_CELL_CORRECTOR[prec_tag],
                "step_frac": BYTES_PER_CELL_STEP[prec_tag] * cells / (ms / args.steps / 1e3) / 1e9 / hbm,
                "profiled_ms_per_step": prof_step_ms, "kernels": per_kernel}
    # instruction issue roof of the corrector: warp instructions of one
    # launch (ncu, same source) over SMs x 4 schedulers x the SM clock
    wi = profile_figure(prec_tag, "warp_inst_per_launch")
    props = torch.cuda.get_device_properties(0)
    mhz = clocks.get("sm_mhz") or 2070.0
    issue_peak = props.multi_processor_count * 4 * mhz * 1e6
    hbm_roof["issue"] = None if wi is None else {
        "achieved_warp_inst_per_s": wi / (corr_ms / 1e3), "peak_warp_inst_per_s": issue_peak,
        "frac": wi / (corr_ms / 1e3) / issue_peak, "warp_inst_per_cell": wi / cells,
        "peak_note": "SMs x 4 schedulers x median SM clock of the timed region"}
    if prec_tag == "f64":
        # FP64 mode is bound by the FP64 pipe: executed FP64 flops of one
        # corrector launch (ncu, same source) against the measured FMA peak
        fl = profile_figure(prec_tag, "fp64_flop_per_launch")
        peak64 = peaks_alu["fp64_tflops"]
        ach = None if fl is None else fl / (corr_ms / 1e3) / 1e12
        roofline = {"bound": "fp64", "achieved": ach, "peak": peak64, "unit": "TFLOP/s",
                    "frac": None if ach is None else ach / peak64, "traffic": traffic,
                    "kernel": "k_stage (corrector)", "peak_source": "measured (icarus_alu_peak, FP64 FMA)",
                    "flop_per_cell": None if fl is None else fl / cells, "hbm": hbm_roof, "kernels": per_kernel}
    else:
        roofline = hbm_roof

    # ---- end to end through the public API, host buffers ----
    from paper_2211_12867_gb300.icarus import Icarus  # noqa: F401
    pin_state = torch.empty(W0.size, dtype=torch.float64).pin_memory().numpy().reshape(W0.shape)
    g.get_state(0, out=pin_state)
    pin_out = torch.empty(W0.size, dtype=torch.float64).pin_memory().numpy().reshape(W0.shape)
    t_now = float(g.step(0)[0])
    earth = I.earth_position(t_now, 0.0)
    barrier()
    w0 = time.perf_counter()
    g.set_state(0, pin_state)                       # h2d: the job's input state
    for s in range(args.steps):
        g.step(1, t_stop=np.inf)                    # h2d t_stop, d2h member time
        g.probe(0, earth[None, :])                  # h2d probe point, d2h 8 primitives
    g.get_state(0, out=pin_out)                     # d2h: the job's output state
    torch.cuda.synchronize()
    barrier()
    e2e_s = grp.max_over_ranks(time.perf_counter() - w0)
    state_bytes = W0.size * 8
    e2e = {"value": grp.job_rate(cells * args.steps, e2e_s), "unit": "cell-updates/s",
           "h2d_bytes_per_step": (state_bytes + args.steps * (8 + 24)) / args.steps,
           "d2h_bytes_per_step": (state_bytes + args.steps * (8 + 64)) / args.steps}

    word, floor_hits = g.status()
    cb = None
    if rank == 0 and not args.skip_cpu_baseline:
        cb = cpu_baseline(args.cpu_seconds, prec_tag)
    if rank == 0:
        line = {"metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec_tag,
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": list(N_CELLS), "block": list(BLOCK),
                           "precision": "fp32+fp64-islands" if prec_tag == "f32" else "fp64",
                           "fp64_islands": {"p_over_e": isl[0], "beta": isl[1]} if prec_tag == "f32" else None,
                           "cells": cells, "l2": "state > L2 (no flush needed)", "parallelism": f"replicas{world}",
                           "tuned": tuned},
                "roofline": roofline, "alu_peaks": peaks_alu, "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": kps * args.steps, "clocks": clocks, "status_word": word, "floor_hits": floor_hits}
        print(json.dumps(line), flush=True)
    grp.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

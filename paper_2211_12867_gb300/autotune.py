"""Tile-shape autotuner of the stage kernel.

Sweeps the (theta x phi) tile of the marching CTA and the radial segment
length over the shapes the library instantiates, times a few steps of the
actual workload for each with CUDA events on the library's stream, and
keeps the fastest.  The state is saved before and restored after the sweep,
so tuning does not advance the simulation.
"""
from __future__ import annotations

import itertools

import numpy as np

TILES = [(8, 32), (4, 32), (12, 20), (10, 24), (8, 24), (6, 36), (12, 12), (8, 8)]


def candidates(block):
    nb0, nb1, nb2 = block
    segs = sorted({s for s in (0, nb0, max(8, nb0 // 2), max(8, nb0 // 4), 16, 32) if 0 <= s <= nb0})
    out = []
    for (tj, tk), s in itertools.product(TILES, segs):
        if tk > 2 * nb2 or tj > 2 * nb1:
            continue
        out.append((tj, tk, s))
    return out


def tune(g, steps=3, members=None):
    """Return ((tile_j, tile_k, seg), ms_per_step) of the fastest shape and
    leave it selected on the context."""
    import torch
    saved = [g.get_state(m) for m in range(g.n_members)]
    t0 = g.step(0)
    best, best_ms = None, float("inf")
    results = []
    for tj, tk, seg in candidates(g.block):
        try:
            g.set_tile(tj, tk, seg)
        except Exception:
            continue
        g.step(1, want_time=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        g.step(steps, want_time=False)
        e1.record(g.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        results.append(((tj, tk, seg), ms))
        if ms < best_ms:
            best, best_ms = (tj, tk, seg), ms
        for m in range(g.n_members):
            g.set_state(m, saved[m])
            g.set_time(m, t0[m])
    g.set_tile(*best)
    return best, best_ms, results

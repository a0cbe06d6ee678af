"""Ensembles: several cone-CME members advanced by the same launches (one
block list over all members, per-member time steps), each against its own
oracle; members with different refinement trees and finest levels."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_common import rel_linf
from paper_2211_12867_gb300 import inputs as I
from paper_2211_12867_gb300.icarus import Icarus

pytestmark = pytest.mark.gpu
SPH = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(1.1, 5 * math.pi / 6, 2 * math.pi))


def _oracle(n, nb, max_level=1, stretch=0, x_min=SPH["x_min"], x_max=SPH["x_max"]):
    return O.Grid(n=n, nb=nb, max_level=max_level, stretch=stretch, xmin=x_min, xmax=x_max, omega=I.OMEGA)


def _member_setup(g, m, o, seed):
    n = g.n_cells
    wm = I.wind_map(n[1], n[2], g.desc.x_min[1], g.desc.x_max[1], seed=seed, r_in=g.desc.x_min[0])
    g.set_inner_boundary(m, wm)
    o.set_boundary_map(wm)
    rc = I.radial_centres(n[0], g.desc.x_min[0], g.desc.x_max[0], g.desc.radial_stretch)
    G = I.initial_prim(wm, rc, g.desc.x_min[0], 1.5, colat_min=g.desc.x_min[1], colat_max=g.desc.x_max[1])
    g.set_state(m, I.global_to_blocks(G, g.tree(m), g.block), prim=True)
    o.set_state(g.get_state(m))


def test_three_members_with_different_cmes():
    n, nb = (60, 16, 32), (12, 8, 8)
    g = Icarus(n_cells=n, block=nb, omega=I.OMEGA, n_members=3, **SPH)
    oracles = [_oracle(n, nb) for _ in range(3)]
    draws = I.cme_ensemble(3)
    for m in range(3):
        _member_setup(g, m, oracles[m], seed=m)
        c = {k: draws[m][k] for k in ("t_max", "colat", "lon", "half_width", "v", "rho", "p")}
        g.inject_cone_cme(m, t_start=0.0, **c)
        oracles[m].set_cme(t_start=0.0, **c)
        oracles[m].snapshot_vbg()
    t = g.step(60)
    # the CMEs (different speeds) set different CFL steps: member times diverge
    assert len(set(np.round(t, 12))) == 3
    for m in range(3):
        oracles[m].advance(60)
        assert abs(t[m] - oracles[m].t) / oracles[m].t < 1e-12
        err = rel_linf(g.get_state(m), oracles[m].get_state())
        assert err.max() < 1e-10, (m, err)


def test_members_stop_at_their_own_t_stop():
    n, nb = (60, 16, 32), (12, 8, 8)
    g = Icarus(n_cells=n, block=nb, omega=I.OMEGA, n_members=2, **SPH)
    oracles = [_oracle(n, nb) for _ in range(2)]
    for m in range(2):
        _member_setup(g, m, oracles[m], seed=10 + m)
    d0 = g.dt()
    stops = np.array([3.5 * d0[0], 9.25 * d0[1]])
    t = g.step(40, t_stop=stops)
    assert np.all(t == stops)
    for m in range(2):
        oracles[m].advance(40, stops[m])
        err = rel_linf(g.get_state(m), oracles[m].get_state())
        assert err.max() < 1e-11


def test_members_with_different_trees_and_levels():
    st = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi))
    n, nb = (24, 16, 32), (8, 8, 8)
    g = Icarus(n_cells=n, block=nb, omega=I.OMEGA, n_members=2, max_level=3, stretch=True, max_blocks=3000, **st)
    g.set_member_max_level(0, 2)
    oracles = [_oracle(n, nb, max_level=2, stretch=1, **{"x_min": st["x_min"], "x_max": st["x_max"]}),
               _oracle(n, nb, max_level=3, stretch=1, **{"x_min": st["x_min"], "x_max": st["x_max"]})]
    for m in range(2):
        _member_setup(g, m, oracles[m], seed=20 + m)
    rng = np.random.default_rng(0)
    for rnd in range(2):
        nl = [g.n_leaves(m) for m in range(2)]
        flags = [(rng.random(k) < 0.2).astype(np.int8) for k in nl]
        if rnd == 1:   # member 1: refine its level-2 leaves to level 3
            flags[1][g.tree(1)[:, 0] == 2] = 1
        g.set_flags(np.concatenate(flags))
        g.regrid()
        for m in range(2):
            oracles[m].regrid(flags[m])
            assert np.array_equal(g.tree(m), oracles[m].tree())
    assert g.tree(0)[:, 0].max() <= 2 and g.tree(1)[:, 0].max() == 3
    g.step(8)
    for m in range(2):
        oracles[m].advance(8)
        err = rel_linf(g.get_state(m), oracles[m].get_state())
        assert err.max() < 1e-10, (m, err)

"""Oracle of the CME density tracer (Sect. 3.1) and of the tracer and combined
criteria (Sects. 3.1, 3.3).

Reading of the tracer's transport (the paper only says that a density
tracer is injected with the CME): the tracer is the CME mass fraction X,
stored as rho X, carried by each face's mass flux with X taken from the
face's upwind cell, in both stages of the midpoint predictor-corrector; it
takes X = 1 in the inner-boundary cells the cone CME covers and X = 0
elsewhere.  Pins: X = 1 everywhere stays rho X = rho (the tracer moves with
the mass), a uniform flow turns the update into first-order upwinding whose
midpoint form has a closed form, a periodic box conserves the tracer mass,
tracer only enters through the CME cells and travels at most one cell per
stage, and the flags follow the brute-force definition."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_12867_gb300 import inputs as I

PER = (O.BC_PERIODIC,) * 3


def _cart(n=(16, 8, 8), nb=(8, 4, 4), tracer=1, bc=PER):
    return O.Grid(geometry=1, n=n, nb=nb, xmin=(0, 0, 0), xmax=(1.0, 0.5, 0.5), gamma=5 / 3, omega=0.0,
                  divb_cd=0.0, bc_lo=bc, bc_hi=bc, tracer=tracer)


def _random_prim(g, seed):
    W = np.zeros((g.nleaves, 8) + g.nb)
    for n in range(g.nleaves):
        W[n] = I.random_state(g.nb, seed + n, 5 / 3, v=0.4, b=0.3)
    return W


def test_unit_fraction_follows_the_mass():
    g = _cart()
    g.set_state(_random_prim(g, 10), prim=True)
    g.set_tracer(g.get_state()[:, 0])          # X = 1
    for _ in range(6):
        g.advance(1)
    U = g.get_state()
    assert np.allclose(g.get_tracer(), U[:, 0], rtol=1e-13, atol=0)


def test_tracer_mass_is_conserved_in_a_periodic_box():
    g = _cart()
    g.set_state(_random_prim(g, 20), prim=True)
    rng = np.random.default_rng(3)
    X = rng.uniform(0.0, 1.0, (g.nleaves,) + g.nb)
    g.set_tracer(X * g.get_state()[:, 0])
    V = (1.0 / 16) * (0.5 / 8) * (0.5 / 8)
    m0 = g.get_tracer().sum() * V
    for _ in range(8):
        g.advance(1)
    assert abs(g.get_tracer().sum() * V - m0) <= 1e-14 * m0


def _global_x(g, T):
    n = tuple(b * k for b, k in zip(g.nb, (2, 2, 2)))
    out = np.zeros(n)
    for m, (_, bi, bj, bk) in enumerate(g.tree()):
        out[bi * g.nb[0]:(bi + 1) * g.nb[0], bj * g.nb[1]:(bj + 1) * g.nb[1], bk * g.nb[2]:(bk + 1) * g.nb[2]] = T[m]
    return out


def test_uniform_flow_is_midpoint_upwinding():
    """rho = 1, v = (u, 0, 0), uniform p, B = 0: every face's TVDLF mass flux
    is exactly rho u, so each stage upwinds X with Courant number
    nu = u dt / dx: T^{n+1} = (1 - nu D + nu^2 D^2 / 2) T^n, D the backward
    difference along x."""
    g = _cart(n=(16, 8, 8), nb=(8, 4, 4))
    W = np.zeros((g.nleaves, 8) + g.nb)
    u = 0.7
    W[:, 0], W[:, 1], W[:, 4] = 1.0, u, 1.0
    g.set_state(W, prim=True)
    x = (np.arange(16) + 0.5) / 16
    X0 = np.exp(-((x - 0.4) / 0.1) ** 2) + (x > 0.7)
    T = np.zeros((g.nleaves,) + g.nb)
    for m, (_, bi, bj, bk) in enumerate(g.tree()):
        T[m] = X0[bi * 8:(bi + 1) * 8][:, None, None]
    g.set_tracer(T)
    dt = 0.5 * g.compute_dt()
    nu = u * dt * 16
    want = X0.copy()
    for _ in range(5):
        g.step(dt)
        D = lambda y: y - np.roll(y, 1)
        want = want - nu * D(want) + 0.5 * nu * nu * D(D(want))
    got = _global_x(g, g.get_tracer())
    assert np.allclose(got, want[:, None, None] * np.ones((16, 8, 8)), rtol=0, atol=1e-13)


def test_tracer_enters_through_the_cme_cells_only():
    n, nb = (24, 16, 32), (8, 8, 8)
    g = O.Grid(n=n, nb=nb, xmin=(0.1, math.pi / 6, 0.0), xmax=(1.1, 5 * math.pi / 6, 2 * math.pi),
               omega=I.OMEGA, tracer=1)
    wm = I.wind_map(n[1], n[2], math.pi / 6, 5 * math.pi / 6, seed=0)
    g.set_boundary_map(wm)
    rc = I.radial_centres(n[0], 0.1, 1.1, 0)
    G = I.initial_prim(wm, rc, 0.1, 1.5, omega=I.OMEGA, colat_min=math.pi / 6, colat_max=5 * math.pi / 6)
    g.set_state(I.global_to_blocks(G, g.tree(), nb), prim=True)
    T0 = g.get_tracer()
    assert np.all(T0 == 0)
    g.advance(3)
    assert np.all(g.get_tracer() == 0), "no CME: no tracer"
    cme = dict(I.cme_config2(seed=0), t_start=g.t)
    g.set_cme(**cme)
    k = 2
    g.advance(k)
    T = g.get_tracer()
    U = g.get_state()
    X = T / U[:, 0]
    assert X.max() <= 1.0 + 1e-12 and X.min() >= -1e-12
    glob = np.zeros(n)
    for m, (_, bi, bj, bk) in enumerate(g.tree()):
        glob[bi * 8:(bi + 1) * 8, bj * 8:(bj + 1) * 8, bk * 8:(bk + 1) * 8] = X[m]
    assert glob[0].max() > 0.5
    # two stages per step, one cell per stage: radially ...
    assert np.all(glob[2 * k:] == 0)
    # ... and sideways from the inner-boundary cells the cone can cover
    th = I.angle_centres(n[1], math.pi / 6, 5 * math.pi / 6)
    ph = I.angle_centres(n[2], 0.0, 2 * math.pi)
    a = np.sin(th)[:, None] * math.sin(cme["colat"]) * np.cos(ph[None, :] - cme["lon"]) + \
        np.cos(th)[:, None] * math.cos(cme["colat"])
    reach = np.arccos(np.clip(a, -1, 1)) <= cme["half_width"]
    for _ in range(2 * k):
        r = reach.copy()
        r[1:] |= reach[:-1]
        r[:-1] |= reach[1:]
        r |= np.roll(reach, 1, axis=1) | np.roll(reach, -1, axis=1)
        reach = r
    assert not reach.all()
    assert np.all(glob[:, ~reach] == 0)


def test_tracer_and_combined_flags():
    n, nb = (16, 36, 48), (8, 6, 8)
    g = O.Grid(n=n, nb=nb, xmin=(0.1, math.pi / 6, 0.0), xmax=(1.1, 5 * math.pi / 6, 2 * math.pi), omega=0.0,
               divb_cd=0.0, bc_lo=(1, 1, 0), bc_hi=(1, 1, 0), tracer=1)
    rng = np.random.default_rng(7)
    W = np.zeros((g.nleaves, 8) + g.nb)
    W[:, 0], W[:, 4] = 1.0, 1.0
    W[:, 1] = 1.0                          # outflow: div v > 0, no shock anywhere
    g.set_state(W, prim=True)
    X = np.where(rng.random((g.nleaves,) + g.nb) < 0.002, 0.3, 0.0)
    g.set_tracer(X)
    g.ghost_fill()
    want = np.where(X.reshape(g.nleaves, -1).max(1) > 0.0, 1, -1)
    assert np.array_equal(g.flag_tracer(), want)
    assert np.array_equal(g.flag_tracer(x_thr=0.5), -np.ones(g.nleaves))
    assert 0 < (want == 1).sum() < g.nleaves
    # combined: a converging flow refines everything the windows allow
    W[:, 1] = -1.0
    g.set_state(W, prim=True)
    g.set_tracer(X)
    g.ghost_fill()
    assert np.all(g.flag_tracer(x_thr=0.5, combined=True) == 1)
    assert np.array_equal(g.flag_tracer(combined=False), want)
    # windows apply to both parts
    g.set_earth(math.pi / 2, math.pi)
    g.set_cme(0.0, 1.0, math.pi / 2, math.pi, 0.3, 5.0, 10.0, 1.0)
    w = (math.radians(30.0), math.radians(10.0), math.radians(90.0))
    f = g.flag_tracer(x_thr=0.5, combined=True, dlon_earth=w[0], dcolat_earth=w[1], dlon_cme=w[2])
    assert np.array_equal(f, g.flag_shock(0.0, *w))

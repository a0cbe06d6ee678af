"""Oracle CFL time step against closed forms.

Reading of the time step (the paper fixes only an explicit second-order
scheme, Sect. 2.1): one global dt per member,
dt = C / max over leaf cells of sum_d (|v_d| + c_f,d) / dx_d with
dx = (dr, r_c dtheta, r_c sin(theta_c) dphi), r_c and theta_c the arithmetic
mid-points of the cell's faces.  For a uniform state the sum is largest in
the cell with the smallest radius and the smallest sin(theta_c): the first
radial cell next to the theta = 30 deg (or 150 deg) edge.  The fast speed has
closed forms for B along one axis: c_f = max(a, b) along B and
sqrt(a^2 + b^2) across it (a^2 = gamma p / rho, b^2 = B^2 / rho).

Each case would fail under a plausible slip: a maximum over the directions
instead of the sum, dx_phi without sin(theta_c), face instead of centre
radii, or the fast speed taken along the wrong axis."""
import math

import numpy as np
import pytest

import oracle as O

GAMMA = 1.5
XMIN = (0.1, math.pi / 6, 0.0)
XMAX = (1.1, 5 * math.pi / 6, 2 * math.pi)
N = (20, 12, 16)
NB = (10, 6, 8)


def _uniform(stretch, W, cfl=0.8):
    g = O.Grid(n=N, nb=NB, stretch=stretch, xmin=XMIN, xmax=XMAX, gamma=GAMMA, cfl=cfl, divb_cd=0.0,
               bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC))
    S = np.zeros((g.nleaves, 8) + g.nb)
    S[:] = np.asarray(W, dtype=float)[None, :, None, None, None]
    g.set_state(S, prim=True)
    return g


def _first_cell():
    """(dr, r_c) of the innermost radial cell on both grids, (dtheta,
    theta_c) of the first colatitude cell, dphi"""
    dth = (XMAX[1] - XMIN[1]) / N[1]
    dph = (XMAX[2] - XMIN[2]) / N[2]
    r0, r1 = XMIN[0], XMAX[0]
    eq = (r1 - r0) / N[0], r0 + 0.5 * (r1 - r0) / N[0]
    q = (r1 / r0) ** (1.0 / N[0])
    st = r0 * (q - 1.0), r0 * (1.0 + q) / 2.0
    return {0: eq, 1: st}, (dth, XMIN[1] + 0.5 * dth), dph


def _expected(stretch, W, cf, cfl=0.8):
    rad, (dth, tc), dph = _first_cell()
    dr, rc = rad[stretch]
    dx = (dr, rc * dth, rc * math.sin(tc) * dph)
    s = sum((abs(W[1 + d]) + cf[d]) / dx[d] for d in range(3))
    return cfl / s


@pytest.mark.parametrize("stretch", [0, 1])
def test_dt_hydro_uniform_state(stretch):
    W = (2.0, 3.0, 0.5, -1.0, 1.5, 0.0, 0.0, 0.0)
    a = math.sqrt(GAMMA * W[4] / W[0])
    g = _uniform(stretch, W)
    want = _expected(stretch, W, (a, a, a))
    assert g.compute_dt() == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("stretch", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_dt_magnetised_uniform_state(stretch, axis):
    """B along one axis: c_f = max(a, b) along it, sqrt(a^2 + b^2) across."""
    W = [1.5, -2.0, 0.7, 1.2, 0.6, 0.0, 0.0, 0.0]
    W[5 + axis] = 2.5
    a2 = GAMMA * W[4] / W[0]
    b2 = W[5 + axis] ** 2 / W[0]
    cf = [math.sqrt(a2 + b2)] * 3
    cf[axis] = math.sqrt(max(a2, b2))
    g = _uniform(stretch, W)
    want = _expected(stretch, W, cf)
    assert g.compute_dt() == pytest.approx(want, rel=1e-13)


def test_dt_scales_with_courant_number():
    W = (1.0, 1.0, 0.0, 0.0, 1.0, 0.3, 0.2, 0.1)
    assert _uniform(1, W, cfl=0.4).compute_dt() == pytest.approx(0.5 * _uniform(1, W, cfl=0.8).compute_dt(),
                                                                 rel=1e-15)


def test_dt_minimum_sits_where_the_state_is_fastest():
    """A single fast cell far from the inner edge decides dt when its speed
    outweighs the geometry: dt follows that cell's own closed form."""
    W = (1.0, 0.0, 0.0, 0.0, 1e-4, 0.0, 0.0, 0.0)
    g = _uniform(0, W)
    S = g.get_state()
    tree = g.tree()
    # the cell (I, J, K) = (15, 6, 3): block (1, 1, 0), local (5, 0, 3)
    n = [i for i, (_, bi, bj, bk) in enumerate(tree) if (bi, bj, bk) == (1, 1, 0)][0]
    vr = 50.0
    S[n, 1, 5, 0, 3] = vr * S[n, 0, 5, 0, 3]       # momentum: v_r = 50
    S[n, 4, 5, 0, 3] += 0.5 * vr * vr * S[n, 0, 5, 0, 3]
    g.set_state(S)
    dr = (XMAX[0] - XMIN[0]) / N[0]
    dth = (XMAX[1] - XMIN[1]) / N[1]
    dph = (XMAX[2] - XMIN[2]) / N[2]
    rc = XMIN[0] + 15.5 * dr
    tc = XMIN[1] + 6.5 * dth
    a = math.sqrt(GAMMA * 1e-4)
    s = (vr + a) / dr + a / (rc * dth) + a / (rc * math.sin(tc) * dph)
    # the slow background's largest sum (innermost cell at the theta edge)
    slow = 1.0 / _expected(0, W, (a, a, a), cfl=1.0)
    assert s > slow
    assert g.compute_dt() == pytest.approx(0.8 / s, rel=1e-12)

"""Oracle invariants: uniform state preserved on the stretched spherical grid
with AMR, radial monopole at second order, closed-box conservation (Cartesian
periodic and spherical wedge with walls, across refinement levels), and
restriction after prolongation returning the coarse state."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_12867_gb300 import inputs as I

SPH = dict(xmin=(0.1, math.pi / 6, 0.0), xmax=(2.0, 5 * math.pi / 6, 2 * math.pi))


def _refine_some(g, pattern):
    f = np.zeros(g.nleaves, dtype=np.int8)
    f[pattern] = 1
    g.regrid(f)


@pytest.mark.parametrize("stretch", [0, 1])
def test_uniform_static_state_preserved_with_amr(stretch):
    g = O.Grid(n=(24, 16, 16), nb=(8, 8, 8), stretch=stretch, max_level=3, omega=0.0,
               bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC), **SPH)
    W = np.zeros((g.nleaves, 8) + g.nb)
    W[:, 0], W[:, 4] = 1.3, 0.7
    g.set_state(W, prim=True)
    _refine_some(g, [0, 5, 9])
    _refine_some(g, [3, 4])
    assert g.balance_violations() == 0
    assert len(set(g.tree()[:, 0])) == 3
    U0 = g.get_state()
    for _ in range(4):
        g.step(g.compute_dt())
    U1 = g.get_state()
    assert np.abs(U1 - U0).max() < 1e-13
    assert np.abs(U1[:, 1:4]).max() < 1e-13


def _monopole_residual(nr):
    g = O.Grid(n=(nr, nr // 2, 8), nb=(8, 8, 8), stretch=1, omega=0.0, divb_cd=0.0,
               bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC), **SPH)
    tree = g.tree()
    W = np.zeros((g.nleaves, 8) + g.nb)
    rc = I.radial_centres(nr, 0.1, 2.0, 1)
    for n, (_, bi, bj, bk) in enumerate(tree):
        r = rc[bi * 8:(bi + 1) * 8][:, None, None]
        W[n, 0], W[n, 4] = 1.0, 1.0
        W[n, 5] = 0.5 * (0.3 / r) ** 2 * np.ones((8, 8, 8))
    g.set_state(W, prim=True)
    U0 = g.get_state()
    g.stage_only(1.0)
    L = g.get_stage_state() - U0       # dU/dt
    # L1 norm of the radial momentum residual away from the walls
    res = []
    th = I.angle_centres(nr // 2, math.pi / 6, 5 * math.pi / 6)
    for n, (_, bi, bj, bk) in enumerate(tree):
        r = rc[bi * 8:(bi + 1) * 8][:, None, None]
        t = th[bj * 8:(bj + 1) * 8][None, :, None]
        m = ((r > 0.4) & (r < 1.2) & (np.abs(t - math.pi / 2) < 0.4)) * np.ones((8, 8, 8))
        res.append(np.abs(L[n, 1]) * m)
    return np.sum(res) / np.sum([np.ones(1)]) / (nr * nr // 2 * 8)


def test_radial_monopole_second_order():
    e1, e2 = _monopole_residual(32), _monopole_residual(64)
    assert e2 < e1
    assert math.log2(e1 / e2) > 1.8


def _smooth_random(g, seed, geometry):
    rng = np.random.default_rng(seed)
    W = np.zeros((g.nleaves, 8) + g.nb)
    for n in range(g.nleaves):
        W[n] = I.random_state(g.nb, seed * 100 + n, g.gamma, v=0.3, b=0.3)
        W[n, 0] = 1.0 + 0.2 * (W[n, 0] - 1.25)
        W[n, 4] = 1.0 + 0.2 * (W[n, 4] - 1.25)
    return W


def test_cartesian_periodic_box_conserves_everything():
    g = O.Grid(geometry=1, n=(16, 16, 16), nb=(8, 8, 8), xmin=(0, 0, 0), xmax=(1, 1, 1),
               divb_cd=0.0, gamma=5 / 3, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0))
    g.set_state(_smooth_random(g, 1, 1), prim=True)
    s0 = g.sums()
    for _ in range(10):
        g.step(g.compute_dt())
    s1 = g.sums()
    scale = np.abs(s0) + 1.0
    assert np.all(np.abs(s1 - s0) / scale < 1e-13), (s1 - s0)


def test_cartesian_cleaning_conserves_B_mass_momentum():
    g = O.Grid(geometry=1, n=(16, 16, 16), nb=(8, 8, 8), xmin=(0, 0, 0), xmax=(1, 1, 1),
               divb_cd=0.8, gamma=5 / 3, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0))
    g.set_state(_smooth_random(g, 2, 1), prim=True)
    s0 = g.sums()
    for _ in range(10):
        g.step(g.compute_dt())
    s1 = g.sums()
    for v in (0, 1, 2, 3, 5, 6, 7):
        assert abs(s1[v] - s0[v]) / (abs(s0[v]) + 1.0) < 1e-13


@pytest.mark.parametrize("amr", [False, True])
def test_spherical_wedge_walls_conserve_mass_energy(amr):
    g = O.Grid(n=(16, 16, 16), nb=(8, 8, 8), stretch=1, max_level=2 if amr else 1,
               omega=0.0, divb_cd=0.0, bc_lo=(O.BC_REFLECT, O.BC_REFLECT, O.BC_PERIODIC),
               bc_hi=(O.BC_REFLECT, O.BC_REFLECT, O.BC_PERIODIC), **SPH)
    g.set_state(_smooth_random(g, 3, 0), prim=True)
    if amr:
        _refine_some(g, [0, 3])
        assert len(set(g.tree()[:, 0])) == 2
    s0 = g.sums()
    for _ in range(6):
        g.step(g.compute_dt())
    s1 = g.sums()
    for v in (0, 4):
        assert abs(s1[v] - s0[v]) / abs(s0[v]) < 1e-13, (v, s1[v] - s0[v])


def test_rotating_wedge_conserves_mass():
    g = O.Grid(n=(16, 16, 16), nb=(8, 8, 8), stretch=1, omega=I.OMEGA, divb_cd=0.8,
               bc_lo=(O.BC_REFLECT, O.BC_REFLECT, O.BC_PERIODIC),
               bc_hi=(O.BC_REFLECT, O.BC_REFLECT, O.BC_PERIODIC), **SPH)
    g.set_state(_smooth_random(g, 4, 0), prim=True)
    s0 = g.sums()
    for _ in range(6):
        g.step(g.compute_dt())
    assert abs(g.sums()[0] - s0[0]) / s0[0] < 1e-13


@pytest.mark.parametrize("stretch", [0, 1])
def test_restriction_after_prolongation_is_identity(stretch):
    g = O.Grid(n=(16, 16, 16), nb=(8, 8, 8), stretch=stretch, max_level=2,
               bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC), **SPH)
    W = _smooth_random(g, 5, 0)
    g.set_state(W, prim=True)
    U0 = g.get_state()
    g.regrid(np.ones(g.nleaves, dtype=np.int8))
    assert g.nleaves == 64 and set(g.tree()[:, 0]) == {2}
    g.regrid(-np.ones(g.nleaves, dtype=np.int8))
    assert g.nleaves == 8
    U1 = g.get_state()
    # error relative to each variable's magnitude (the prolongation slopes of a
    # cell-random field are as large as the values themselves)
    scale = np.abs(U0).max(axis=(0, 2, 3, 4), keepdims=True)
    rel = np.abs(U1 - U0) / scale
    assert rel.max() <= 4 * 2.0 ** -52


def test_mass_weighted_prolongation_conserves():
    """Refinement alone keeps every conserved total (sum V U over leaves)."""
    g = O.Grid(n=(16, 16, 16), nb=(8, 8, 8), stretch=1, max_level=2,
               bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC), **SPH)
    g.set_state(_smooth_random(g, 6, 0), prim=True)
    s0 = g.sums()
    g.regrid(np.array([1, 0, 1, 0, 0, 0, 0, 1], dtype=np.int8))
    s1 = g.sums()
    assert np.all(np.abs(s1 - s0) / (np.abs(s0) + 1e-3) < 1e-13)

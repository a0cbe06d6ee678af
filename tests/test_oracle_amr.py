"""Oracle AMR pins: 2:1 balance by brute force, the regrid as the least
balanced refinement (a second, independent algorithm), coarsening rules,
Morton order, the Loehner block flags, the cone-CME inner-boundary overlay
against a 3D sphere intersection, and the probe on linear fields."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_12867_gb300 import inputs as I

SPH = dict(xmin=(0.1, math.pi / 6, 0.0), xmax=(2.0, 5 * math.pi / 6, 2 * math.pi))


def _grid(n=(16, 16, 16), nb=(4, 4, 4), max_level=3, **kw):
    return O.Grid(n=n, nb=nb, max_level=max_level, stretch=1,
                  bc_lo=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC), **SPH, **kw)


def _uniform(g):
    W = np.zeros((g.nleaves, 8) + g.nb)
    W[:, 0], W[:, 4] = 1.0, 1.0
    g.set_state(W, prim=True)


def _boxes(tree, nbase, max_level):
    """closed index boxes of the leaves at the finest level"""
    out = []
    for lev, i, j, k in tree:
        s = 1 << (max_level - lev)
        out.append((lev, np.array([i, j, k]) * s, (np.array([i, j, k]) + 1) * s))
    return out


def _adjacent(a, b, period):
    """boxes touch (share a face, edge or corner), phi periodic"""
    _, lo1, hi1 = a
    _, lo2, hi2 = b
    for d in range(3):
        if d == 2:
            ok = False
            for sh in (-period, 0, period):
                if lo1[d] <= hi2[d] + sh and lo2[d] + sh <= hi1[d]:
                    ok = True
            if not ok:
                return False
        elif not (lo1[d] <= hi2[d] and lo2[d] <= hi1[d]):
            return False
    return True


def _violations(tree, g):
    nbase = [g.n[d] // g.nb[d] for d in range(3)]
    bx = _boxes(tree, nbase, g.max_level)
    period = nbase[2] << (g.max_level - 1)
    bad = 0
    for a, b in itertools.combinations(bx, 2):
        if abs(a[0] - b[0]) > 1 and _adjacent(a, b, period):
            bad += 1
    return bad


def _least_balanced(old_tree, flags, g):
    """Independent algorithm: refine the flagged leaves, then keep refining
    the coarser leaf of any adjacent pair more than one level apart."""
    leaves = set()
    for (lev, i, j, k), f in zip(map(tuple, old_tree), flags):
        if f > 0 and lev < g.max_level:
            for a, b, c in itertools.product((0, 1), repeat=3):
                leaves.add((lev + 1, 2 * i + a, 2 * j + b, 2 * k + c))
        else:
            leaves.add((lev, i, j, k))
    nbase = [g.n[d] // g.nb[d] for d in range(3)]
    period = nbase[2] << (g.max_level - 1)
    while True:
        lst = sorted(leaves)
        bx = _boxes(lst, nbase, g.max_level)
        todo = set()
        for a, b in itertools.combinations(range(len(lst)), 2):
            if abs(bx[a][0] - bx[b][0]) > 1 and _adjacent(bx[a], bx[b], period):
                todo.add(lst[a] if bx[a][0] < bx[b][0] else lst[b])
        if not todo:
            return leaves
        for lev, i, j, k in todo:
            leaves.discard((lev, i, j, k))
            for a, b, c in itertools.product((0, 1), repeat=3):
                leaves.add((lev + 1, 2 * i + a, 2 * j + b, 2 * k + c))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_regrid_is_least_balanced_refinement(seed):
    rng = np.random.default_rng(seed)
    g = _grid(n=(12, 12, 16), nb=(4, 4, 4), max_level=3)
    _uniform(g)
    for rnd in range(3):
        old = g.tree().copy()
        flags = (rng.random(g.nleaves) < 0.08).astype(np.int8)
        g.regrid(flags)
        new = set(map(tuple, g.tree()))
        assert new == _least_balanced(old, flags, g)
        assert _violations(g.tree(), g) == 0
        assert g.balance_violations() == 0


def test_morton_order():
    g = _grid(n=(12, 12, 16), nb=(4, 4, 4), max_level=3)
    _uniform(g)
    f = np.zeros(g.nleaves, dtype=np.int8)
    f[[1, 7, 20]] = 1
    g.regrid(f)

    def key(row):
        lev, i, j, k = row
        s = g.max_level - lev
        x = [i << s, j << s, k << s]
        out = 0
        for bit in range(20, -1, -1):
            for d in range(3):
                out = (out << 1) | ((x[d] >> bit) & 1)
        return out

    keys = [key(r) for r in g.tree()]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_coarsening_rules():
    g = _grid(n=(8, 8, 16), nb=(4, 4, 4), max_level=3)
    _uniform(g)
    g.regrid(np.ones(g.nleaves, dtype=np.int8))            # everything to level 2
    f = np.zeros(g.nleaves, dtype=np.int8)
    f[0] = 1
    g.regrid(f)                                            # one level-3 family
    tree = g.tree()
    assert (tree[:, 0] == 3).sum() == 8
    # every leaf asks to coarsen: the level-3 family coarsens; level-2
    # families touching it may not (that would put level 1 next to level 3)
    g.regrid(-np.ones(g.nleaves, dtype=np.int8))
    assert g.balance_violations() == 0 and _violations(g.tree(), g) == 0
    assert set(g.tree()[:, 0]) <= {1, 2}
    g.regrid(-np.ones(g.nleaves, dtype=np.int8))
    assert set(g.tree()[:, 0]) == {1}
    # a partial family does not coarsen; refinement wins over coarsening
    g.regrid(np.ones(g.nleaves, dtype=np.int8))
    f = -np.ones(g.nleaves, dtype=np.int8)
    f[3] = 0
    f[20] = 1
    g.regrid(f)
    lv = g.tree()[:, 0]
    assert 3 in lv and 2 in lv


def _set_field(g, fn):
    rc = I.radial_centres(g.n[0], 0.1, 2.0, 1)
    th = I.angle_centres(g.n[1], *SPH["xmin"][1:2], *SPH["xmax"][1:2])
    ph = I.angle_centres(g.n[2], 0, 2 * math.pi)
    W = np.zeros((g.nleaves, 8) + g.nb)
    nb = g.nb
    for n, (_, bi, bj, bk) in enumerate(g.tree()):
        R = rc[bi * nb[0]:(bi + 1) * nb[0]][:, None, None] * np.ones(nb)
        T = th[bj * nb[1]:(bj + 1) * nb[1]][None, :, None] * np.ones(nb)
        P = ph[bk * nb[2]:(bk + 1) * nb[2]][None, None, :] * np.ones(nb)
        W[n] = fn(R, T, P)
    g.set_state(W, prim=True)


def test_loehner_flags():
    g = _grid(n=(24, 8, 8), nb=(8, 8, 8), max_level=2, divb_cd=0.0)
    nbase = 24 * 8 * 8
    rc = I.radial_centres(24, 0.1, 2.0, 1)

    def linear(R, T, P):
        W = np.zeros((8,) + R.shape)
        W[0] = 1.0 + 0.1 * np.searchsorted(rc, R)        # linear in the index
        W[1] = 5.0
        W[4] = 1.0
        return W

    def step(R, T, P):
        W = np.zeros((8,) + R.shape)
        W[0] = np.where(R < 0.6, 2.0, 1.0)
        W[1] = 5.0
        W[4] = 1.0
        return W

    # linear field, gate open: E = 0 away from the zero-gradient walls
    _set_field(g, linear)
    g.set_vbg(np.zeros(nbase))
    g.ghost_fill()
    flags = g.flag()
    for f, row in zip(flags, g.tree()):
        if row[1] == 1:                                   # middle radial block
            assert f == -1
    # density step inside the middle block, gate open -> refine it
    _set_field(g, step)
    g.ghost_fill()
    flags = g.flag()
    jb = int(np.searchsorted(rc, 0.6) // 8)
    assert jb == 1
    for f, row in zip(flags, g.tree()):
        if row[1] == 1:
            assert f == 1
    # same step, gate closed (v_r not above background + 50 km/s): no refine
    g.set_vbg(np.full(nbase, 5.0))
    assert np.all(g.flag() == -1)
    # no background yet (before the CME): nothing is ever flagged to refine
    g2 = _grid(n=(24, 8, 8), nb=(8, 8, 8), max_level=2, divb_cd=0.0)
    _set_field(g2, step)
    g2.ghost_fill()
    assert np.all(g2.flag() == -1)


def test_cme_overlay_on_inner_ghosts():
    """Inner-boundary ghosts hold the CME state exactly where the 3D sphere of
    radius r_half centred at R_c(t) on the CME axis contains the point
    (R, theta, phi) at the ghost centre (Eqs. 1-4)."""
    g = _grid(n=(8, 16, 32), nb=(8, 8, 8), max_level=1)
    g2 = O.Grid(n=(8, 16, 32), nb=(8, 8, 8), max_level=1, stretch=1,
                bc_lo=(O.BC_INNER, O.BC_OUTFLOW, O.BC_PERIODIC),
                bc_hi=(O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_PERIODIC), omega=I.OMEGA, **SPH)
    del g
    wm = I.wind_map(16, 32, SPH["xmin"][1], SPH["xmax"][1], seed=0)
    g2.set_boundary_map(wm)
    _uniform(g2)
    cme = dict(t_max=I.hours(6), colat=math.radians(80), lon=math.radians(100),
               half_width=math.radians(30), v=I.kms(1000), rho=1000.0, p=I.pressure(1000, 8e5))
    g2.set_cme(t_start=0.0, **cme)
    R = 0.1
    rh = R * math.sin(cme["half_width"])
    t = 0.5 * (2 * rh / cme["v"])
    g2.ghost_fill(0, t)
    Rc = t * cme["v"] + R - rh
    ax = np.array([math.sin(cme["colat"]) * math.cos(cme["lon"]),
                   math.sin(cme["colat"]) * math.sin(cme["lon"]), math.cos(cme["colat"])])
    th = I.angle_centres(16, SPH["xmin"][1], SPH["xmax"][1])
    ph = I.angle_centres(32, 0, 2 * math.pi)
    hits = 0
    for n, (_, bi, bj, bk) in enumerate(g2.tree()):
        if bi != 0:
            continue
        Pd = g2.get_padded(n, 0)
        for j in range(8):
            for k in range(8):
                J, K = bj * 8 + j, bk * 8 + k
                p = R * np.array([math.sin(th[J]) * math.cos(ph[K]),
                                  math.sin(th[J]) * math.sin(ph[K]), math.cos(th[J])])
                inside = np.sum((p - Rc * ax) ** 2) <= rh * rh
                for gl in (0, 1):
                    rho = Pd[0, gl, j + 2, k + 2]
                    if inside:
                        hits += 1
                        assert rho == 1000.0
                        # radial CME flow, co-rotating frame: v_phi = -Omega R sin(theta)
                        assert abs(Pd[3, gl, j + 2, k + 2] / rho + I.OMEGA * R * math.sin(th[J])) < 1e-12
                        assert Pd[5, gl, j + 2, k + 2] == 0.0
                    else:
                        assert rho == wm[0, J, K]
    assert hits > 10


def test_probe_is_exact_on_linear_fields():
    g = _grid(n=(16, 16, 16), nb=(8, 8, 8), max_level=2)

    def lin(R, T, P):
        W = np.zeros((8,) + R.shape)
        W[0] = 1.0 + 0.3 * R + 0.2 * T + 0.05 * P
        W[1] = 2.0 - R
        W[4] = 1.0 + T
        W[5] = 0.1 * P
        return W

    _set_field(g, lin)
    rng = np.random.default_rng(7)
    rf = g.faces(1, 0)
    pts = np.stack([rng.uniform(rf[1], rf[-2], 30), rng.uniform(0.8, 2.3, 30),
                    rng.uniform(0.5, 5.5, 30)], axis=1)
    out = g.probe(pts)
    ex = lin(pts[:, 0], pts[:, 1], pts[:, 2])
    for v in (0, 1, 4, 5):
        assert np.allclose(out[:, v], ex[v], rtol=1e-12, atol=1e-12)

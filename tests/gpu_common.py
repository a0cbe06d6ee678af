"""Shared set-up of the GPU parity tests: matched CUDA and oracle grids on the
same seeded inputs."""
import math

import numpy as np

import oracle as O
from paper_2211_12867_gb300 import inputs as I

SPH = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(1.1, 5 * math.pi / 6, 2 * math.pi))


def make_pair(*, n, nb, x_min=SPH["x_min"], x_max=SPH["x_max"], max_level=1, stretch=False, geometry=0,
              gamma=1.5, omega=I.OMEGA, cfl=0.8, divb_cd=0.8, bc_lo=(3, 1, 0), bc_hi=(1, 1, 0),
              precision=0, max_blocks=0, n_members=1, tracer=False):
    from paper_2211_12867_gb300.icarus import Icarus
    g = Icarus(n_cells=n, block=nb, max_level=max_level, stretch=stretch, geometry=geometry, x_min=x_min,
               x_max=x_max, gamma=gamma, omega=omega, cfl=cfl, divb_cd=divb_cd, bc_lo=bc_lo, bc_hi=bc_hi,
               precision=precision, max_blocks=max_blocks, n_members=n_members, tracer=tracer)
    o = O.Grid(geometry=geometry, n=n, nb=nb, max_level=max_level, stretch=int(stretch), xmin=x_min, xmax=x_max,
               gamma=gamma, omega=omega, cfl=cfl, divb_cd=divb_cd, bc_lo=bc_lo, bc_hi=bc_hi, tracer=tracer)
    return g, o


def wind_setup(g, o, seed=0, member=0):
    """seeded boundary wind + spherically expanding start state on both"""
    n = g.n_cells
    wm = I.wind_map(n[1], n[2], g.desc.x_min[1], g.desc.x_max[1], seed=seed, r_in=g.desc.x_min[0])
    g.set_inner_boundary(member, wm)
    o.set_boundary_map(wm)
    rc = I.radial_centres(n[0], g.desc.x_min[0], g.desc.x_max[0], g.desc.radial_stretch)
    G = I.initial_prim(wm, rc, g.desc.x_min[0], g.desc.gamma, omega=g.desc.omega,
                       colat_min=g.desc.x_min[1], colat_max=g.desc.x_max[1])
    tree = g.tree(member)
    assert np.array_equal(tree, o.tree())
    W = I.global_to_blocks(G, tree, g.block)
    g.set_state(member, W, prim=True)
    # the oracle starts from the bits the GPU holds
    o.set_state(g.get_state(member))
    return wm


def rel_linf(a, b):
    """max over variables of max|a-b| / max|b| (per-variable magnitude)"""
    out = []
    for v in range(8):
        scale = np.abs(b[:, v]).max()
        out.append(np.abs(a[:, v] - b[:, v]).max() / (scale if scale > 0 else 1.0))
    return np.array(out)

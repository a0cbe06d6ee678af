"""Seeded synthetic inputs: units, boundary wind, initial state, cone-CME draws.

This module holds the input recipe only, none of the method's arithmetic; it
serves both the CUDA library and the oracle.  The paper drives its inner
boundary with WSA coronal-model maps (Sect. 2.1) that are not available; an
analytic, seeded wind with the paper's geometry (0.1 AU inner boundary,
+-60 degrees, 360 degrees) stands in for them.

Normalised units: length 1 AU, speed 100 km/s, density m_p per cm^3, pressure
rho0 v0^2, magnetic field sqrt(mu0 rho0 v0^2) (mu0 absorbed), time 1 AU/100 km/s.
"""
from __future__ import annotations

import math

import numpy as np

# physical constants and normalisation
AU_M = 1.495978707e11
R_SUN_M = 6.957e8
V0_MS = 1.0e5
M_P = 1.67262192e-27
K_B = 1.380649e-23
MU0 = 4.0e-7 * math.pi
RHO0 = M_P * 1.0e6
P0 = RHO0 * V0_MS ** 2
B0_T = math.sqrt(MU0 * RHO0 * V0_MS ** 2)
T0_S = AU_M / V0_MS
DAY_S = 86400.0
HOUR_S = 3600.0

OMEGA_SUN_S = 2.0 * math.pi / (25.38 * DAY_S)   # sidereal rotation rate
OMEGA = OMEGA_SUN_S * T0_S                      # normalised
OMEGA_SYN = (OMEGA_SUN_S - 2.0 * math.pi / (365.25 * DAY_S)) * T0_S


def days(x):
    return x * DAY_S / T0_S


def hours(x):
    return x * HOUR_S / T0_S


def kms(v):
    return v * 1.0e3 / V0_MS


def pressure(n_cc, T_K):
    """p = 2 n k_B T (electrons + protons, T_e = T_p), normalised."""
    return 2.0 * n_cc * 1.0e6 * K_B * T_K / P0


def bfield(b_nT):
    return b_nT * 1.0e-9 / B0_T


# ---------------------------------------------------------------- grids
def angle_centres(n, lo, hi):
    e = lo + (hi - lo) * np.arange(n + 1) / n
    return 0.5 * (e[:-1] + e[1:])


def radial_centres(n, r_in, r_out, stretch):
    k = np.arange(n + 1) / n
    e = r_in * (r_out / r_in) ** k if stretch else r_in + (r_out - r_in) * k
    return 0.5 * (e[:-1] + e[1:])


def eq5_cells(r_in, r_out, dtheta):
    """Eq. 5 (Sect. 2.2): radial cell count that keeps cells near cubical."""
    return math.log(r_out / r_in) / math.log((2.0 + dtheta) / (2.0 - dtheta))


# ---------------------------------------------------------------- wind
def wind_map(n_theta, n_phi, colat_min, colat_max, seed=0, r_in=0.1,
             phi_min=0.0, phi_max=2 * math.pi):
    """Primitive inner-boundary map [8][n_theta][n_phi] (normalised).

    Slow wind (350 km/s) within +-15 degrees of latitude rising to 750 km/s
    through a tanh of width 5 degrees; n = 300 (v/450)^-2 cm^-3; T = 1.5 MK;
    B_r = +-200 nT across a sector boundary lambda_s = 10 deg sin(phi - phi_s)
    with a seeded phase; Parker B_phi = -B_r Omega r sin(theta) / v_r;
    co-rotating-frame v_phi = -Omega r_in sin(theta)."""
    rng = np.random.default_rng(seed)
    phi_s = rng.uniform(0.0, 2 * math.pi)
    th = angle_centres(n_theta, colat_min, colat_max)[:, None]
    ph = angle_centres(n_phi, phi_min, phi_max)[None, :]
    lat = 0.5 * math.pi - th
    deg = math.pi / 180.0
    v_kms = 350.0 + 400.0 * 0.5 * (1.0 + np.tanh((np.abs(lat) - 15 * deg) / (5 * deg)))
    n_cc = 300.0 * (v_kms / 450.0) ** -2
    lam_s = 10 * deg * np.sin(ph - phi_s)
    sgn = np.where(lat - lam_s >= 0.0, 1.0, -1.0)
    vr = kms(v_kms) * np.ones_like(sgn)
    Br = bfield(200.0) * sgn
    Bp = -Br * OMEGA * r_in * np.sin(th) / vr
    W = np.zeros((8, n_theta, n_phi))
    W[0] = n_cc * np.ones_like(sgn)
    W[1] = vr
    W[3] = -OMEGA * r_in * np.sin(th) * np.ones_like(sgn)
    W[4] = pressure(n_cc, 1.5e6) * np.ones_like(sgn)
    W[5] = Br
    W[7] = Bp
    return W


def initial_prim(wmap, r_c, r_in, gamma, omega=OMEGA, colat_min=None, colat_max=None):
    """Spherically expanding start state from the map (global [8][nr][nth][nph]):
    rho ~ (r_in/r)^2, v_r constant, p ~ rho^gamma, B_r ~ r^-2, B_phi ~ r^-1,
    v_phi = -Omega r sin(theta)."""
    nth, nph = wmap.shape[1:]
    x = (r_in / r_c)[:, None, None]
    W = np.zeros((8, len(r_c), nth, nph))
    W[0] = wmap[0][None] * x ** 2
    W[1] = wmap[1][None] * np.ones_like(x)
    W[4] = wmap[4][None] * x ** (2 * gamma)
    W[5] = wmap[5][None] * x ** 2
    W[7] = wmap[7][None] * x
    if colat_min is not None:
        th = angle_centres(nth, colat_min, colat_max)
        W[3] = -omega * r_c[:, None, None] * np.sin(th)[None, :, None] * np.ones((1, 1, nph))
    return W


def global_to_blocks(G, tree, nb):
    """[v][I][J][K] base-level array -> [leaf][v][i][j][k] in the given leaf
    order (tree rows (level, bi, bj, bk), all level 1)."""
    out = np.empty((len(tree), G.shape[0]) + tuple(nb), dtype=G.dtype)
    for n, (lev, bi, bj, bk) in enumerate(tree):
        assert lev == 1
        out[n] = G[:, bi * nb[0]:(bi + 1) * nb[0], bj * nb[1]:(bj + 1) * nb[1],
                   bk * nb[2]:(bk + 1) * nb[2]]
    return out


def blocks_to_global(B, tree, nb, n):
    """Inverse of global_to_blocks for a single-level grid."""
    G = np.empty((B.shape[1],) + tuple(n), dtype=B.dtype)
    for k, (lev, bi, bj, bk) in enumerate(tree):
        G[:, bi * nb[0]:(bi + 1) * nb[0], bj * nb[1]:(bj + 1) * nb[1],
          bk * nb[2]:(bk + 1) * nb[2]] = B[k]
    return G


def random_state(shape, seed, gamma, rho=(0.5, 2.0), v=1.0, p=(0.5, 2.0), b=1.0):
    """Generic positive random primitive field [8][...] for unit checks."""
    rng = np.random.default_rng(seed)
    W = np.zeros((8,) + tuple(shape))
    W[0] = rng.uniform(*rho, size=shape)
    W[1:4] = rng.uniform(-v, v, size=(3,) + tuple(shape))
    W[4] = rng.uniform(*p, size=shape)
    W[5:8] = rng.uniform(-b, b, size=(3,) + tuple(shape))
    return W


# ---------------------------------------------------------------- CME draws
def cme_config2(seed=0, earth_lon=math.pi):
    """Cone CME of the 512x60x180 single-level workload: half-width 30 deg,
    latitude ~ U(+-20 deg) seeded, Earth-directed in longitude, 1000 km/s,
    n = 1000 cm^-3, T = 8e5 K, B = 0, injected for at most 6 h."""
    rng = np.random.default_rng(seed)
    lat = math.radians(rng.uniform(-20.0, 20.0))
    return dict(t_max=hours(6.0), colat=0.5 * math.pi - lat, lon=earth_lon,
                half_width=math.radians(30.0), v=kms(1000.0), rho=1000.0,
                p=pressure(1000.0, 8.0e5))


def cme_ensemble(n_members, seed0=1000, earth_lon=math.pi):
    """Ensemble draws: speed U(600,1800) km/s, half-width U(15,45) deg,
    latitude and longitude U(+-20 deg) about Earth, n U(500,2000) cm^-3,
    T = 8e5 K, maximum AMR level 3 or 4."""
    out = []
    for m in range(n_members):
        rng = np.random.default_rng(seed0 + m)
        v = rng.uniform(600.0, 1800.0)
        hw = rng.uniform(15.0, 45.0)
        lat = rng.uniform(-20.0, 20.0)
        lon = rng.uniform(-20.0, 20.0)
        n = rng.uniform(500.0, 2000.0)
        lvl = int(rng.integers(3, 5))
        out.append(dict(t_max=hours(6.0), colat=0.5 * math.pi - math.radians(lat),
                        lon=earth_lon + math.radians(lon), half_width=math.radians(hw),
                        v=kms(v), rho=n, p=pressure(n, 8.0e5), max_level=lvl))
    return out


def earth_position(t, t_inj, earth_lon0=math.pi, r=1.0):
    """Earth in the co-rotating frame: r = 1 AU, latitude 0, longitude
    drifting at the synodic rate."""
    return np.array([r, 0.5 * math.pi,
                     (earth_lon0 - OMEGA_SYN * (t - t_inj)) % (2 * math.pi)])


# ---------------------------------------------------------------- MLP init
MLP_IN, MLP_H = 64, 128


def mlp_init(seed):
    """He-normal initial weights of the 64-128-128-1 refinement predictor,
    zero biases (seeded); layout W1[128,64], b1, W2[128,128], b2, w3[128], b3."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / MLP_IN), (MLP_H, MLP_IN))
    W2 = rng.normal(0.0, math.sqrt(2.0 / MLP_H), (MLP_H, MLP_H))
    w3 = rng.normal(0.0, math.sqrt(2.0 / MLP_H), MLP_H)
    return np.concatenate([W1.ravel(), np.zeros(MLP_H), W2.ravel(), np.zeros(MLP_H), w3, [0.0]])

"""Plain FP64 CPU oracle of the Icarus MHD update (arXiv 2211.12867).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_2211_12867_gb300``: its C sources
(``or_physics.c``, ``or_grid.c``) implement the method independently, in FP64,
in natural loop order, from the paper (Sect. 2.1, 2.2, 3, Eqs. 1-5); where
the paper is silent the C sources state the reading they take at each use.
``mlp.py`` holds the NumPy oracle of the learned refinement predictor.

Every routine here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, textbook solutions and the numbers the paper prints.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["or_physics.c", "or_grid.c"]
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_OUTFLOW, BC_REFLECT, BC_INNER = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    hdr = os.path.join(_HERE, "or_internal.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("geometry", C.c_int), ("n", C.c_int * 3), ("nb", C.c_int * 3),
        ("max_level", C.c_int), ("stretch", C.c_int),
        ("xmin", C.c_double * 3), ("xmax", C.c_double * 3),
        ("gamma", C.c_double), ("omega", C.c_double), ("cfl", C.c_double),
        ("divb_cd", C.c_double), ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("p_floor", C.c_double), ("rho_floor", C.c_double), ("tracer", C.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P, D, I, V = C.c_void_p, C.c_double, C.c_int, None
            dp = C.POINTER(C.c_double)
            sig = {
                "or_create": (P, [C.POINTER(Params)]),
                "or_destroy": (V, [P]),
                "or_nleaves": (I, [P]),
                "or_time": (D, [P]),
                "or_set_time": (V, [P, D]),
                "or_floor_hits": (C.c_long, [P]),
                "or_set_threads": (V, [P, I]),
                "or_max_threads": (I, []),
                "or_get_tree": (V, [P, P]),
                "or_state_size": (C.c_size_t, [P]),
                "or_set_state": (V, [P, P, I]),
                "or_get_state": (V, [P, P]),
                "or_get_padded": (V, [P, I, I, P]),
                "or_set_padded": (V, [P, I, I, P]),
                "or_set_boundary_map": (V, [P, P]),
                "or_set_cme": (V, [P, P]),
                "or_snapshot_vbg": (I, [P]),
                "or_set_vbg": (V, [P, P]),
                "or_ghost_fill": (V, [P, I, D]),
                "or_compute_dt": (D, [P]),
                "or_step": (V, [P, D]),
                "or_advance": (I, [P, I, D]),
                "or_flag": (V, [P, P, P]),
                "or_set_earth": (V, [P, P]),
                "or_flag_shock": (V, [P, P, P]),
                "or_divv": (V, [P, I, P]),
                "or_get_tracer": (V, [P, P]),
                "or_set_tracer": (V, [P, P]),
                "or_flag_tracer": (V, [P, P, P]),
                "or_regrid": (V, [P, P]),
                "or_probe": (V, [P, I, P, P]),
                "or_sums": (V, [P, P]),
                "or_total_volume": (D, [P]),
                "or_get_faces": (V, [P, I, I, P]),
                "or_get_offsets": (V, [P, I, I, P]),
                "or_stage_only": (V, [P, D, D]),
                "or_get_stage_state": (V, [P, P]),
                "or_balance_violations": (I, [P]),
                "or_prim2cons": (V, [dp, dp, D]),
                "or_cons2prim": (V, [dp, dp, D]),
                "or_fast_speed": (D, [dp, I, D]),
                "or_mc_slope": (D, [D, D, D]),
                "or_tvdlf": (V, [dp, dp, I, D, dp]),
                "or_loehner": (D, [dp, dp, dp, D]),
                "or_cme_eval": (V, [dp, D, D, D, D, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- pointwise
def prim2cons(W, gamma):
    W = np.ascontiguousarray(W, dtype=np.float64)
    U = np.zeros(8)
    lib().or_prim2cons(_dp(W), _dp(U), gamma)
    return U


def cons2prim(U, gamma):
    U = np.ascontiguousarray(U, dtype=np.float64)
    W = np.zeros(8)
    lib().or_cons2prim(_dp(U), _dp(W), gamma)
    return W


def fast_speed(W, d, gamma):
    W = np.ascontiguousarray(W, dtype=np.float64)
    return lib().or_fast_speed(_dp(W), d, gamma)


def mc_slope(um, u0, up):
    return lib().or_mc_slope(um, u0, up)


def tvdlf(WL, WR, d, gamma):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(8)
    lib().or_tvdlf(_dp(WL), _dp(WR), d, gamma, _dp(F))
    return F


def loehner(um, u0, up, eps):
    um = np.ascontiguousarray(um, dtype=np.float64)
    up = np.ascontiguousarray(up, dtype=np.float64)
    c = np.array([u0], dtype=np.float64)
    return lib().or_loehner(_dp(um), _dp(c), _dp(up), eps)


def cme_eval(t_start, t_max, colat, lon, half_width, v, R, t, pcolat, plon):
    """(opening angle theta(t), angular distance d) of Eqs. 1-4; theta < 0
    when the CME sphere no longer crosses the shell or the window is closed."""
    c = np.array([t_start, t_max, colat, lon, half_width, v], dtype=np.float64)
    out = np.zeros(2)
    lib().or_cme_eval(_dp(c), R, t, pcolat, plon, _dp(out))
    return out[0], out[1]


# ---------------------------------------------------------------- grid
class Grid:
    """One member of the oracle's block-structured grid."""

    def __init__(self, *, geometry=0, n=(60, 16, 32), nb=(12, 8, 8), max_level=1,
                 stretch=0, xmin=(0.1, np.pi / 6, 0.0), xmax=(1.1, 5 * np.pi / 6, 2 * np.pi),
                 gamma=1.5, omega=0.0, cfl=0.8, divb_cd=0.8,
                 bc_lo=(BC_INNER, BC_OUTFLOW, BC_PERIODIC),
                 bc_hi=(BC_OUTFLOW, BC_OUTFLOW, BC_PERIODIC),
                 p_floor=1e-8, rho_floor=1e-8, tracer=0, threads=0):
        p = Params()
        p.geometry = geometry
        p.n[:] = list(n)
        p.nb[:] = list(nb)
        p.max_level = max_level
        p.stretch = stretch
        p.xmin[:] = list(xmin)
        p.xmax[:] = list(xmax)
        p.gamma, p.omega, p.cfl, p.divb_cd = gamma, omega, cfl, divb_cd
        p.bc_lo[:] = list(bc_lo)
        p.bc_hi[:] = list(bc_hi)
        p.p_floor, p.rho_floor = p_floor, rho_floor
        p.tracer = int(bool(tracer))
        self.params = p
        self.n, self.nb, self.gamma = tuple(n), tuple(nb), gamma
        self.max_level = max_level
        self._g = lib().or_create(C.byref(p))
        if not self._g:
            raise ValueError("oracle: block size must divide the base grid")
        if threads:
            lib().or_set_threads(self._g, threads)

    def __del__(self):
        g = getattr(self, "_g", None)
        if g:
            lib().or_destroy(g)
            self._g = None

    # -- properties
    @property
    def nleaves(self):
        return lib().or_nleaves(self._g)

    @property
    def t(self):
        return lib().or_time(self._g)

    @t.setter
    def t(self, v):
        lib().or_set_time(self._g, float(v))

    @property
    def floor_hits(self):
        return lib().or_floor_hits(self._g)

    def tree(self):
        out = np.zeros((self.nleaves, 4), dtype=np.int32)
        lib().or_get_tree(self._g, _ptr(out))
        return out

    def block_cells(self):
        return self.nb[0] * self.nb[1] * self.nb[2]

    # -- state
    def get_state(self):
        out = np.zeros((self.nleaves, 8) + self.nb)
        lib().or_get_state(self._g, _ptr(out))
        return out

    def set_state(self, U, prim=False):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape((self.nleaves, 8) + self.nb)
        lib().or_set_state(self._g, _ptr(U), 1 if prim else 0)

    def get_stage_state(self):
        out = np.zeros((self.nleaves, 8) + self.nb)
        lib().or_get_stage_state(self._g, _ptr(out))
        return out

    def get_padded(self, n, which=0):
        P = tuple(x + 4 for x in self.nb)
        out = np.zeros((8,) + P)
        lib().or_get_padded(self._g, n, which, _ptr(out))
        return out

    def set_padded(self, n, P, which=0):
        """overwrite leaf n's padded block, ghost layers included"""
        P = np.ascontiguousarray(P, dtype=np.float64).reshape((8,) + tuple(x + 4 for x in self.nb))
        lib().or_set_padded(self._g, n, which, _ptr(P))

    def set_boundary_map(self, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        assert prim.shape == (8, self.n[1], self.n[2])
        lib().or_set_boundary_map(self._g, _ptr(prim))

    def set_cme(self, t_start, t_max, colat, lon, half_width, v, rho, p):
        c = np.array([t_start, t_max, colat, lon, half_width, v, rho, p], dtype=np.float64)
        lib().or_set_cme(self._g, _ptr(c))

    def snapshot_vbg(self):
        if lib().or_snapshot_vbg(self._g) != 0:
            raise RuntimeError("oracle: background speed needs an unrefined grid")

    def set_vbg(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        lib().or_set_vbg(self._g, _ptr(v))

    # -- method
    def ghost_fill(self, which=0, t=None):
        lib().or_ghost_fill(self._g, which, self.t if t is None else float(t))

    def compute_dt(self):
        return lib().or_compute_dt(self._g)

    def step(self, dt):
        lib().or_step(self._g, float(dt))

    def advance(self, nsteps, t_stop=np.inf):
        return lib().or_advance(self._g, int(nsteps), float(t_stop))

    def stage_only(self, dtf, t=None):
        lib().or_stage_only(self._g, float(dtf), self.t if t is None else float(t))

    def flag(self, e_refine=0.1, e_coarsen=0.0125, eps=0.01, dv=0.5):
        crit = np.array([e_refine, e_coarsen, eps, dv], dtype=np.float64)
        out = np.zeros(self.nleaves, dtype=np.int8)
        lib().or_flag(self._g, _ptr(crit), _ptr(out))
        return out

    def set_earth(self, colat, lon0, t0=0.0, rate=0.0):
        """Earth at colatitude colat, longitude lon0 - rate (t - t0)"""
        e = np.array([colat, lon0, t0, rate], dtype=np.float64)
        lib().or_set_earth(self._g, _ptr(e))

    def flag_shock(self, div_thr=0.0, dlon_earth=np.radians(30.0), dcolat_earth=np.radians(10.0),
                   dlon_cme=np.radians(90.0)):
        """shock criterion (Sect. 3.2) after a ghost fill: +1 / -1 per leaf"""
        crit = np.array([div_thr, dlon_earth, dcolat_earth, dlon_cme], dtype=np.float64)
        out = np.zeros(self.nleaves, dtype=np.int8)
        lib().or_flag_shock(self._g, _ptr(crit), _ptr(out))
        return out

    def get_tracer(self):
        """rho X of the interior cells, [leaf][i][j][k]"""
        out = np.zeros((self.nleaves,) + self.nb)
        lib().or_get_tracer(self._g, _ptr(out))
        return out

    def set_tracer(self, T):
        T = np.ascontiguousarray(T, dtype=np.float64).reshape((self.nleaves,) + self.nb)
        lib().or_set_tracer(self._g, _ptr(T))

    def flag_tracer(self, x_thr=0.0, div_thr=0.0, dlon_earth=0.0, dcolat_earth=0.0, dlon_cme=0.0,
                    combined=False):
        """tracer criterion (Sect. 3.1) or, combined, tracer or shock (Sect. 3.3)"""
        crit = np.array([x_thr, div_thr, dlon_earth, dcolat_earth, dlon_cme, 1.0 if combined else 0.0])
        out = np.zeros(self.nleaves, dtype=np.int8)
        lib().or_flag_tracer(self._g, _ptr(crit), _ptr(out))
        return out

    def divv(self, n):
        """interior velocity divergence of leaf n (after a ghost fill)"""
        out = np.zeros(self.nb)
        lib().or_divv(self._g, n, _ptr(out))
        return out

    def regrid(self, flags):
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.nleaves,)
        lib().or_regrid(self._g, _ptr(flags))

    def balance_violations(self):
        return lib().or_balance_violations(self._g)

    def probe(self, pts):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 8))
        lib().or_probe(self._g, pts.shape[0], _ptr(pts), _ptr(out))
        return out

    def sums(self):
        out = np.zeros(8)
        lib().or_sums(self._g, _ptr(out))
        return out

    def total_volume(self):
        return lib().or_total_volume(self._g)

    def faces(self, level, d):
        N = self.n[d] << (level - 1)
        out = np.zeros(N + 1)
        lib().or_get_faces(self._g, level, d, _ptr(out))
        return out

    def offsets(self, level, d):
        N = self.n[d] << (level - 1)
        out = np.zeros((N, 2))
        lib().or_get_offsets(self._g, level, d, _ptr(out))
        return out


def max_threads() -> int:
    return lib().or_max_threads()

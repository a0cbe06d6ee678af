"""Python binding of libicarus (ctypes): argument marshalling only.

Every step of the method runs in the CUDA kernels behind the C ABI declared in
``include/icarus.h``.  PyTorch supplies the device arena (one uint8 tensor)
and a CUDA stream; there is no CPU or PyTorch fallback: if the shared library
is missing or no GPU is present the constructor raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libicarus.so")
_lock = threading.Lock()
_lib = None

FP64, FP32_MIXED = 0, 1
SPHERICAL, CARTESIAN = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_REFLECT, BC_INNER = 0, 1, 2, 3
FLAG_PLAIN, FLAG_LEARNED, FLAG_BOTH, FLAG_SHOCK, FLAG_TRACER, FLAG_COMBINED = 0, 1, 2, 3, 4, 5
# the shock criterion's windows of the paper (Sect. 3.2): Earth longitude
# +-30 deg, Earth colatitude +-10 deg, CME longitude +-90 deg
SHOCK_WINDOWS = (math.radians(30.0), math.radians(10.0), math.radians(90.0))

STATUS = {0: "ok", 1: "invalid argument", 2: "arena too small", 3: "CUDA error",
          4: "non-physical state", 5: "device wait timed out", 6: "call out of order",
          7: "block pool capacity exceeded"}

EXPORTS = [
    "icarus_arena_bytes", "icarus_init_grid", "icarus_set_inner_boundary", "icarus_inject_cone_cme",
    "icarus_step", "icarus_flag_refine", "icarus_set_flags", "icarus_regrid", "icarus_probe",
    "icarus_n_leaves", "icarus_get_tree", "icarus_set_state", "icarus_get_state", "icarus_set_time",
    "icarus_set_member_max_level", "icarus_ghost_fill", "icarus_conservation_sums", "icarus_get_dt",
    "icarus_status_word", "icarus_set_tile", "icarus_use_graph", "icarus_kernels_per_step",
    "icarus_profile", "icarus_profile_read", "icarus_set_fp64_islands", "icarus_conservation_sums_static",
    "icarus_set_floor_budget", "icarus_get_padded", "icarus_set_earth", "icarus_get_tracer",
    "icarus_set_tracer", "icarus_alu_peak", "icarus_set_direct_halo",
    "icarus_mlp_set_params", "icarus_mlp_get_params", "icarus_mlp_features", "icarus_mlp_predict_leaves",
    "icarus_mlp_predict", "icarus_mlp_grad", "icarus_mlp_dataset_clear", "icarus_mlp_dataset_add",
    "icarus_mlp_train", "icarus_cell_updates", "icarus_save", "icarus_load", "icarus_destroy",
    "icarus_status_string",
]


class IcarusError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn}: {STATUS.get(code, code)} ({code})")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [
        ("n_cells", C.c_int * 3), ("block", C.c_int * 3), ("max_level", C.c_int),
        ("radial_stretch", C.c_int), ("geometry", C.c_int),
        ("x_min", C.c_double * 3), ("x_max", C.c_double * 3),
        ("gamma", C.c_double), ("omega", C.c_double), ("cfl", C.c_double), ("divb_cd", C.c_double),
        ("p_floor", C.c_double), ("rho_floor", C.c_double),
        ("precision", C.c_int), ("n_members", C.c_int),
        ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3), ("max_blocks", C.c_int),
        ("arena", C.c_void_p), ("arena_bytes", C.c_size_t), ("stream", C.c_void_p), ("tracer", C.c_int),
    ]


class Cone(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("t_start", "t_max", "colat", "lon", "half_width", "v", "rho", "p")]


class Refine(C.Structure):
    _fields_ = [("e_refine", C.c_double), ("e_coarsen", C.c_double), ("eps", C.c_double),
                ("dv", C.c_double), ("mode", C.c_int),
                ("div_thr", C.c_double), ("dlon_earth", C.c_double), ("dcolat_earth", C.c_double),
                ("dlon_cme", C.c_double), ("x_thr", C.c_double)]


def load(build_if_missing: bool = True):
    """Load libicarus.so (compiling it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise ImportError(f"libicarus.so is not built ({LIB_PATH})")
            from . import build as _b
            _b.build()
        L = C.CDLL(LIB_PATH)
        P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        dp = C.POINTER(C.c_double)
        sig = {
            "icarus_arena_bytes": [C.POINTER(GridDesc), C.POINTER(S)],
            "icarus_init_grid": [C.POINTER(GridDesc), C.POINTER(P)],
            "icarus_set_inner_boundary": [P, I, dp],
            "icarus_inject_cone_cme": [P, I, C.POINTER(Cone)],
            "icarus_step": [P, I, dp, dp],
            "icarus_flag_refine": [P, C.POINTER(Refine), P],
            "icarus_set_flags": [P, P],
            "icarus_regrid": [P],
            "icarus_probe": [P, I, I, dp, dp],
            "icarus_n_leaves": [P, I, C.POINTER(I)],
            "icarus_get_tree": [P, I, P, I, C.POINTER(I)],
            "icarus_set_state": [P, I, dp, S, I],
            "icarus_get_state": [P, I, dp, S],
            "icarus_set_time": [P, I, D],
            "icarus_set_member_max_level": [P, I, I],
            "icarus_ghost_fill": [P],
            "icarus_conservation_sums": [P, I, dp],
            "icarus_get_dt": [P, dp],
            "icarus_status_word": [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)],
            "icarus_set_tile": [P, I, I, I],
            "icarus_use_graph": [P, I],
            "icarus_kernels_per_step": [P, C.POINTER(I)],
            "icarus_profile": [P, I],
            "icarus_profile_read": [P, dp, C.POINTER(I), I],
            "icarus_set_floor_budget": [P, D],
            "icarus_get_padded": [P, I, I, dp, S],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = args
        L.icarus_destroy.restype = None
        L.icarus_destroy.argtypes = [P]
        L.icarus_status_string.restype = C.c_char_p
        L.icarus_status_string.argtypes = [C.c_int]
        _lib = L
        return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _chk(fn, code):
    if code != 0:
        raise IcarusError(fn, code)


class Icarus:
    """A libicarus context on one GPU: all members of one ensemble."""

    def __init__(self, *, n_cells, block, max_level=1, stretch=False, geometry=SPHERICAL,
                 x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi),
                 gamma=1.5, omega=0.0, cfl=0.8, divb_cd=0.8, p_floor=1e-8, rho_floor=1e-8,
                 precision=FP64, n_members=1, bc_lo=(BC_INNER, BC_OUTFLOW, BC_PERIODIC),
                 bc_hi=(BC_OUTFLOW, BC_OUTFLOW, BC_PERIODIC), max_blocks=0, tracer=False, device=None,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libicarus needs a CUDA GPU; no fallback path exists")
        self.lib = load()
        d = GridDesc()
        d.n_cells[:] = list(n_cells)
        d.block[:] = list(block)
        d.max_level = max_level
        d.radial_stretch = int(bool(stretch))
        d.geometry = geometry
        d.x_min[:] = list(x_min)
        d.x_max[:] = list(x_max)
        d.gamma, d.omega, d.cfl, d.divb_cd = gamma, omega, cfl, divb_cd
        d.p_floor, d.rho_floor = p_floor, rho_floor
        d.precision = precision
        d.n_members = n_members
        d.bc_lo[:] = list(bc_lo)
        d.bc_hi[:] = list(bc_hi)
        d.max_blocks = max_blocks
        d.tracer = int(bool(tracer))
        nbytes = C.c_size_t(0)
        _chk("icarus_arena_bytes", self.lib.icarus_arena_bytes(C.byref(d), C.byref(nbytes)))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.arena = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = self.arena.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        d.arena = aligned
        d.arena_bytes = nbytes.value
        d.stream = self.stream.cuda_stream
        self.desc = d
        self.n_cells, self.block = tuple(n_cells), tuple(block)
        self.n_members, self.max_level = n_members, max_level
        self.precision = precision
        self.arena_bytes = nbytes.value
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            _chk("icarus_init_grid", self.lib.icarus_init_grid(C.byref(d), C.byref(ctx)))
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            self.stream.synchronize()
            self.lib.icarus_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- helpers
    @property
    def cells_per_block(self):
        return self.block[0] * self.block[1] * self.block[2]

    def n_leaves(self, member=-1):
        n = C.c_int(0)
        _chk("icarus_n_leaves", self.lib.icarus_n_leaves(self.ctx, member, C.byref(n)))
        return n.value

    def tree(self, member=0):
        n = self.n_leaves(member)
        rows = np.zeros((n, 4), dtype=np.int32)
        got = C.c_int(0)
        _chk("icarus_get_tree", self.lib.icarus_get_tree(self.ctx, member, rows.ctypes.data_as(C.c_void_p), n,
                                                         C.byref(got)))
        return rows

    # ---------------------------------------------------------------- the ABI
    def set_inner_boundary(self, member, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        assert prim.shape == (8, self.n_cells[1], self.n_cells[2])
        _chk("icarus_set_inner_boundary", self.lib.icarus_set_inner_boundary(self.ctx, member, _dp(prim)))

    def inject_cone_cme(self, member, *, t_start, t_max, colat, lon, half_width, v, rho, p):
        c = Cone(t_start, t_max, colat, lon, half_width, v, rho, p)
        _chk("icarus_inject_cone_cme", self.lib.icarus_inject_cone_cme(self.ctx, member, C.byref(c)))

    def step(self, n_steps, t_stop=None, want_time=True):
        ts = np.full(self.n_members, np.inf) if t_stop is None else np.broadcast_to(
            np.asarray(t_stop, dtype=np.float64), (self.n_members,)).copy()
        out = np.zeros(self.n_members) if want_time else None
        _chk("icarus_step", self.lib.icarus_step(self.ctx, int(n_steps), _dp(ts),
                                                 _dp(out) if want_time else None))
        return out

    def flag_refine(self, e_refine=0.1, e_coarsen=0.0125, eps=0.01, dv=0.5, mode=FLAG_PLAIN, div_thr=0.0,
                    windows=SHOCK_WINDOWS, x_thr=0.0):
        crit = Refine(e_refine, e_coarsen, eps, dv, mode, div_thr, *windows, x_thr)
        out = np.zeros(self.n_leaves(-1), dtype=np.int8)
        _chk("icarus_flag_refine", self.lib.icarus_flag_refine(self.ctx, C.byref(crit),
                                                               out.ctypes.data_as(C.c_void_p)))
        return out

    def set_flags(self, flags):
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.n_leaves(-1),)
        _chk("icarus_set_flags", self.lib.icarus_set_flags(self.ctx, flags.ctypes.data_as(C.c_void_p)))

    def regrid(self):
        _chk("icarus_regrid", self.lib.icarus_regrid(self.ctx))

    def probe(self, member, pts):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 8))
        _chk("icarus_probe", self.lib.icarus_probe(self.ctx, member, pts.shape[0], _dp(pts), _dp(out)))
        return out

    def set_state(self, member, U, prim=False):
        n = self.n_leaves(member)
        U = np.ascontiguousarray(U, dtype=np.float64).reshape((n, 8) + self.block)
        _chk("icarus_set_state", self.lib.icarus_set_state(self.ctx, member, _dp(U), U.size, int(bool(prim))))

    def get_state(self, member=0, out=None):
        """conserved state of a member (host FP64); `out` (optional, e.g. a
        pinned buffer) receives it in place"""
        n = self.n_leaves(member)
        if out is None:
            out = np.zeros((n, 8) + self.block)
        elif out.shape != (n, 8) + self.block or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("get_state: out must be a C-contiguous float64 array of the state's shape")
        _chk("icarus_get_state", self.lib.icarus_get_state(self.ctx, member, _dp(out), out.size))
        return out

    def get_tracer(self, member=0):
        """CME tracer rho X of a member's interior cells, [leaf][i][j][k]"""
        out = np.zeros((self.n_leaves(member),) + self.block)
        f = self.lib.icarus_get_tracer
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_size_t]
        _chk("icarus_get_tracer", f(self.ctx, member, _dp(out), out.size))
        return out

    def set_tracer(self, member, T):
        T = np.ascontiguousarray(T, dtype=np.float64).reshape((self.n_leaves(member),) + self.block)
        f = self.lib.icarus_set_tracer
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_size_t]
        _chk("icarus_set_tracer", f(self.ctx, member, _dp(T), T.size))

    def get_padded(self, member, leaf):
        """a leaf block with its ghost layers as last filled (FP64 conserved)"""
        out = np.zeros((8,) + tuple(b + 4 for b in self.block))
        _chk("icarus_get_padded", self.lib.icarus_get_padded(self.ctx, member, leaf, _dp(out), out.size))
        return out

    def set_time(self, member, t):
        _chk("icarus_set_time", self.lib.icarus_set_time(self.ctx, member, float(t)))

    def set_earth(self, member, colat, lon0, t0=0.0, rate=0.0):
        """Earth at colatitude colat, longitude lon0 - rate (t - t0) (shock windows)"""
        f = self.lib.icarus_set_earth
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        _chk("icarus_set_earth", f(self.ctx, member, float(colat), float(lon0), float(t0), float(rate)))

    def set_member_max_level(self, member, level):
        _chk("icarus_set_member_max_level", self.lib.icarus_set_member_max_level(self.ctx, member, level))

    def ghost_fill(self):
        _chk("icarus_ghost_fill", self.lib.icarus_ghost_fill(self.ctx))

    def sums(self, member=0):
        out = np.zeros(8)
        _chk("icarus_conservation_sums", self.lib.icarus_conservation_sums(self.ctx, member, _dp(out)))
        return out

    def dt(self):
        out = np.zeros(self.n_members)
        _chk("icarus_get_dt", self.lib.icarus_get_dt(self.ctx, _dp(out)))
        return out

    def cell_updates(self):
        out = np.zeros(self.n_members)
        f = self.lib.icarus_cell_updates
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
        _chk("icarus_cell_updates", f(self.ctx, _dp(out)))
        return out

    def status(self):
        w, f = C.c_uint32(0), C.c_uint64(0)
        _chk("icarus_status_word", self.lib.icarus_status_word(self.ctx, C.byref(w), C.byref(f)))
        return w.value, f.value

    def set_floor_budget(self, max_fraction):
        """Poison the context when a step's floor hits exceed this fraction of
        the leaf cells it advanced (0 disables the budget)."""
        _chk("icarus_set_floor_budget", self.lib.icarus_set_floor_budget(self.ctx, float(max_fraction)))

    def set_tile(self, tile_theta=0, tile_phi=0, r_segment=0):
        _chk("icarus_set_tile", self.lib.icarus_set_tile(self.ctx, tile_theta, tile_phi, r_segment))

    def set_direct_halo(self, enable=True):
        """stage kernels read same-level halos from the neighbouring leaves (1)
        or from ghost layers filled before every stage (0); same results"""
        f = self.lib.icarus_set_direct_halo
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.c_int]
        _chk("icarus_set_direct_halo", f(self.ctx, int(bool(enable))))

    def use_graph(self, enable=True):
        _chk("icarus_use_graph", self.lib.icarus_use_graph(self.ctx, int(bool(enable))))

    def kernels_per_step(self):
        n = C.c_int(0)
        _chk("icarus_kernels_per_step", self.lib.icarus_kernels_per_step(self.ctx, C.byref(n)))
        return n.value

    def save(self, path):
        """Checkpoint the context to a host file (see icarus_save)."""
        f = self.lib.icarus_save
        f.restype, f.argtypes = C.c_int, [C.c_void_p, C.c_char_p]
        _chk("icarus_save", f(self.ctx, os.fsencode(path)))

    def load(self, path):
        """Resume from a checkpoint written by a context with the same
        descriptor (see icarus_load)."""
        f = self.lib.icarus_load
        f.restype, f.argtypes = C.c_int, [C.c_void_p, C.c_char_p]
        _chk("icarus_load", f(self.ctx, os.fsencode(path)))

    def profile(self, enable=True):
        _chk("icarus_profile", self.lib.icarus_profile(self.ctx, int(bool(enable))))

    def profile_read(self):
        """(ms, count) per kernel kind since the last read (see PROFILE_KINDS)."""
        nk = len(PROFILE_KINDS)
        ms = np.zeros(nk)
        cnt = np.zeros(nk, dtype=np.int32)
        _chk("icarus_profile_read", self.lib.icarus_profile_read(self.ctx, _dp(ms),
                                                                 cnt.ctypes.data_as(C.POINTER(C.c_int)), nk))
        return ms, cnt


    # ---------------------------------------------------------------- learned pre-flagger
    def _mlp(self, name, *argtypes):
        f = getattr(self.lib, name)
        f.restype = C.c_int
        f.argtypes = [C.c_void_p] + list(argtypes)
        return f

    def mlp_set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _chk("icarus_mlp_set_params", self._mlp("icarus_mlp_set_params", C.c_void_p, C.c_size_t)(
            self.ctx, th.ctypes.data_as(C.c_void_p), th.size))

    def mlp_get_params(self):
        th = np.zeros(MLP_PARAMS, dtype=np.float32)
        _chk("icarus_mlp_get_params", self._mlp("icarus_mlp_get_params", C.c_void_p, C.c_size_t)(
            self.ctx, th.ctypes.data_as(C.c_void_p), th.size))
        return th

    def mlp_features(self):
        out = np.zeros((self.n_leaves(-1), 64), dtype=np.float32)
        _chk("icarus_mlp_features", self._mlp("icarus_mlp_features", C.c_void_p)(
            self.ctx, out.ctypes.data_as(C.c_void_p)))
        return out

    def mlp_predict_leaves(self):
        out = np.zeros(self.n_leaves(-1), dtype=np.float32)
        _chk("icarus_mlp_predict_leaves", self._mlp("icarus_mlp_predict_leaves", C.c_void_p)(
            self.ctx, out.ctypes.data_as(C.c_void_p)))
        return out

    def mlp_predict(self, X):
        """Probabilities of host feature rows (sent in batches of 4096, the
        entry point's limit)."""
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 64)
        y = np.zeros(X.shape[0], dtype=np.float32)
        f = self._mlp("icarus_mlp_predict", C.c_void_p, C.c_int, C.c_void_p)
        for a in range(0, X.shape[0], 4096):
            xa = np.ascontiguousarray(X[a:a + 4096])
            ya = np.zeros(xa.shape[0], dtype=np.float32)
            _chk("icarus_mlp_predict", f(self.ctx, xa.ctypes.data_as(C.c_void_p), xa.shape[0],
                                         ya.ctypes.data_as(C.c_void_p)))
            y[a:a + xa.shape[0]] = ya
        return y

    def mlp_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 64)
        T = np.ascontiguousarray(T, dtype=np.float32)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = C.c_float(0)
        f = self._mlp("icarus_mlp_grad", C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_float))
        _chk("icarus_mlp_grad", f(self.ctx, X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p), X.shape[0],
                                  g.ctypes.data_as(C.c_void_p), C.byref(loss)))
        return g, loss.value

    def mlp_dataset_clear(self):
        _chk("icarus_mlp_dataset_clear", self._mlp("icarus_mlp_dataset_clear")(self.ctx))

    def mlp_dataset_add(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 64)
        T = np.ascontiguousarray(T, dtype=np.float32)
        tot = C.c_int(0)
        f = self._mlp("icarus_mlp_dataset_add", C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int))
        _chk("icarus_mlp_dataset_add", f(self.ctx, X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p),
                                         X.shape[0], C.byref(tot)))
        return tot.value

    def mlp_train(self, n_train, epochs, batch=1024, lr=1e-3, seed=0):
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        f = self._mlp("icarus_mlp_train", C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_void_p)
        _chk("icarus_mlp_train", f(self.ctx, n_train, epochs, batch, lr, seed, losses.ctypes.data_as(C.c_void_p)))
        return losses[:epochs] / n_train


MLP_PARAMS = 128 * 64 + 128 + 128 * 128 + 128 + 128 + 1

PROFILE_KINDS = ["dt_begin", "ghost_neighbour", "ghost_physical", "stage_predictor", "stage_corrector",
                 "reflux", "dt_finalize", "estimator", "regrid_move", "dt_full"]
STEP_KINDS = 7   # the first seven kinds are the step's launches


def conservation_sums_static(g, member=0):
    """Sums of V * U over a member's leaves through the entry point that
    allocates nothing (its scratch is a fixed array inside the library)."""
    lib = g.lib
    f = lib.icarus_conservation_sums_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double)]
    out = np.zeros(8)
    _chk("icarus_conservation_sums_static", f(g.ctx, member, _dp(out)))
    return out


def alu_peak(kind, stream=None):
    """measured FMA throughput (flop/s): kind 0 FP64, 1 FP32, 2 FP32 packed pairs"""
    L = load()
    f = L.icarus_alu_peak
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    out = C.c_double(0.0)
    _chk("icarus_alu_peak", f(int(kind), stream, C.byref(out)))
    return out.value


def set_fp64_islands(g, p_over_e=0.002, beta=0.1):
    """FP32 mode: FP64 pressure recovery where p < p_over_e * e or p < beta * B^2/2."""
    f = g.lib.icarus_set_fp64_islands
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_double, C.c_double]
    _chk("icarus_set_fp64_islands", f(g.ctx, float(p_over_e), float(beta)))

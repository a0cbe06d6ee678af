"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/icarus.h declares."""
import ctypes
import os
import re

from paper_2211_12867_gb300 import build, icarus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(icarus_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(icarus.EXPORTS) <= names


def test_status_strings_without_gpu():
    lib = icarus.load()
    for code in range(8):
        s = lib.icarus_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0


def test_arena_size_and_argument_checks_without_gpu():
    lib = icarus.load()
    d = icarus.GridDesc()
    d.n_cells[:] = [60, 16, 32]
    d.block[:] = [12, 8, 8]
    d.max_level = 1
    d.x_min[:] = [0.1, 0.5, 0.0]
    d.x_max[:] = [1.1, 2.6, 6.283185307179586]
    d.gamma, d.cfl, d.divb_cd = 1.5, 0.8, 0.8
    d.n_members = 1
    d.bc_lo[:] = [3, 1, 0]
    d.bc_hi[:] = [1, 1, 0]
    n = ctypes.c_size_t(0)
    assert lib.icarus_arena_bytes(ctypes.byref(d), ctypes.byref(n)) == 0
    # FP64 state and stage buffers alone: 2 x 40 blocks x 8 x 16*12*12 x 8 bytes
    assert n.value >= 2 * 40 * 8 * 16 * 12 * 12 * 8
    d.block[:] = [7, 8, 8]        # odd block: rejected
    assert lib.icarus_arena_bytes(ctypes.byref(d), ctypes.byref(n)) == 1
    d.block[:] = [12, 8, 8]
    d.bc_lo[2] = 1                # periodic on one side only: rejected
    assert lib.icarus_arena_bytes(ctypes.byref(d), ctypes.byref(n)) == 1
    ctx = ctypes.c_void_p()
    d.bc_lo[2] = 0
    d.arena = None
    assert lib.icarus_init_grid(ctypes.byref(d), ctypes.byref(ctx)) == 2   # no arena

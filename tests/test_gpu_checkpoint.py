"""Checkpoint and resume: a context restored from icarus_save continues bit
for bit as the saved one does (single level FP64, and AMR FP32 with a cone
CME across regrids); a checkpoint of another descriptor or a foreign file is
refused and leaves the context as it was."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, wind_setup
from paper_2211_12867_gb300 import inputs as I
from paper_2211_12867_gb300.icarus import FP32_MIXED, IcarusError

pytestmark = pytest.mark.gpu
STR = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi), stretch=True)
CRIT = dict(e_refine=0.05, e_coarsen=0.01, eps=0.01, dv=I.kms(50.0))


def test_resume_single_level_fp64(tmp_path):
    g, o = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    wind_setup(g, o)
    g.step(5)
    path = str(tmp_path / "a.ck")
    g.save(path)
    t_a = g.step(7)
    A = g.get_state(0)
    h, _ = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    h.load(path)
    t_b = h.step(7)
    assert np.array_equal(t_a, t_b)
    assert np.array_equal(A, h.get_state(0))
    assert np.array_equal(g.cell_updates(), h.cell_updates())


def test_resume_amr_fp32_across_regrids(tmp_path):
    def run(g, n):
        for _ in range(n):
            g.step(4)
            g.flag_refine(**CRIT)
            g.regrid()
    g, o = make_pair(n=(48, 24, 48), nb=(12, 12, 12), max_level=3, precision=FP32_MIXED, max_blocks=3000, **STR)
    wind_setup(g, o)
    g.step(20)
    t0 = g.step(0)[0]
    g.inject_cone_cme(0, t_start=t0, **I.cme_config2(seed=0))
    run(g, 3)
    path = str(tmp_path / "b.ck")
    g.save(path)
    run(g, 3)
    t_a = g.step(3)
    h, _ = make_pair(n=(48, 24, 48), nb=(12, 12, 12), max_level=3, precision=FP32_MIXED, max_blocks=4000, **STR)
    h.load(path)
    run(h, 3)
    t_b = h.step(3)
    assert np.array_equal(g.tree(0), h.tree(0))
    assert g.tree(0)[:, 0].max() > 1, "the run must refine"
    assert np.array_equal(t_a, t_b)
    assert np.array_equal(g.get_state(0), h.get_state(0))


def test_foreign_or_mismatched_checkpoints_are_refused(tmp_path):
    g, o = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    wind_setup(g, o)
    g.step(2)
    path = str(tmp_path / "c.ck")
    g.save(path)
    other, _ = make_pair(n=(48, 16, 32), nb=(12, 8, 8), cfl=0.5)
    before = other.get_state(0)
    with pytest.raises(IcarusError):
        other.load(path)
    assert np.array_equal(before, other.get_state(0))
    bad = tmp_path / "d.ck"
    bad.write_bytes(b"not a checkpoint" * 8)
    with pytest.raises(IcarusError):
        g.load(str(bad))
    with pytest.raises(IcarusError):
        g.load(str(tmp_path / "missing.ck"))


def test_checkpoint_without_preflagger_clears_the_loaded_one(tmp_path):
    """A context restored from a checkpoint saved without pre-flagger
    parameters has none either, even if it had some before the load."""
    g, o = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    wind_setup(g, o)
    path = str(tmp_path / "e.ck")
    g.save(path)
    h, _ = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    h.mlp_set_params(I.mlp_init(1).astype(np.float32))
    h.mlp_predict(np.zeros((4, 64), np.float32))
    h.load(path)
    with pytest.raises(IcarusError):
        h.mlp_predict(np.zeros((4, 64), np.float32))


def _ck_rows_offset(raw):
    # magic, version, field count, descriptor fields, then member 0's
    # (max level, leaf count) and its cone CME record (8 doubles, 2 ints)
    nfp = int(np.frombuffer(bytes(raw[12:16]), dtype=np.uint32)[0])
    return 8 + 4 + 4 + 8 * nfp + 8 + 72


def test_corrupt_trees_are_refused(tmp_path):
    """A checkpoint whose leaf list is not a valid tree (a duplicate leaf, a
    leaf count beyond the pool) is refused and the context is unchanged."""
    g, o = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    wind_setup(g, o)
    path = tmp_path / "f.ck"
    g.save(str(path))
    raw = bytearray(path.read_bytes())
    off = _ck_rows_offset(raw)
    rows = np.frombuffer(bytes(raw[off:off + 16 * 32]), dtype=np.int32).reshape(32, 4)
    assert np.array_equal(rows, g.tree(0))          # the offsets above are right
    dup = bytearray(raw)
    dup[off + 16:off + 32] = raw[off:off + 16]
    (tmp_path / "dup.ck").write_bytes(bytes(dup))
    big = bytearray(raw)
    big[off - 76:off - 72] = np.int32(2 ** 30).tobytes()
    (tmp_path / "big.ck").write_bytes(bytes(big))
    h, _ = make_pair(n=(48, 16, 32), nb=(12, 8, 8))
    wind_setup(h, _)
    h.step(1)
    before = h.get_state(0)
    for name in ("dup.ck", "big.ck"):
        with pytest.raises(IcarusError):
            h.load(str(tmp_path / name))
        assert np.array_equal(before, h.get_state(0))

"""Floors and the floor budget on the GPU.

Density and pressure floors are applied after every stage and counted.  A
step whose floor hits exceed the budget (a fraction of the leaf cells it
advanced) sets the floor bit of the sticky status word; the next call that
reads the word returns ICARUS_ERR_NONPHYSICAL and the context is poisoned.
Non-physical states are made on the host (negative pressure written through
icarus_set_state); nothing here faults the device."""
import numpy as np
import pytest

from gpu_common import make_pair, wind_setup
from paper_2211_12867_gb300.icarus import IcarusError

pytestmark = pytest.mark.gpu
NONPHYSICAL, STATE = 4, 6


def _negative_pressure(g, o, cells=10, p=-1e6):
    """the wind state with `cells` cells of block 3 at pressure p (deep
    enough that the fluxes cannot refill the cell within one stage)"""
    wind_setup(g, o)
    U = g.get_state(0)
    for q in range(cells):
        i, j, k = 2 + q % 5, 2 + q // 5, 3
        ke = 0.5 * (U[3, 1, i, j, k] ** 2 + U[3, 2, i, j, k] ** 2 + U[3, 3, i, j, k] ** 2) / U[3, 0, i, j, k]
        me = 0.5 * (U[3, 5, i, j, k] ** 2 + U[3, 6, i, j, k] ** 2 + U[3, 7, i, j, k] ** 2)
        U[3, 4, i, j, k] = ke + me + p / (g.desc.gamma - 1.0)
    g.set_state(0, U)


def test_floors_are_counted_within_the_budget():
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    _negative_pressure(g, o)
    w0, h0 = g.status()
    g.step(2)
    w, h = g.status()
    assert h > h0, "the negative pressures must be floored"
    assert w == 0, "10 cells of 30720 stay within the default budget"
    # the state is physical again
    U = g.get_state(0)
    p = (g.desc.gamma - 1) * (U[:, 4] - 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / U[:, 0]
                              - 0.5 * (U[:, 5] ** 2 + U[:, 6] ** 2 + U[:, 7] ** 2))
    assert p.min() > 0


def test_budget_exceeded_poisons_the_context():
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    _negative_pressure(g, o)
    g.set_floor_budget(1e-9)            # any floor hit is over budget
    with pytest.raises(IcarusError) as e:
        g.step(1)
    assert e.value.code == NONPHYSICAL
    w, h = g.status()
    assert w & 2 and h > 0
    with pytest.raises(IcarusError) as e:
        g.step(1)
    assert e.value.code == STATE
    g.get_state(0)                      # still readable


def test_budget_off_and_physical_state_untouched():
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    _negative_pressure(g, o)
    g.set_floor_budget(0.0)             # no budget: floors are only counted
    g.step(2)
    assert g.status()[0] == 0
    h, _ = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    wind_setup(h, _)
    h.set_floor_budget(1e-9)
    h.step(5)                           # the plain wind needs no floor
    assert h.status() == (0, 0)


def test_status_of_an_unsynchronised_step_reaches_the_next_call():
    """step without times and without stop times does not synchronise; its
    status word follows it to the host and the next step reports it."""
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8))
    _negative_pressure(g, o)
    g.set_floor_budget(1e-9)
    g.step(1, want_time=False)          # returns at once, no error yet
    g.stream.synchronize()
    with pytest.raises(IcarusError) as e:
        g.step(1, want_time=False)
    assert e.value.code == NONPHYSICAL

"""FP32 mode (FP32 state and stencil, FP64 pressure islands, FP64 time-step
reduction) against the FP64 oracle on the same seeded inputs.  The error is
reported per variable; the bound is a sanity bound for a second-order scheme
run in single precision, not a parity claim."""
import json
import os

import numpy as np
import pytest

from gpu_common import make_pair, rel_linf, wind_setup
from paper_2211_12867_gb300.icarus import set_fp64_islands

pytestmark = pytest.mark.gpu
# reports of measured figures go to $ICARUS_REPORT_DIR (default: reports/)
OUT = os.environ.get("ICARUS_REPORT_DIR",
                     os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "reports"))


@pytest.mark.parametrize("islands", [(0.05, 0.1), (0.002, 0.1), (0.0, 0.0)])
def test_fp32_mode_error_vs_oracle(islands):
    g, o = make_pair(n=(60, 16, 32), nb=(12, 8, 8), precision=1)
    set_fp64_islands(g, *islands)
    wind_setup(g, o)
    # the oracle starts from the FP32-rounded state the GPU holds
    errs = []
    for chunk in range(4):
        t = g.step(50)
        o.advance(50)
        assert abs(t[0] - o.t) / o.t < 1e-4
        errs.append(rel_linf(g.get_state(0), o.get_state()).tolist())
    os.makedirs(OUT, exist_ok=True)
    with open(os.path.join(OUT, f"fp32_err_{islands[0]}_{islands[1]}.json"), "w") as f:
        json.dump({"islands": islands, "steps": [50, 100, 150, 200], "rel_linf_per_var": errs}, f)
    assert max(errs[-1]) < 1e-2, errs[-1]

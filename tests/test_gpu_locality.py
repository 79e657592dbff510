"""The locality-model sweep runs through the library on the GPU and yields
finite predicted and measured speedups for both restructured layouts."""
import math

import pytest

from paper_2511_21535_gb300 import locality as lm

pytestmark = pytest.mark.gpu


def test_locality_sweep_small(dev):
    res = lm.sweep(steps=2, warmup=1, names=["grid64_leaf4"], device=dev)
    rows = res["rows"]
    assert {r["layout"] for r in rows} == {"redundant", "pairtask"}
    for r in rows:
        for k in ("pred_x_compute", "meas_x_kernel", "pred_x_p2p", "meas_x_e2e"):
            assert math.isfinite(r[k]) and r[k] > 0
        assert r["D_layout"] < r["D_indirect"]
    assert "| grid64_leaf4 |" in lm.to_markdown(res)

"""The checked library variant on randomized plans, and the release library on
inconsistent imported structures.

The checked variant (built with P2P_CHECKED) validates every work item of the
P2P loop -- box, target range, neighbour source ranges, partial-result slots
-- against the plan's capacities and records P2P_FLAG_BOUNDS instead of
touching memory out of range.  Randomized plans across kernels, layouts,
evaluation modes, boundary conditions, distributions and tunings must run
with no failed check and match the FP64 oracle.  It runs in a child process
so that the variant is the library that process loads.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2511_21535_gb300 import build as cuda_build
from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAG_CAPACITY, FLAG_BOUNDS = 0x4, 0x10


@pytest.mark.parametrize("seed", [1, 2])
def test_checked_variant_randomized(seed):
    cuda_build.build(variants=("checked",))
    env = dict(os.environ, P2P_GB300_VARIANT="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), "40", str(seed)],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    rows = [json.loads(line) for line in r.stdout.splitlines() if line.startswith("{")]
    assert len(rows) == 40
    ran = [x for x in rows if "refused" not in x]
    for x in rows:
        if "refused" in x:
            assert x["refused"] in (1, 5), x       # invalid argument / unsupported combination
    assert len(ran) >= 36                           # the draws avoid the combinations refused by design
    for x in ran:
        assert x["status"] == 0 and not (x["flags"] & FLAG_BOUNDS), x
        assert x["err"] <= x["tol"], x
    modes = {x["case"]["mode"] for x in ran}
    assert {"indirect", "redundant", "pairtask"} <= modes


def _tree(prob):
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    return {k: np.array(t[k], dtype=np.int32) for k in ("perm", "box_start", "nbr_start", "nbr_idx")}


def _corrupt(t, how):
    t = {k: v.copy() for k, v in t.items()}
    if how == "nbr_idx_out_of_range":
        t["nbr_idx"][len(t["nbr_idx"]) // 2] = len(t["box_start"]) - 1
    elif how == "negative_nbr_idx":
        t["nbr_idx"][3] = -1
    elif how == "perm_out_of_range":
        t["perm"][7] = len(t["perm"])
    elif how == "empty_box":
        t["box_start"][2] = t["box_start"][1]
    elif how == "box_bounds_short":
        t["box_start"][-1] -= 1
    elif how == "neighbour_bounds_decreasing":
        t["nbr_start"][5], t["nbr_start"][6] = t["nbr_start"][6], t["nbr_start"][5]
    return t


@pytest.mark.parametrize("layout", ["indirect", "redundant", "pairtask"])
@pytest.mark.parametrize("how", ["nbr_idx_out_of_range", "negative_nbr_idx", "perm_out_of_range", "empty_box",
                                 "box_bounds_short", "neighbour_bounds_decreasing"])
def test_inconsistent_import_is_rejected(dev, layout, how):
    """An imported structure that breaks its invariants sets P2P_FLAG_CAPACITY on
    the device; restructuring and the operator then do no work and the counters
    report P2P_ERR_INVALID_ARG.  A consistent import afterwards works again."""
    prob = wl.uniform_gravity(n=4096, level=3)
    good = _tree(prob)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    m = torch.from_numpy(prob.strength).to(dev)
    bad = _corrupt(good, how)
    plan.tree_import(*(torch.from_numpy(bad[k]).to(dev) for k in ("perm", "box_start", "nbr_start", "nbr_idx")))
    plan.restructure(pos, m)
    plan.gravity(prob.eps)
    c = plan.counters()
    assert c["status"] == 1 and (c["flags"] & FLAG_CAPACITY), c
    plan.tree_import(*(torch.from_numpy(good[k]).to(dev) for k in ("perm", "box_start", "nbr_start", "nbr_idx")))
    plan.restructure(pos, m)
    phi, acc = plan.gravity(prob.eps)
    c = plan.counters()
    assert c["status"] == 0 and c["flags"] == 0, c
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert np.linalg.norm(phi.cpu().numpy() - ophi) <= 1e-5 * np.linalg.norm(ophi)

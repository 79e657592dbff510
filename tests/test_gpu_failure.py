"""Failure detection without a GPU fault: a bounded device wait that nothing
completes runs out and reports P2P_ERR_TIMEOUT; the context stays usable.
Errors the host can see (bad arguments, out-of-domain points, calls out of
order) come back as status codes."""
import time

import numpy as np
import pytest
import torch

from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports(dev):
    t0 = time.perf_counter()
    st = p2p.selftest_bounded_wait(limit_ns=5_000_000, device=dev)     # 5 ms
    dt = time.perf_counter() - t0
    assert st == 4                                                    # P2P_ERR_TIMEOUT
    assert dt < 5.0
    # the context is still usable: a normal operator call afterwards works
    prob = wl.uniform_gravity(n=2000, level=2)
    pos = torch.from_numpy(prob.pos).to(dev)
    m = torch.from_numpy(prob.strength).to(dev)
    phi, acc = p2p.gravity(pos, m, prob.level, prob.lo, prob.edge, prob.eps)
    torch.cuda.synchronize()
    assert torch.isfinite(phi).all() and torch.isfinite(acc).all()


def test_selftest_rejects_bad_limits(dev):
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    lib = p2p.load()
    assert lib.p2p_selftest_bounded_wait(0, flags.data_ptr(), None) == 1
    assert lib.p2p_selftest_bounded_wait(20_000_000_000, flags.data_ptr(), None) == 1


def test_host_visible_errors(dev):
    prob = wl.uniform_gravity(n=500, level=2)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    with pytest.raises(TypeError):
        plan.tree_build(pos.double())
    with pytest.raises(p2p.P2PError) as e:
        plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))   # before the tree
    assert e.value.status == 8
    small = torch.empty(16, dtype=torch.uint8, device=dev)
    with pytest.raises(ValueError):
        p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, device=dev, workspace=small)
    bad = prob.pos.copy()
    bad[3] = np.nan
    plan.tree_build(torch.from_numpy(bad).to(dev))
    assert plan.counters()["status"] == 6                              # P2P_ERR_DOMAIN

"""One step from host buffers (P2P_PLAN_HOST_IO): the copies, tree build,
restructuring, operator and copy back in one call give bitwise the results of
the device-pointer calls on the same plan, with pinned or pageable buffers."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def host(t, pinned):
    t = torch.from_numpy(np.ascontiguousarray(t))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("layout,symmetric", [("redundant", False), ("indirect", False), ("pairtask", False),
                                              ("redundant", True)])
@pytest.mark.parametrize("pinned", [True, False])
def test_gravity_host_step(dev, layout, symmetric, pinned):
    prob = wl.plummer_gravity(n=30000, level=5, eps=1e-3, seed=9)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, symmetric=symmetric,
                    host_io=True, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    m = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, m)
    phi_d, acc_d = (t.cpu().numpy() for t in plan.gravity(prob.eps))
    phi_h = host(np.zeros(prob.n, np.float32), pinned)
    acc_h = host(np.zeros((prob.n, 3), np.float32), pinned)
    plan.gravity_host(prob.eps, host(prob.pos, pinned), host(prob.strength, pinned), phi_h, acc_h)
    torch.cuda.synchronize()
    assert plan.counters()["status"] == 0
    np.testing.assert_array_equal(phi_h.numpy(), phi_d)
    np.testing.assert_array_equal(acc_h.numpy(), acc_d)


@pytest.mark.parametrize("nrhs,symmetric", [(1, False), (2, True), (3, False)])
def test_helmholtz_host_step(dev, nrhs, symmetric):
    prob = wl.grid_helmholtz(edge_points=24, nrhs=nrhs, seed=nrhs)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=nrhs, symmetric=symmetric,
                    host_io=True, timing=True, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u_d = plan.helmholtz(prob.k).cpu().numpy()
    u_h = host(np.zeros((nrhs, prob.n), np.complex64), True)
    for _ in range(3):   # repeated steps reuse the plan's copy stream
        plan.helmholtz_host(prob.k, host(prob.pos, True), host(prob.strength, True), u_h)
    torch.cuda.synchronize()
    assert plan.counters()["status"] == 0
    np.testing.assert_array_equal(u_h.numpy(), u_d)
    assert plan.timing()["tree"] > 0
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert np.linalg.norm(u_h.numpy() - ou) <= 2e-5 * np.linalg.norm(ou)


def test_host_step_needs_the_flag(dev):
    prob = wl.uniform_gravity(n=1000, level=3)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, device=dev)
    z = torch.zeros(prob.n)
    with pytest.raises(p2p.P2PError) as e:
        plan.gravity_host(prob.eps, torch.from_numpy(prob.pos), torch.from_numpy(prob.strength), z,
                          torch.zeros(prob.n, 3))
    assert e.value.status == 5

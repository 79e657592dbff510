"""Pattern mode (tabulated G for particles on a regular lattice, the DBIM
solver's precomputed-pattern P2P) against the FP64 oracle on the actual
float32 positions, and its input checks."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_COMPLEX = 2e-5


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_pattern(prob, dev, layout, tpl=2, group=4, pattern=True):
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout, device=dev)
    plan.set_tuning(tpl, 64, 0, group)
    if pattern:
        plan.set_grid(wl.SPACING, wl.LEAF_EDGE_POINTS)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k)
    torch.cuda.synchronize()
    return plan, u.cpu().numpy()


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("edge,nrhs,tpl,group", [(16, 1, 2, 4), (24, 2, 1, 1), (32, 3, 2, 4), (16, 8, 1, 4)])
def test_pattern_matches_oracle(dev, layout, edge, nrhs, tpl, group):
    prob = wl.grid_helmholtz(edge_points=edge, nrhs=nrhs, seed=edge + nrhs)
    plan, u = run_pattern(prob, dev, layout, tpl, group)
    assert plan.counters(check=True)["flags"] == 0
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_pattern_full_64_grid(dev):
    prob = wl.grid_helmholtz()
    _, u = run_pattern(prob, dev, "redundant")
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    e = rel_l2(u, ou)
    print(f"\nACCURACY grid_helmholtz_64 pattern mode: rel-L2 {e:.3e}")
    assert e <= TOL_COMPLEX


def test_pattern_rejects_off_lattice_points(dev):
    prob = wl.grid_helmholtz(edge_points=16)
    pos = prob.pos.copy()
    pos[100, 0] += np.float32(0.02)      # 20 % of a spacing off the lattice
    bad = wl.Problem("bad", pos, prob.strength, prob.level, prob.lo, prob.edge, "helmholtz", k=prob.k)
    plan, u = run_pattern(bad, dev, "redundant")
    c = plan.counters()
    assert c["flags"] & p2p.FLAG_LATTICE and c["status"] == 1


def test_pattern_argument_checks(dev):
    prob = wl.grid_helmholtz(edge_points=16)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, device=dev)
    with pytest.raises(p2p.P2PError):
        plan.set_grid(0.1, 5)           # table would not fit
    with pytest.raises(p2p.P2PError):
        plan.set_grid(0.1, 3)           # 3 points of 0.1 do not make the 0.4 leaf box
    plan.set_grid(0.1, 4)
    plan.set_grid(0.0, 0)               # off again


def test_pattern_adjoint_q(dev):
    prob = wl.grid_helmholtz(edge_points=24, nrhs=1, seed=9)
    rng = np.random.default_rng(10)
    gbar = wl.complex_normal((1, prob.n), rng)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=1, device=dev)
    plan.set_grid(wl.SPACING, wl.LEAF_EDGE_POINTS)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    gq, _ = plan.helmholtz_adjoint(prob.k, pos, torch.from_numpy(gbar).to(dev), want_q=True, want_pos=False)
    torch.cuda.synchronize()
    oq, _ = oracle.helmholtz_adjoint(prob.pos, prob.strength, gbar, prob.level, prob.lo, prob.edge, prob.k)
    assert rel_l2(gq.cpu().numpy(), oq) <= TOL_COMPLEX
    # the forward afterwards (records rebuilt) is still right
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k).cpu().numpy()
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert rel_l2(u, ou) <= TOL_COMPLEX

"""Pair-task layout on the GPU: one task per (target box, source box) entry,
block [records of b | records of c] per task, partial results per task and
a deterministic reduction in neighbour order.

The task list, task-stream bounds, partial-slot bounds and gather map must
be bit-exact against what the oracle's tree implies; sums must meet the
usual relative-L2 tolerances against the FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_REAL = 1e-5
TOL_COMPLEX = 2e-5


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def expected_tasks(t):
    """Task list implied by a tree: target box, block bounds, slot bounds, gather map."""
    bs = t["box_start"].astype(np.int64)
    ns = t["nbr_start"].astype(np.int64)
    ni = t["nbr_idx"].astype(np.int64)
    occ = np.diff(bs)
    ent = np.repeat(np.arange(t["n_boxes"]), np.diff(ns))
    blk = occ[ent] + occ[ni]
    pt_start = np.concatenate([[0], np.cumsum(blk)])
    part_start = np.concatenate([[0], np.cumsum(occ[ent])])
    gather = np.concatenate([np.concatenate([np.arange(bs[b], bs[b + 1]), np.arange(bs[c], bs[c + 1])])
                             for b, c in zip(ent, ni)]) if len(ent) else np.zeros(0, np.int64)
    return ent, pt_start, part_start, gather


def run(prob, dev, tpl=None, tile=64, group=4, periodic=False, gather=True):
    plan = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout="pairtask",
                    gather_map=gather, periodic=periodic, device=dev)
    if tpl:
        plan.set_tuning(tpl, tile, 0, group)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    if prob.kind == "gravity":
        phi, acc = plan.gravity(prob.eps)
        torch.cuda.synchronize()
        return plan, (phi.cpu().numpy(), acc.cpu().numpy())
    u = plan.helmholtz(prob.k)
    torch.cuda.synchronize()
    return plan, u.cpu().numpy()


def random_helmholtz(n, level, nrhs, seed, k=2 * math.pi):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3), dtype=np.float32)
    q = wl.complex_normal((nrhs, n), rng)
    return wl.Problem("random_helm", pos, q, level, (0.0, 0.0, 0.0), 1.0, "helmholtz", k=float(np.float32(k)))


CASES = {
    "uniform_8192_L3": lambda: wl.uniform_gravity(),
    "uniform_5_L1": lambda: wl.uniform_gravity(n=5, level=1),
    "plummer_60000_L6": lambda: wl.plummer_gravity(n=60000, level=6, eps=1e-3, seed=1),
    "grid16_r1": lambda: wl.grid_helmholtz(edge_points=16, nrhs=1),
    "grid24_r3": lambda: wl.grid_helmholtz(edge_points=24, nrhs=3, seed=1),
    "random_r16": lambda: random_helmholtz(2000, 2, 16, 9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_pairtask_structures_bit_exact(dev, name):
    prob = CASES[name]()
    plan, _ = run(prob, dev)
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    ent, pt_start, part_start, gather = expected_tasks(t)
    c = plan.counters(check=True)
    E = t["n_nbr"]
    assert c["n_nbr"] == E
    assert c["total_src"] == pt_start[-1]
    np.testing.assert_array_equal(plan.array("ent_box", E).cpu().numpy(), ent)
    np.testing.assert_array_equal(plan.array("pt_start", E + 1).cpu().numpy(), pt_start)
    np.testing.assert_array_equal(plan.array("part_start", E + 1).cpu().numpy(), part_start)
    np.testing.assert_array_equal(plan.array("gather_idx", int(pt_start[-1])).cpu().numpy().view(np.uint32), gather)
    assert c["pairs"] == oracle.pair_count(prob.pos, prob.level, prob.lo, prob.edge)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tpl,tile,group", [(1, 32, 1), (2, 64, 2), (2, 64, 4), (4, 64, 1)])
def test_pairtask_parity(dev, name, tpl, tile, group):
    prob = CASES[name]()
    _, out = run(prob, dev, tpl, tile, group)
    if prob.kind == "gravity":
        ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
        phi, acc = out
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
        assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL
    else:
        ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
        assert rel_l2(out, ou) <= TOL_COMPLEX


def test_pairtask_gravity_tpl4(dev):
    prob = wl.plummer_gravity(n=40000, level=5, eps=1e-3, seed=3)
    _, (phi, acc) = run(prob, dev, 4, 64, 4)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL


def test_pairtask_deterministic_and_close_to_target_owned(dev):
    prob = wl.plummer_gravity(n=40000, level=5, eps=1e-3, seed=4)
    _, (p1, a1) = run(prob, dev)
    _, (p2, a2) = run(prob, dev)
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(a1, a2)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout="redundant", device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    p3, a3 = (t.cpu().numpy() for t in plan.gravity(prob.eps))
    assert rel_l2(p1, p3) < 1e-6 and rel_l2(a1, a3) < 1e-6


def test_pairtask_periodic(dev):
    prob = wl.uniform_gravity(n=20000, level=4, seed=6)
    plan, (phi, acc) = run(prob, dev, periodic=True)
    ophi, oacc, pairs = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps,
                                       periodic=True)
    assert plan.counters(check=True)["pairs"] == pairs
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL
    hprob = wl.grid_helmholtz(edge_points=16, nrhs=2, seed=7)
    _, u = run(hprob, dev, periodic=True)
    ou, _ = oracle.helmholtz(hprob.pos, hprob.strength, hprob.level, hprob.lo, hprob.edge, hprob.k, periodic=True)
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_pairtask_grid_64_full(dev):
    prob = wl.grid_helmholtz()
    plan, u = run(prob, dev, gather=False)
    ou, pairs = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert plan.counters(check=True)["pairs"] == pairs
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_pairtask_plummer_full_sampled(dev):
    # the clustered 4M-particle workload: heavy boxes give tasks of very unequal cost
    prob = wl.plummer_gravity()
    plan, (phi, acc) = run(prob, dev, gather=False)
    c = plan.counters(check=True)
    tg = np.random.default_rng(0).choice(prob.n, 3000, replace=False)
    bs = plan.array("box_start", c["n_boxes"] + 1).cpu().numpy()
    b = int(np.argmax(np.diff(bs)))
    perm = plan.array("perm", prob.n).cpu().numpy()
    tg = np.unique(np.concatenate([tg, perm[bs[b]:bs[b + 1]]]))
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, targets=tg)
    assert rel_l2(phi[tg], ophi) <= TOL_REAL and rel_l2(acc[tg], oacc) <= TOL_REAL


def test_pairtask_refusals(dev):
    prob = wl.grid_helmholtz(edge_points=16)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, layout="pairtask", device=dev)
    with pytest.raises(p2p.P2PError) as e:
        plan.set_grid(wl.SPACING, 4)
    assert e.value.status == 5                                          # P2P_ERR_UNSUPPORTED
    pos = torch.from_numpy(prob.pos).to(dev)
    q = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(pos)
    with pytest.raises(p2p.P2PError) as e:
        plan.helmholtz_adjoint(prob.k, pos, q)
    assert e.value.status == 5
    with pytest.raises(p2p.P2PError) as e:
        p2p.Plan("gravity", 100, 2, (0, 0, 0), 1.0, layout="pairtask", adjoint=True, device=dev)
    assert e.value.status == 1                                          # P2P_ERR_INVALID_ARG

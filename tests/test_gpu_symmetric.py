"""Symmetric pair tasks on the GPU: mutual tasks evaluate each pair of an
unordered box pair once and credit both particles; the task kinds, mirrors,
block and slot bounds must be bit-exact against what the oracle's tree
implies, the sums within the usual relative-L2 tolerances of the FP64 oracle.
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
MUTUAL_MAX = 64          # largest box a mutual task holds (two targets per lane)
NONE, SELF, MUTUAL, ONESIDED = 0, 1, 2, 3


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def expected_tasks(t):
    """Task kinds, mirrors, block and slot bounds implied by a tree."""
    bs = t["box_start"].astype(np.int64)
    ns = t["nbr_start"].astype(np.int64)
    ni = t["nbr_idx"].astype(np.int64)
    occ = np.diff(bs)
    kinds, mirror, blk, slots = [], [], [], []
    for b in range(t["n_boxes"]):
        for e in range(ns[b], ns[b + 1]):
            c = int(ni[e])
            if c == b:
                k = SELF
            else:
                lo, hi = min(b, c), max(b, c)
                lane = lo if occ[lo] <= MUTUAL_MAX else (hi if occ[hi] <= MUTUAL_MAX else -1)
                k = ONESIDED if lane < 0 else (MUTUAL if lane == b else NONE)
            m = -1
            if k == NONE:
                lst = list(ni[ns[c]:ns[c + 1]])
                m = int(ns[c]) + lst.index(b)
            kinds.append(k)
            mirror.append(m)
            blk.append(0 if k == NONE else (occ[b] if k == SELF else occ[b] + occ[c]))
            slots.append(0 if k == NONE else (occ[b] + occ[c] if k == MUTUAL else occ[b]))
    return (np.array(kinds), np.array(mirror), np.concatenate([[0], np.cumsum(blk)]),
            np.concatenate([[0], np.cumsum(slots)]))


def run(prob, dev, group=None, periodic=False, plain=False):
    plan = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout="symmetric",
                    periodic=periodic, plain_fp32=plain, device=dev)
    if group:
        plan.set_tuning(2, 64, 0, group)
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
    "uniform_40000_L3_onesided": lambda: wl.uniform_gravity(n=40000, level=3, seed=3),
    "uniform_5_L1": lambda: wl.uniform_gravity(n=5, level=1),
    "plummer_60000_L6": lambda: wl.plummer_gravity(n=60000, level=6, eps=1e-3, seed=1),
    "grid16_r1": lambda: wl.grid_helmholtz(edge_points=16, nrhs=1),
    "grid24_r2": lambda: wl.grid_helmholtz(edge_points=24, nrhs=2, seed=1),
    "random_r2_ragged": lambda: random_helmholtz(3001, 2, 2, 9),
    "random_r1_onesided": lambda: random_helmholtz(9000, 2, 1, 10),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_symmetric_structures_bit_exact(dev, name):
    prob = CASES[name]()
    plan, _ = run(prob, dev)
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    kinds, mirror, pt_start, part_start = expected_tasks(t)
    E = t["n_nbr"]
    c = plan.counters(check=True)
    assert c["n_nbr"] == E and c["total_src"] == pt_start[-1]
    np.testing.assert_array_equal(plan.array("task_kind", E).cpu().numpy(), kinds)
    got_m = plan.array("mirror", E).cpu().numpy()
    np.testing.assert_array_equal(got_m[kinds == NONE], mirror[kinds == NONE])
    np.testing.assert_array_equal(plan.array("pt_start", E + 1).cpu().numpy(), pt_start)
    np.testing.assert_array_equal(plan.array("part_start", E + 1).cpu().numpy(), part_start)
    assert c["pairs"] == oracle.pair_count(prob.pos, prob.level, prob.lo, prob.edge)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("group", [1, 2, 4])
def test_symmetric_parity(dev, name, group):
    prob = CASES[name]()
    _, out = run(prob, dev, group)
    if prob.kind == "gravity":
        ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
        phi, acc = out
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
        if prob.n > 1:
            assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL
    else:
        ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
        assert np.all(np.isfinite(out))
        assert rel_l2(out, ou) <= TOL_COMPLEX


def test_symmetric_uses_mutual_tasks(dev):
    prob = wl.grid_helmholtz(edge_points=16)
    plan, _ = run(prob, dev)
    E = plan.counters()["n_nbr"]
    kinds = plan.array("task_kind", E).cpu().numpy()
    assert (kinds == MUTUAL).sum() == (kinds == NONE).sum() == (E - (kinds == SELF).sum()) // 2


def test_symmetric_deterministic(dev):
    prob = wl.plummer_gravity(n=40000, level=5, eps=1e-3, seed=4)
    _, (p1, a1) = run(prob, dev)
    _, (p2, a2) = run(prob, dev)
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(a1, a2)


def test_symmetric_momentum(dev):
    prob = wl.uniform_gravity(n=30000, level=4, seed=10)
    _, (_, acc) = run(prob, dev)
    f = acc.astype(np.float64) * prob.strength.astype(np.float64)[:, None]
    assert np.abs(f.sum(axis=0)).max() <= 1e-6 * np.abs(f).sum()


def test_symmetric_periodic(dev):
    prob = wl.uniform_gravity(n=20000, level=4, seed=6)
    _, (phi, acc) = run(prob, dev, periodic=True)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, periodic=True)
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL
    hprob = wl.grid_helmholtz(edge_points=16, nrhs=2, seed=7)
    _, u = run(hprob, dev, periodic=True)
    ou, _ = oracle.helmholtz(hprob.pos, hprob.strength, hprob.level, hprob.lo, hprob.edge, hprob.k, periodic=True)
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_symmetric_grid_64_full(dev):
    prob = wl.grid_helmholtz()
    plan, u = run(prob, dev)
    ou, pairs = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert plan.counters(check=True)["pairs"] == pairs
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_symmetric_plummer_full_sampled(dev):
    prob = wl.plummer_gravity()
    plan, (phi, acc) = run(prob, dev)
    c = plan.counters(check=True)
    tg = np.random.default_rng(0).choice(prob.n, 3000, replace=False)
    bs = plan.array("box_start", c["n_boxes"] + 1).cpu().numpy()
    b = int(np.argmax(np.diff(bs)))
    perm = plan.array("perm", prob.n).cpu().numpy()
    tg = np.unique(np.concatenate([tg, perm[bs[b]:bs[b + 1]]]))
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, targets=tg)
    assert rel_l2(phi[tg], ophi) <= TOL_REAL and rel_l2(acc[tg], oacc) <= TOL_REAL


def test_symmetric_refusals(dev):
    with pytest.raises(p2p.P2PError) as e:
        p2p.Plan("helmholtz", 100, 2, (0, 0, 0), 1.0, nrhs=3, layout="symmetric", device=dev)
    assert e.value.status == 1
    prob = random_helmholtz(4000, 2, 1, 11, k=60.0)          # k r_max > 32: accurate sine/cosine path
    with pytest.raises(p2p.P2PError) as e:
        run(prob, dev)
    assert e.value.status == 5
    prob = wl.grid_helmholtz(edge_points=16)
    with pytest.raises(p2p.P2PError) as e:
        run(prob, dev, plain=True)
    assert e.value.status == 5
    plan = p2p.Plan("gravity", 8192, 3, (0, 0, 0), 1.0, layout="symmetric", device=dev)
    plan.set_tuning(1, 64, 0, 1)
    g = wl.uniform_gravity()
    pos = torch.from_numpy(g.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(g.strength).to(dev))
    with pytest.raises(p2p.P2PError) as e:
        plan.gravity(g.eps)
    assert e.value.status == 5


# ---------------------------------------------------------------------------
# symmetric evaluation on the target-owned layouts (P2P_PLAN_SYMMETRIC)
# ---------------------------------------------------------------------------

def expected_flag_arrays(t):
    """Kinds, mirrors and source-sum slots of a symmetric plan, from the tree."""
    kinds, mirror, _, _ = expected_tasks(t)
    ni = t["nbr_idx"].astype(np.int64)
    occ = np.diff(t["box_start"].astype(np.int64))
    bsz = np.where(kinds == MUTUAL, occ[ni], 0)
    bslot = np.concatenate([[0], np.cumsum(bsz)])[:-1]
    return kinds, mirror, bslot, int(bsz.sum())


def run_flag(prob, dev, layout, group=None, periodic=False):
    plan = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    periodic=periodic, symmetric=True, device=dev)
    if group:
        plan.set_tuning(2, 64, 0, group)
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


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_symmetric_flag_structures(dev, name, layout):
    prob = CASES[name]()
    plan, _ = run_flag(prob, dev, layout)
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    kinds, mirror, bslot, btotal = expected_flag_arrays(t)
    E = t["n_nbr"]
    c = plan.counters(check=True)
    np.testing.assert_array_equal(plan.array("task_kind", E).cpu().numpy(), kinds)
    got_m = plan.array("mirror", E).cpu().numpy()
    np.testing.assert_array_equal(got_m[kinds == NONE], mirror[kinds == NONE])
    got_b = plan.array("bslot", E).cpu().numpy()
    np.testing.assert_array_equal(got_b[kinds == MUTUAL], bslot[kinds == MUTUAL])
    assert c["pairs"] == oracle.pair_count(prob.pos, prob.level, prob.lo, prob.edge)
    # evaluations: every ordered pair except the mirror entries' (evaluated by the mutual side)
    occ = np.diff(t["box_start"].astype(np.int64))
    ent = np.repeat(np.arange(t["n_boxes"]), np.diff(t["nbr_start"]))
    ni = t["nbr_idx"].astype(np.int64)
    assert c["evals"] == int((occ[ent] * occ[ni])[kinds != NONE].sum()) - prob.n
    if layout == "redundant":
        assert c["total_src"] == int(occ[ni][kinds != NONE].sum())


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("group", [1, 2, 4])
def test_symmetric_flag_parity(dev, name, layout, group):
    prob = CASES[name]()
    _, out = run_flag(prob, dev, layout, group)
    if prob.kind == "gravity":
        ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
        phi, acc = out
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
        if prob.n > 1:
            assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL
    else:
        ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
        assert np.all(np.isfinite(out))
        assert rel_l2(out, ou) <= TOL_COMPLEX


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_symmetric_flag_periodic(dev, layout):
    prob = wl.uniform_gravity(n=20000, level=4, seed=6)
    _, (phi, acc) = run_flag(prob, dev, layout, periodic=True)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, periodic=True)
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL
    hprob = wl.grid_helmholtz(edge_points=16, nrhs=2, seed=7)
    _, u = run_flag(hprob, dev, layout, periodic=True)
    ou, _ = oracle.helmholtz(hprob.pos, hprob.strength, hprob.level, hprob.lo, hprob.edge, hprob.k, periodic=True)
    assert rel_l2(u, ou) <= TOL_COMPLEX


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_symmetric_flag_grid_64_full(dev, layout):
    prob = wl.grid_helmholtz()
    plan, u = run_flag(prob, dev, layout)
    ou, pairs = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert plan.counters(check=True)["pairs"] == pairs
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_symmetric_flag_deterministic_and_momentum(dev):
    prob = wl.uniform_gravity(n=30000, level=4, seed=10)
    _, (p1, a1) = run_flag(prob, dev, "redundant")
    _, (p2, a2) = run_flag(prob, dev, "redundant")
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(a1, a2)
    f = a1.astype(np.float64) * prob.strength.astype(np.float64)[:, None]
    assert np.abs(f.sum(axis=0)).max() <= 1e-6 * np.abs(f).sum()


def test_symmetric_flag_plummer_sampled(dev):
    prob = wl.plummer_gravity(n=1 << 20, level=6)
    plan, (phi, acc) = run_flag(prob, dev, "redundant")
    tg = np.random.default_rng(3).choice(prob.n, 3000, replace=False)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, targets=tg)
    assert rel_l2(phi[tg], ophi) <= TOL_REAL and rel_l2(acc[tg], oacc) <= TOL_REAL


def test_symmetric_flag_refusals(dev):
    for kw in (dict(kind="helmholtz", nrhs=3, layout="redundant"), dict(kind="gravity", layout="pairtask"),
               dict(kind="gravity", layout="redundant", adjoint=True)):
        kind = kw.pop("kind")
        with pytest.raises(p2p.P2PError) as e:
            p2p.Plan(kind, 100, 2, (0, 0, 0), 1.0, symmetric=True, device=dev, **kw)
        assert e.value.status == 1
    prob = wl.grid_helmholtz(edge_points=16)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, symmetric=True, device=dev)
    with pytest.raises(p2p.P2PError) as e:
        plan.set_grid(wl.SPACING, 4)
    assert e.value.status == 5
    pos = torch.from_numpy(prob.pos).to(dev)
    q = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(pos)
    with pytest.raises(p2p.P2PError) as e:
        plan.helmholtz_adjoint(prob.k, pos, q)
    assert e.value.status == 5

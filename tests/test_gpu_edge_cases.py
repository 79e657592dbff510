"""Degenerate and extreme inputs on the GPU against the FP64 oracle:
coincident particles (softened gravity), every particle in one box,
particles on the faces of the boxing domain, and the largest plan size."""
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


def gravity(prob, dev, layout="redundant", symmetric=False, gather=True):
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, symmetric=symmetric,
                    gather_map=gather, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    phi, acc = plan.gravity(prob.eps)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy(), acc.cpu().numpy()


@pytest.mark.parametrize("layout,symmetric", [("redundant", False), ("indirect", False), ("redundant", True),
                                              ("pairtask", False), ("symmetric", False)])
def test_coincident_particles_softened(dev, layout, symmetric):
    # every particle has a twin at the same position: distinct particles at r = 0 interact through eps
    rng = np.random.default_rng(21)
    base = rng.random((3000, 3), dtype=np.float32)
    pos = np.concatenate([base, base]).astype(np.float32)
    mass = rng.uniform(0.5, 1.5, 6000).astype(np.float32)
    prob = wl.Problem("twins", pos, mass, 3, (0.0, 0.0, 0.0), 1.0, "gravity", eps=float(np.float32(1e-3)))
    _, phi, acc = gravity(prob, dev, layout, symmetric)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL


@pytest.mark.parametrize("layout", ["redundant", "indirect", "pairtask"])
def test_all_particles_in_one_box(dev, layout):
    rng = np.random.default_rng(22)
    pos = (0.5 + 0.01 * rng.random((5000, 3), dtype=np.float32)).astype(np.float32)
    mass = rng.uniform(0.5, 1.5, 5000).astype(np.float32)
    prob = wl.Problem("one_box", pos, mass, 4, (0.0, 0.0, 0.0), 1.0, "gravity", eps=float(np.float32(1e-4)))
    plan, phi, acc = gravity(prob, dev, layout)
    c = plan.counters(check=True)
    assert c["n_boxes"] == 1 and c["n_nbr"] == 1 and c["pairs"] == 5000 * 4999
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL


def test_particles_on_domain_faces(dev):
    # u = (x - lo) s equal to 0 or to 2^L lands in the first or the last cell
    rng = np.random.default_rng(23)
    pos = rng.random((4000, 3), dtype=np.float32)
    pos[:100, 0] = 1.0
    pos[100:200, 1] = 0.0
    pos[200:300] = 1.0
    mass = rng.uniform(0.5, 1.5, 4000).astype(np.float32)
    prob = wl.Problem("faces", pos, mass, 3, (0.0, 0.0, 0.0), 1.0, "gravity", eps=float(np.float32(1e-3)))
    plan, phi, acc = gravity(prob, dev)
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    np.testing.assert_array_equal(plan.array("perm", prob.n).cpu().numpy(), t["perm"])
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL


def test_helmholtz_single_particle_per_box(dev):
    # level 4 with 4096 lattice points: one particle per box, every pair crosses boxes
    e = 16
    pos = wl.grid_points(e, h=1.0 / e)
    q = wl.complex_normal((1, pos.shape[0]), np.random.default_rng(24))
    prob = wl.Problem("one_per_box", pos, q, 4, (0.0, 0.0, 0.0), 1.0, "helmholtz", k=float(np.float32(20.0)))
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, device=dev)
    pt = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pt)
    plan.restructure(pt, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k).cpu().numpy()
    assert plan.counters(check=True)["n_boxes"] == 4096
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_largest_plan(dev):
    # P2P_MAX_N = 2^26 particles, level 8 (16.8 M cells, ~4 per box); sampled against the oracle
    n = 1 << 26
    rng = np.random.default_rng(25)
    pos = rng.random((n, 3), dtype=np.float32)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    prob = wl.Problem("max", pos, mass, 8, (0.0, 0.0, 0.0), 1.0, "gravity", eps=float(np.float32(1e-4)))
    plan, phi, acc = gravity(prob, dev, gather=False)
    c = plan.counters(check=True)
    bs = plan.array("box_start", c["n_boxes"] + 1).cpu().numpy()
    assert bs[0] == 0 and bs[-1] == n and np.all(np.diff(bs) > 0)
    tg = rng.choice(n, 2000, replace=False)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, targets=tg)
    assert rel_l2(phi[tg], ophi) <= TOL_REAL and rel_l2(acc[tg], oacc) <= TOL_REAL
    with pytest.raises(p2p.P2PError) as e:
        p2p.Plan("gravity", n + 1, 8, (0, 0, 0), 1.0, device=dev)
    assert e.value.status == 1

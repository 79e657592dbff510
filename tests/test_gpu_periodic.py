"""Periodic (toroidal) neighbourhoods on the GPU against the FP64 oracle.

A periodic plan wraps the E2 neighbour cells around the domain (levels >= 2,
where the 3 x 3 x 3 block of wrapped cells never repeats a box) and tags each
neighbour entry with its image code (ox+1) + 3(oy+1) + 9(oz+1).  The
redundant layout bakes the image shift x_j + o edge into the gathered
records; the indirect layout moves the targets by -o edge per neighbour range.
Structures must be bit-exact, sums within the usual relative-L2 tolerances.
"""
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


def shifted_box(n, level, lo, edge, seed):
    """Uniform points in [lo, lo + edge)^3 (float32, strictly inside)."""
    rng = np.random.default_rng(seed)
    lo32 = np.asarray(lo, np.float32)
    e32 = np.float32(edge)
    pos = (rng.random((n, 3), dtype=np.float32) * e32 + lo32).astype(np.float32)
    hi = np.nextafter(lo32 + e32, np.float32(-np.inf)).astype(np.float32)
    pos = np.minimum(np.maximum(pos, lo32), hi).astype(np.float32)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return wl.Problem("periodic_box", pos, mass, level, tuple(float(v) for v in lo32), float(e32), "gravity",
                      eps=float(np.float32(1e-3)))


GRAV_CASES = {
    "uniform_8192_L3": lambda: wl.uniform_gravity(),
    "uniform_20000_L4": lambda: wl.uniform_gravity(n=20000, level=4, seed=3),
    "uniform_3_L2": lambda: wl.uniform_gravity(n=3, level=2, seed=4),
    "shifted_12000_L3": lambda: shifted_box(12000, 3, (-1.0, 0.25, -3.5), 2.5, 5),
    "plummer_60000_L6": lambda: wl.plummer_gravity(n=60000, level=6, eps=1e-3, seed=1),
}

HELM_CASES = {
    "grid16_r1": lambda: wl.grid_helmholtz(edge_points=16, nrhs=1),
    "grid24_r2": lambda: wl.grid_helmholtz(edge_points=24, nrhs=2, seed=1),
    "grid16_r8": lambda: wl.grid_helmholtz(edge_points=16, nrhs=8, seed=2),
}


def grav_plan(prob, dev, layout, tpl=None, tile=64, group=4, gather=True):
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, gather_map=gather,
                    periodic=True, device=dev)
    if tpl:
        plan.set_tuning(tpl, tile, 0, group)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    phi, acc = plan.gravity(prob.eps)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy(), acc.cpu().numpy()


def helm_plan(prob, dev, layout, tpl=None, tile=64, group=4):
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    gather_map=True, periodic=True, device=dev)
    if tpl:
        plan.set_tuning(tpl, tile, 0, group)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k)
    torch.cuda.synchronize()
    return plan, u.cpu().numpy()


def check_structures(plan, prob, layout):
    ref = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge, periodic=True)
    c = plan.counters(check=True)
    B, E = ref["n_boxes"], ref["n_nbr"]
    assert c["n_boxes"] == B and c["n_nbr"] == E
    np.testing.assert_array_equal(plan.array("perm", prob.n).cpu().numpy(), ref["perm"])
    np.testing.assert_array_equal(plan.array("box_start", B + 1).cpu().numpy(), ref["box_start"])
    np.testing.assert_array_equal(plan.array("nbr_start", B + 1).cpu().numpy(), ref["nbr_start"])
    np.testing.assert_array_equal(plan.array("nbr_idx", E).cpu().numpy(), ref["nbr_idx"])
    np.testing.assert_array_equal(plan.array("nbr_img", E).cpu().numpy(), ref["nbr_img"])
    if layout == "redundant":
        r = oracle.redundant(ref)
        assert c["total_src"] == r["total"]
        np.testing.assert_array_equal(plan.array("red_start", B + 1).cpu().numpy(), r["red_start"])
        np.testing.assert_array_equal(plan.array("red_self", B).cpu().numpy(), r["red_self"])
        np.testing.assert_array_equal(plan.array("gather_idx", r["total"]).cpu().numpy().view(np.uint32),
                                      r["gather_idx"])


@pytest.mark.parametrize("layout,symmetric", [("redundant", False), ("indirect", False), ("indirect", True)])
def test_periodic_grid_helmholtz_64_full(dev, layout, symmetric):
    """The bench's --periodic Helmholtz workload at full size (452,722,688 pairs
    through 27 images) against the FP64 periodic oracle, one-sided and symmetric."""
    prob = wl.grid_helmholtz()
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, layout=layout, periodic=True,
                    symmetric=symmetric, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k).cpu().numpy()
    ou, pairs = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k, periodic=True)
    assert plan.counters(check=True)["pairs"] == pairs == 452_722_688
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_periodic_structures_bit_exact_full_size(dev):
    """The 4.2 M-point Plummer sphere with toroidal boundaries (the bench's
    --periodic gravity workload): wrapped neighbour lists, image codes,
    redundant bounds and gather map equal the oracle's, bit for bit."""
    prob = wl.plummer_gravity()
    plan, _, _ = grav_plan(prob, dev, "redundant")
    check_structures(plan, prob, "redundant")


@pytest.mark.parametrize("name", sorted(GRAV_CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_periodic_structures_bit_exact(dev, name, layout):
    prob = GRAV_CASES[name]()
    plan, _, _ = grav_plan(prob, dev, layout)
    check_structures(plan, prob, layout)


@pytest.mark.parametrize("name", sorted(GRAV_CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("tpl,tile,group", [(1, 32, 1), (2, 64, 2), (4, 64, 4)])
def test_periodic_gravity_parity(dev, name, layout, tpl, tile, group):
    prob = GRAV_CASES[name]()
    plan, phi, acc = grav_plan(prob, dev, layout, tpl, tile, group)
    ophi, oacc, pairs = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps,
                                       periodic=True)
    assert plan.counters(check=True)["pairs"] == pairs
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
    if prob.n > 1:
        assert rel_l2(phi, ophi) <= TOL_REAL
        assert rel_l2(acc, oacc) <= TOL_REAL


@pytest.mark.parametrize("name", sorted(HELM_CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("tpl,tile,group", [(1, 32, 1), (2, 64, 4), (4, 64, 4)])
def test_periodic_helmholtz_parity(dev, name, layout, tpl, tile, group):
    prob = HELM_CASES[name]()
    plan, u = helm_plan(prob, dev, layout, tpl, tile, group)
    ou, pairs = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k, periodic=True)
    assert plan.counters(check=True)["pairs"] == pairs
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_periodic_lattice_every_box_sees_27(dev):
    # a 16^3 lattice filling its 4^3-box domain: every box has 27 wrapped neighbours
    prob = wl.grid_helmholtz(edge_points=16)
    plan, _ = helm_plan(prob, dev, "redundant")
    c = plan.counters(check=True)
    assert c["n_boxes"] == 64 and c["n_nbr"] == 64 * 27
    assert c["pairs"] == prob.n * (27 * 64 - 1)


def test_periodic_interior_matches_open(dev):
    # targets whose 27-box neighbourhood does not touch the boundary see the same
    # sources in the same order in both modes: identical results
    prob = wl.uniform_gravity(n=40000, level=4, seed=8)
    _, phi_p, acc_p = grav_plan(prob, dev, "redundant")
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout="redundant", device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    phi_o, acc_o = (t.cpu().numpy() for t in plan.gravity(prob.eps))
    cell, _ = oracle.cells(prob.pos, prob.level, prob.lo, prob.edge)
    side = 1 << prob.level
    inner = np.all((cell >= 1) & (cell <= side - 2), axis=1)
    assert inner.sum() > 1000
    np.testing.assert_array_equal(phi_p[inner], phi_o[inner])
    np.testing.assert_array_equal(acc_p[inner], acc_o[inner])
    assert not np.array_equal(phi_p[~inner], phi_o[~inner])


def test_periodic_translation_by_a_box(dev):
    # moving every particle by one box edge (wrapping) relabels boxes only
    prob = wl.uniform_gravity(n=20000, level=3, seed=9)
    _, phi, acc = grav_plan(prob, dev, "indirect")
    moved = prob.pos.copy()
    moved[:, 0] = (moved[:, 0] + np.float32(0.125)).astype(np.float32)
    moved[:, 0] = np.where(moved[:, 0] >= 1.0, moved[:, 0] - np.float32(1.0), moved[:, 0]).astype(np.float32)
    prob2 = wl.Problem("moved", moved, prob.strength, prob.level, prob.lo, prob.edge, "gravity", eps=prob.eps)
    _, phi2, acc2 = grav_plan(prob2, dev, "redundant")
    # the wrapped coordinates are rounded, so compare to rounding, not bitwise
    assert rel_l2(phi2, phi) <= TOL_REAL and rel_l2(acc2, acc) <= TOL_REAL


def test_periodic_momentum(dev):
    prob = wl.uniform_gravity(n=30000, level=4, seed=10)
    _, _, acc = grav_plan(prob, dev, "redundant")
    f = acc.astype(np.float64) * prob.strength.astype(np.float64)[:, None]
    assert np.abs(f.sum(axis=0)).max() <= 1e-6 * np.abs(f).sum()


def test_periodic_grid_64_sampled(dev):
    prob = wl.grid_helmholtz(edge_points=64, seed=3)
    for layout in ("indirect", "redundant"):
        plan, u = helm_plan(prob, dev, layout)
        assert plan.counters(check=True)["pairs"] == prob.n * (27 * 64 - 1)
        tg = np.random.default_rng(2).choice(prob.n, 3000, replace=False)
        tg = np.unique(np.concatenate([tg, np.arange(64)]))       # a corner row touches every wrap
        ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k, targets=tg,
                                 periodic=True)
        assert rel_l2(u[:, tg], ou) <= TOL_COMPLEX


def test_periodic_helmholtz_adjoint_q(dev):
    # grad_q = P^H gbar; with P symmetric under the wrapped neighbourhood,
    # <P q, g> = <q, P^H g> checks the adjoint without an oracle of its own
    prob = wl.grid_helmholtz(edge_points=16, nrhs=2, seed=4)
    for layout in ("indirect", "redundant"):
        plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=2, layout=layout,
                        periodic=True, device=dev)
        pos = torch.from_numpy(prob.pos).to(dev)
        q = torch.from_numpy(prob.strength).to(dev)
        g = torch.from_numpy(wl.complex_normal((2, prob.n), np.random.default_rng(5))).to(dev)
        plan.tree_build(pos)
        plan.restructure(pos, q)
        u = plan.helmholtz(prob.k)
        gq, _ = plan.helmholtz_adjoint(prob.k, pos, g)
        lhs = torch.sum(torch.conj(g.to(torch.complex128)) * u.to(torch.complex128)).item()
        rhs = torch.sum(torch.conj(gq.to(torch.complex128)) * q.to(torch.complex128)).item()
        assert abs(lhs - rhs) <= 2e-5 * abs(lhs)
        ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k, periodic=True)
        assert rel_l2(u.cpu().numpy(), ou) <= TOL_COMPLEX


def test_periodic_refusals(dev):
    with pytest.raises(p2p.P2PError) as e:
        p2p.Plan("gravity", 100, 1, (0, 0, 0), 1.0, periodic=True, device=dev)
    assert e.value.status == 1                                          # P2P_ERR_INVALID_ARG
    prob = wl.grid_helmholtz(edge_points=16)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, periodic=True, device=dev)
    with pytest.raises(p2p.P2PError) as e:
        plan.set_grid(wl.SPACING, 4)
    assert e.value.status == 5                                          # P2P_ERR_UNSUPPORTED
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge, periodic=True)
    with pytest.raises(p2p.P2PError) as e:
        plan.tree_import(*(torch.from_numpy(t[k]).to(dev) for k in ("perm", "box_start", "nbr_start", "nbr_idx")))
    assert e.value.status == 5

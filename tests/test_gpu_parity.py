"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Structures (permutation, box bounds, neighbour lists, redundant stream
bounds, gather map) must be bit-exact; sums must meet the relative-L2
tolerances: 1e-5 for float32 real outputs (phi and acc separately), 2e-5
for complex64 outputs, against the FP64 oracle on the same inputs.
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


def run_gravity(prob, dev, layout, tpl=None, tile=None, plain=False, gather=True, group=4):
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, gather_map=gather,
                    plain_fp32=plain, device=dev)
    if tpl:
        plan.set_tuning(tpl, tile or 64, 0, group)
    pos = torch.from_numpy(prob.pos).to(dev)
    m = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, m)
    phi, acc = plan.gravity(prob.eps)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy(), acc.cpu().numpy()


def run_helmholtz(prob, dev, layout, tpl=None, tile=None, plain=False, group=4):
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    gather_map=True, plain_fp32=plain, device=dev)
    if tpl:
        plan.set_tuning(tpl, tile or 64, 0, group)
    pos = torch.from_numpy(prob.pos).to(dev)
    q = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, q)
    u = plan.helmholtz(prob.k)
    torch.cuda.synchronize()
    return plan, u.cpu().numpy()


def check_structures(plan, prob, layout):
    ref = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    c = plan.counters(check=True)
    B, E = ref["n_boxes"], ref["n_nbr"]
    assert c["n_boxes"] == B
    assert c["n_nbr"] == E
    np.testing.assert_array_equal(plan.array("perm", prob.n).cpu().numpy(), ref["perm"])
    np.testing.assert_array_equal(plan.array("box_key", B).cpu().numpy().view(np.uint32), ref["box_key"])
    np.testing.assert_array_equal(plan.array("box_start", B + 1).cpu().numpy(), ref["box_start"])
    np.testing.assert_array_equal(plan.array("nbr_start", B + 1).cpu().numpy(), ref["nbr_start"])
    np.testing.assert_array_equal(plan.array("nbr_idx", E).cpu().numpy(), ref["nbr_idx"])
    _, key = oracle.cells(prob.pos, prob.level, prob.lo, prob.edge)
    np.testing.assert_array_equal(plan.array("sorted_key", prob.n).cpu().numpy().view(np.uint32),
                                  key[ref["perm"]])
    assert c["pairs"] == oracle.pair_count(prob.pos, prob.level, prob.lo, prob.edge)
    if layout == "redundant":
        r = oracle.redundant(ref)
        assert c["total_src"] == r["total"]
        np.testing.assert_array_equal(plan.array("red_start", B + 1).cpu().numpy(), r["red_start"])
        np.testing.assert_array_equal(plan.array("red_self", B).cpu().numpy(), r["red_self"])
        np.testing.assert_array_equal(plan.array("gather_idx", r["total"]).cpu().numpy().view(np.uint32),
                                      r["gather_idx"])


# ---------------------------------------------------------------------------
# structures
# ---------------------------------------------------------------------------

STRUCT_CASES = {
    "uniform_8192_L3": lambda: wl.uniform_gravity(),
    "uniform_1_L2": lambda: wl.uniform_gravity(n=1, level=2),
    "uniform_37_L1": lambda: wl.uniform_gravity(n=37, level=1),
    "uniform_50000_L9_bsearch": lambda: wl.uniform_gravity(n=50000, level=9),
    "plummer_60000_L6": lambda: wl.plummer_gravity(n=60000, level=6, eps=1e-3),
    "grid_24": lambda: wl.grid_helmholtz(edge_points=24),
    "grid_16": lambda: wl.grid_helmholtz(edge_points=16),
    # sort-tile edges (2,048 keys a tile) and every digit width: level 8 = three
    # passes of 8 bits (256 digits), level 5 = two of 8, level 4 = two of 6
    "uniform_2048_L8": lambda: wl.uniform_gravity(n=2048, level=8, seed=5),
    "uniform_2049_L5": lambda: wl.uniform_gravity(n=2049, level=5, seed=6),
    "plummer_4097_L4": lambda: wl.plummer_gravity(n=4097, level=4, eps=1e-3, seed=7),
    "plummer_6143_L8": lambda: wl.plummer_gravity(n=6143, level=8, eps=1e-3, seed=8),
}


@pytest.mark.parametrize("name", sorted(STRUCT_CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_structures_bit_exact(dev, name, layout):
    prob = STRUCT_CASES[name]()
    if prob.kind == "gravity":
        plan, _, _ = run_gravity(prob, dev, layout)
    else:
        plan, _ = run_helmholtz(prob, dev, layout)
    check_structures(plan, prob, layout)


def test_sort_many_radix_passes(dev):
    # level 10 = 30-bit keys, 4 passes; heavy ties
    rng = np.random.default_rng(9)
    pos = (rng.integers(0, 64, (200000, 3)) / 64.0 + 1e-4).astype(np.float32)
    prob = wl.Problem("ties", pos, np.ones(200000, np.float32), 10, (0.0, 0.0, 0.0), 1.0, "gravity", eps=1e-3)
    plan = p2p.Plan("gravity", prob.n, 10, prob.lo, prob.edge, layout="indirect", device=dev)
    plan.tree_build(torch.from_numpy(pos).to(dev))
    ref = oracle.tree(pos, 10, prob.lo, prob.edge)
    np.testing.assert_array_equal(plan.array("perm", prob.n).cpu().numpy(), ref["perm"])
    assert plan.counters(check=True)["n_boxes"] == ref["n_boxes"]


def test_domain_error_is_reported(dev):
    prob = wl.uniform_gravity(n=1000, level=3)
    pos = prob.pos.copy()
    pos[17, 1] = 1.5
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, device=dev)
    plan.tree_build(torch.from_numpy(pos).to(dev))
    c = plan.counters()
    assert c["flags"] & p2p.FLAG_DOMAIN
    assert c["status"] == 6
    # the next build of valid positions clears the flag
    plan.tree_build(torch.from_numpy(prob.pos).to(dev))
    assert plan.counters(check=True)["flags"] == 0


def test_operator_before_tree_is_a_state_error(dev):
    plan = p2p.Plan("gravity", 100, 2, (0, 0, 0), 1.0, device=dev)
    with pytest.raises(p2p.P2PError) as e:
        plan.gravity(1e-3)
    assert e.value.status == 8


# ---------------------------------------------------------------------------
# gravity sums
# ---------------------------------------------------------------------------

GRAV_CASES = {
    "uniform_8192_L3": lambda: wl.uniform_gravity(),
    "uniform_20000_L4": lambda: wl.uniform_gravity(n=20000, level=4, seed=3),
    "plummer_60000_L6": lambda: wl.plummer_gravity(n=60000, level=6, eps=1e-3, seed=1),
    "uniform_5_L1": lambda: wl.uniform_gravity(n=5, level=1),
}


@pytest.mark.parametrize("name", sorted(GRAV_CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("tpl,tile,group", [(1, 32, 1), (2, 64, 2), (4, 64, 4), (2, 32, 4)])
def test_gravity_parity(dev, name, layout, tpl, tile, group):
    prob = GRAV_CASES[name]()
    _, phi, acc = run_gravity(prob, dev, layout, tpl, tile, group=group)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
    assert rel_l2(phi, ophi) <= TOL_REAL
    assert rel_l2(acc, oacc) <= TOL_REAL


def test_gravity_layouts_agree_bitwise(dev):
    # both layouts visit sources in the same order with the same tile cuts
    # only when ranges align; they must at least agree to rounding
    prob = wl.plummer_gravity(n=40000, level=5, eps=1e-3, seed=2)
    _, p1, a1 = run_gravity(prob, dev, "indirect")
    _, p2, a2 = run_gravity(prob, dev, "redundant")
    assert rel_l2(p1, p2) < 1e-6 and rel_l2(a1, a2) < 1e-6


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_gravity_packed_kernels_agree(dev, layout):
    """Two and four targets per lane run the packed two-wide kernel: targets of
    items of more than 32 targets sum their sources in the same order (bitwise
    equal between the two); an item of at most 32 targets with two per lane runs
    source-split (even and odd sources in the two halves, added at the end), and
    one per lane is the scalar kernel: equal to rounding."""
    prob = wl.plummer_gravity(n=40000, level=5, eps=1e-3, seed=2)
    plan, p1, a1 = run_gravity(prob, dev, layout, 1, 64, group=4)
    _, p2, a2 = run_gravity(prob, dev, layout, 2, 64, group=4)
    _, p4, a4 = run_gravity(prob, dev, layout, 4, 64, group=4)
    assert rel_l2(p1, p2) < 1e-6 and rel_l2(a1, a2) < 1e-6
    assert rel_l2(p4, p2) < 1e-6 and rel_l2(a4, a2) < 1e-6
    # targets in whole 64-target items of two per lane are summed as with four per lane
    bs = plan.array("box_start", plan.counters()["n_boxes"] + 1).cpu().numpy()
    perm = plan.array("perm", prob.n).cpu().numpy()
    occ = np.diff(bs)
    full = np.concatenate([perm[bs[b]:bs[b] + (occ[b] // 128) * 128] for b in range(len(occ)) if occ[b] >= 128])
    assert full.size > 1000
    np.testing.assert_array_equal(p2[full], p4[full])
    np.testing.assert_array_equal(a2[full], a4[full])


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("n,level", [(3000, 3), (24000, 3), (20000, 2)])
def test_gravity_source_split_items(dev, layout, n, level):
    """Boxes of at most 32 particles (every item source-split), of 33-64 (packed
    targets), and larger boxes whose last item holds <= 32 targets; odd and even
    tile counts; against the FP64 oracle."""
    prob = wl.uniform_gravity(n=n, level=level, seed=n)
    for tile in (64, 128):
        _, phi, acc = run_gravity(prob, dev, layout, 2, tile, group=1)
        ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
        assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL


def test_gravity_deterministic(dev):
    prob = wl.plummer_gravity(n=40000, level=5, eps=1e-3, seed=4)
    _, p1, a1 = run_gravity(prob, dev, "redundant")
    _, p2, a2 = run_gravity(prob, dev, "redundant")
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(a1, a2)


def test_gravity_momentum_invariant(dev):
    prob = wl.plummer_gravity(n=60000, level=6, eps=1e-3, seed=5)
    _, _, acc = run_gravity(prob, dev, "redundant")
    f = torch.from_numpy(acc).to(dev, torch.float64) * torch.from_numpy(prob.strength).to(dev, torch.float64)[:, None]
    tot = f.sum(dim=0).abs().max().item()
    assert tot <= 1e-6 * f.abs().sum().item()


def test_compensated_beats_plain(dev):
    prob = wl.plummer_gravity(n=60000, level=5, eps=1e-3, seed=6)
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    _, pc, ac = run_gravity(prob, dev, "redundant")
    _, pp, ap = run_gravity(prob, dev, "redundant", plain=True)
    ec, ep = rel_l2(pc, ophi), rel_l2(pp, ophi)
    assert ec <= TOL_REAL and ep <= 1e-4
    assert ec <= ep


# ---------------------------------------------------------------------------
# Helmholtz sums
# ---------------------------------------------------------------------------

def random_helmholtz(n, level, nrhs, seed, k=2 * math.pi):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3), dtype=np.float32)
    q = wl.complex_normal((nrhs, n), rng)
    return wl.Problem("random_helm", pos, q, level, (0.0, 0.0, 0.0), 1.0, "helmholtz", k=float(np.float32(k)))


HELM_CASES = {
    "grid16_r1": lambda: wl.grid_helmholtz(edge_points=16, nrhs=1),
    "grid24_r2": lambda: wl.grid_helmholtz(edge_points=24, nrhs=2, seed=1),
    "grid16_r8": lambda: wl.grid_helmholtz(edge_points=16, nrhs=8, seed=2),
    "random_r3": lambda: random_helmholtz(20000, 4, 3, 7),
    "random_r5": lambda: random_helmholtz(3000, 3, 5, 8, k=20.0),
    "random_r16": lambda: random_helmholtz(2000, 2, 16, 9),
}


@pytest.mark.parametrize("name", sorted(HELM_CASES))
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("tpl,tile,group", [(1, 32, 1), (2, 64, 2), (2, 64, 4), (1, 64, 4), (4, 64, 4), (4, 32, 1),
                                            (4, 64, 2), (4, 48, 4), (2, 48, 2)])
def test_helmholtz_parity(dev, name, layout, tpl, tile, group):
    prob = HELM_CASES[name]()
    _, u = run_helmholtz(prob, dev, layout, tpl, tile, group=group)
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert np.all(np.isfinite(u))
    assert rel_l2(u, ou) <= TOL_COMPLEX


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_multi_rhs_equals_single_rhs_bitwise(dev, plain, layout):
    """Several right-hand sides per pass accumulate each RHS with packed
    (real, imaginary) FMAs in the scalar order: every RHS of an 8-RHS plan equals,
    bit for bit, a one-RHS plan on that RHS with the same tuning (32-record tiles:
    the tile wide 8-RHS records get, so the compensated sums fold at the same points)."""
    prob = wl.grid_helmholtz(edge_points=24, nrhs=8, seed=4)
    _, u8 = run_helmholtz(prob, dev, layout, 2, 32, plain=plain, group=4)
    for r in (0, 3, 7):
        one = wl.Problem(prob.name, prob.pos, prob.strength[r:r + 1].copy(), prob.level, prob.lo, prob.edge,
                         "helmholtz", k=prob.k)
        _, u1 = run_helmholtz(one, dev, layout, 2, 32, plain=plain, group=4)
        np.testing.assert_array_equal(u8[r], u1[0])


@pytest.mark.parametrize("group", [1, 4])
def test_helmholtz_plain_fp32(dev, group):
    prob = wl.grid_helmholtz(edge_points=24, nrhs=3, seed=6)
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    _, uc = run_helmholtz(prob, dev, "redundant", 2, 64, group=group)
    _, up = run_helmholtz(prob, dev, "redundant", 2, 64, plain=True, group=group)
    assert rel_l2(uc, ou) <= TOL_COMPLEX and rel_l2(up, ou) <= 1e-4


@pytest.mark.parametrize("tpl,group", [(1, 1), (2, 4), (2, 2)])
def test_helmholtz_precise_phase_path(dev, tpl, group):
    # boxes of edge 1/4 with k = 60: k * rmax ~ 52 > 32 selects the accurate sine/cosine
    prob = random_helmholtz(4000, 2, 1, 11, k=60.0)
    _, u = run_helmholtz(prob, dev, "redundant", tpl, 64, group=group)
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert rel_l2(u, ou) <= TOL_COMPLEX


def test_helmholtz_reciprocity_gpu(dev):
    prob = wl.grid_helmholtz(edge_points=24, nrhs=2, seed=3)
    _, u = run_helmholtz(prob, dev, "redundant")
    a, b = prob.strength[0].astype(np.complex128), prob.strength[1].astype(np.complex128)
    lhs = np.sum(b * u[0].astype(np.complex128))
    rhs = np.sum(a * u[1].astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# ---------------------------------------------------------------------------
# full-size workloads (sampled where the oracle cannot do everything)
# ---------------------------------------------------------------------------

def test_uniform_gravity_full(dev):
    prob = wl.uniform_gravity()
    for layout in ("indirect", "redundant"):
        plan, phi, acc = run_gravity(prob, dev, layout)
        ophi, oacc, pairs = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
        assert plan.counters(check=True)["pairs"] == pairs == 2732724
        assert rel_l2(phi, ophi) <= TOL_REAL and rel_l2(acc, oacc) <= TOL_REAL


def test_grid_helmholtz_64_full(dev):
    prob = wl.grid_helmholtz()
    ou, pairs = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    assert pairs == 398426112
    for layout in ("indirect", "redundant"):
        plan, u = run_helmholtz(prob, dev, layout)
        assert plan.counters(check=True)["pairs"] == pairs
        assert rel_l2(u, ou) <= TOL_COMPLEX


def _sample_targets(prob, plan, count, seed):
    """Random targets plus every target of the most occupied box."""
    rng = np.random.default_rng(seed)
    bs = plan.array("box_start", plan.counters()["n_boxes"] + 1).cpu().numpy()
    occ = np.diff(bs)
    b = int(np.argmax(occ))
    perm = plan.array("perm", prob.n).cpu().numpy()
    heavy = perm[bs[b]:bs[b + 1]]
    return np.unique(np.concatenate([rng.choice(prob.n, count, replace=False), heavy]))


@pytest.mark.parametrize("name", ["grid_helmholtz_64", "grid_helmholtz_128", "plummer_gravity_4m"])
def test_structures_bit_exact_full_size(dev, name):
    """The bench workloads at full size: keys, permutation, boxes, neighbour lists,
    redundant stream bounds, self offsets, gather map and pair count equal the
    oracle's, bit for bit (up to 4,194,304 particles, 605,596 boxes, 102 M stream records)."""
    prob = {"grid_helmholtz_64": wl.grid_helmholtz, "grid_helmholtz_128": lambda: wl.grid_helmholtz(edge_points=128),
            "plummer_gravity_4m": wl.plummer_gravity}[name]()
    if prob.kind == "gravity":
        plan, _, _ = run_gravity(prob, dev, "redundant", gather=True)
    else:
        plan, _ = run_helmholtz(prob, dev, "redundant")
    check_structures(plan, prob, "redundant")


def test_plummer_gravity_full_sampled(dev):
    prob = wl.plummer_gravity()
    for layout in ("indirect", "redundant"):
        plan, phi, acc = run_gravity(prob, dev, layout, gather=False)
        tg = _sample_targets(prob, plan, 3000, 0)
        ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, targets=tg)
        assert rel_l2(phi[tg], ophi) <= TOL_REAL
        assert rel_l2(acc[tg], oacc) <= TOL_REAL
        c = plan.counters(check=True)
        assert c["n_boxes"] == oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)["n_boxes"]


def test_grid_helmholtz_128_sampled(dev):
    prob = wl.grid_helmholtz(edge_points=128, seed=5)
    plan, u = run_helmholtz(prob, dev, "redundant")
    assert plan.counters(check=True)["pairs"] == 3399974912
    tg = np.random.default_rng(1).choice(prob.n, 4000, replace=False)
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k, targets=tg)
    assert rel_l2(u[:, tg], ou) <= TOL_COMPLEX

"""Error of the FP32 kernels against the FP64 oracle, compensated (Kahan
per tile) vs plain accumulation, on the benchmark workloads (sampled where
the oracle cannot do everything).  Prints one line per case."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("plain", [False, True])
def test_accuracy_grid_helmholtz_64(dev, plain):
    prob = wl.grid_helmholtz()
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, plain_fp32=plain, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k).cpu().numpy()
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    e, m = rel_l2(u, ou), max_rel(u, ou)
    print(f"\nACCURACY grid_helmholtz_64 {'plain' if plain else 'compensated'}: rel-L2 {e:.3e}, max-rel {m:.3e}")
    assert e <= (2e-5 if not plain else 1e-4)


@pytest.mark.parametrize("plain", [False, True])
def test_accuracy_plummer_gravity(dev, plain):
    prob = wl.plummer_gravity()
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, plain_fp32=plain, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    phi, acc = plan.gravity(prob.eps)
    phi, acc = phi.cpu().numpy(), acc.cpu().numpy()
    rng = np.random.default_rng(0)
    bs = plan.array("box_start", plan.counters()["n_boxes"] + 1).cpu().numpy()
    b = int(np.argmax(np.diff(bs)))
    heavy = plan.array("perm", prob.n).cpu().numpy()[bs[b]:bs[b + 1]]
    tg = np.unique(np.concatenate([rng.choice(prob.n, 3000, replace=False), heavy]))
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps, targets=tg)
    ep, ea = rel_l2(phi[tg], ophi), rel_l2(acc[tg], oacc)
    print(f"\nACCURACY plummer_gravity {'plain' if plain else 'compensated'} ({len(tg)} targets incl. the "
          f"heaviest box): phi rel-L2 {ep:.3e}, acc rel-L2 {ea:.3e}")
    assert ep <= (1e-5 if not plain else 1e-4) and ea <= (1e-5 if not plain else 1e-4)


@pytest.mark.parametrize("mode", ["symmetric", "pattern", "indirect", "pairtask", "four_per_lane",
                                  "symmetric_pairtask"])
def test_accuracy_grid_helmholtz_64_variants(dev, mode):
    prob = wl.grid_helmholtz()
    kw = {"indirect": dict(layout="indirect"), "pairtask": dict(layout="pairtask"),
          "symmetric_pairtask": dict(layout="symmetric")}.get(mode, {})
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, symmetric=(mode == "symmetric"),
                    device=dev, **kw)
    if mode == "four_per_lane":
        plan.set_tuning(4, 64, 0, 4)
    if mode == "pattern":
        plan.set_grid(wl.SPACING, wl.LEAF_EDGE_POINTS)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k).cpu().numpy()
    ou, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k)
    e, m = rel_l2(u, ou), max_rel(u, ou)
    print(f"\nACCURACY grid_helmholtz_64 {mode}: rel-L2 {e:.3e}, max-rel {m:.3e}")
    assert e <= 2e-5


def test_accuracy_batched_forward_adjoint(dev):
    """64 uneven grid instances x 8 RHS in one launch: u = P q and g = conj(P) y, against the
    FP64 oracle on four instances (the smallest, two middle ones, the largest)."""
    probs = wl.batched_helmholtz()
    nrhs, k = probs[0].nrhs, probs[0].k
    batch = p2p.Batch([(p.n, p.level, p.lo, p.edge) for p in probs], nrhs, k, pair=True, device=dev)
    pos = torch.from_numpy(np.concatenate([p.pos for p in probs])).to(dev)
    q = torch.from_numpy(np.concatenate([p.strength for p in probs], axis=1)).to(dev)
    y = torch.from_numpy(wl.complex_normal((nrhs, batch.N), np.random.default_rng(123))).to(dev)
    batch.build(pos)
    u, g = batch.run(pos, q, y)
    u, g = u.cpu().numpy(), g.cpu().numpy()
    yn = y.cpu().numpy()
    order = np.argsort([p.n for p in probs])
    eu, eg = [], []
    for i in (order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]):
        p = probs[i]
        o0, o1 = batch.offsets[i], batch.offsets[i + 1]
        ou, _ = oracle.helmholtz(p.pos, p.strength, p.level, p.lo, p.edge, k)
        og, _ = oracle.helmholtz(p.pos, np.conj(yn[:, o0:o1]), p.level, p.lo, p.edge, k)
        eu.append(rel_l2(u[:, o0:o1], ou))
        eg.append(rel_l2(g[:, o0:o1], np.conj(og)))
    print(f"\nACCURACY batched forward + adjoint (4 of 64 instances, 8 RHS): u rel-L2 max {max(eu):.3e}, "
          f"g rel-L2 max {max(eg):.3e}")
    assert max(eu) <= 2e-5 and max(eg) <= 2e-5

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

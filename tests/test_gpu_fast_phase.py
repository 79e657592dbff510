"""Parity at the top of the hardware sine/cosine range.

Plans whose largest phase k * r_max (r_max = 2 sqrt(3) x box edge, the
largest distance between points of neighbouring boxes) is at most 32 take
sin/cos from the MUFU approximation; above it the accurate routine.  The
approximation's absolute error grows with the argument, so these cases put
k * r_max just below the switch (k = 73 on level-3 boxes of the unit cube:
73 x 0.4330127 = 31.6) and check every kernel that evaluates phases on the
fast path against the FP64 oracle at the complex64 tolerance: the one-sided
tile kernel (four targets per lane, 1-2 right-hand sides), the one- and
two-target kernels (1 and 8 right-hand sides), plain FP32 accumulation,
symmetric evaluation (per-box and pair-task layouts), one-sided pair tasks,
periodic neighbourhoods, the adjoint (strengths and positions) and the batch.
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
LEVEL = 3
K_FAST = float(np.float32(73.0))       # k * r_max = 31.6 on level-3 boxes of the unit cube
K_ABOVE = float(np.float32(74.0))      # k * r_max = 32.04: the accurate routine


def rmax(level: int, edge: float = 1.0) -> float:
    """r_max as the library computes it, in float32."""
    f = np.float32
    return float(f(2.0) * (f(edge) / f(1 << level)) * f(1.7320508))


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# pairs of points near opposite corners of two diagonally adjacent level-3 boxes
# (cells c and c + (1, 1, 1)): their distance is 0.9993 r_max, so every case
# evaluates phases up to k * 0.9993 r_max
FAR_CELLS = ((0, 0, 0), (3, 2, 5), (6, 6, 6), (1, 5, 2))


def far_pairs(level=LEVEL):
    h = 1.0 / (1 << level)
    d = 1e-4
    pts = []
    for c in FAR_CELLS:
        lo = np.array(c, np.float64) * h
        pts.append(lo + d)
        pts.append(lo + 2 * h - d)
    return np.array(pts, np.float32)


def problem(n, nrhs, seed, k=K_FAST, level=LEVEL):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3), dtype=np.float32)
    pos[:2 * len(FAR_CELLS)] = far_pairs(level)
    q = wl.complex_normal((nrhs, n), rng)
    return wl.Problem("fast_phase", pos, q, level, (0.0, 0.0, 0.0), 1.0, "helmholtz", k=k)


def run(prob, dev, layout="redundant", tpl=None, tile=64, group=4, plain=False, symmetric=False, periodic=False):
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    plain_fp32=plain, symmetric=symmetric, periodic=periodic, device=dev)
    if tpl:
        plan.set_tuning(tpl, tile, 0, group)
    pos = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, torch.from_numpy(prob.strength).to(dev))
    u = plan.helmholtz(prob.k)
    torch.cuda.synchronize()
    assert plan.counters()["status"] == 0
    return u.cpu().numpy()


def oracle_u(prob, periodic=False):
    u, _ = oracle.helmholtz(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.k, periodic=periodic)
    return u


def test_phase_range_is_just_below_the_switch():
    assert 31.0 < K_FAST * rmax(LEVEL) <= 32.0
    assert K_ABOVE * rmax(LEVEL) > 32.0
    # every case holds neighbouring pairs at the top of the range (boxes at Chebyshev distance 1)
    prob = problem(8000, 1, 1)
    cells, _ = oracle.cells(prob.pos, LEVEL, prob.lo, prob.edge)
    for i in range(len(FAR_CELLS)):
        a, b = 2 * i, 2 * i + 1
        assert np.abs(cells[a] - cells[b]).max() == 1
        d = np.linalg.norm(prob.pos[a].astype(np.float64) - prob.pos[b])
        assert K_FAST * d > 31.5


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("nrhs", [1, 2])
@pytest.mark.parametrize("group", [1, 2, 4])
def test_tile_kernel(dev, layout, nrhs, group):
    """Four targets per lane (k_helmtile), the default for one or two right-hand sides."""
    prob = problem(8000, nrhs, 10 + nrhs)
    u = run(prob, dev, layout, 4, 64, group)
    assert rel_l2(u, oracle_u(prob)) <= TOL_COMPLEX


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("tpl,nrhs", [(1, 1), (2, 1), (1, 8), (2, 8), (2, 4), (2, 3)])
def test_one_and_two_targets_per_lane(dev, layout, tpl, nrhs):
    """One or two targets per lane (k_helmholtz), 1 to 8 right-hand sides per pass."""
    prob = problem(6000, nrhs, 20 + nrhs)
    u = run(prob, dev, layout, tpl, 64 if nrhs <= 2 else 32, 4)
    assert rel_l2(u, oracle_u(prob)) <= TOL_COMPLEX


@pytest.mark.parametrize("group", [1, 4])
def test_plain_fp32(dev, group):
    prob = problem(6000, 2, 31)
    u = run(prob, dev, "redundant", 2, 64, group, plain=True)
    assert rel_l2(u, oracle_u(prob)) <= 1e-4


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_symmetric_per_box(dev, layout, nrhs):
    prob = problem(8000, nrhs, 40 + nrhs)
    u = run(prob, dev, layout, symmetric=True)
    assert rel_l2(u, oracle_u(prob)) <= TOL_COMPLEX


@pytest.mark.parametrize("layout", ["symmetric", "pairtask"])
def test_pair_tasks(dev, layout):
    prob = problem(8000, 1, 50)
    u = run(prob, dev, layout)
    assert rel_l2(u, oracle_u(prob)) <= TOL_COMPLEX


@pytest.mark.parametrize("symmetric", [False, True])
def test_periodic(dev, symmetric):
    prob = problem(8000, 1, 60)
    u = run(prob, dev, "redundant", symmetric=symmetric, periodic=True)
    assert rel_l2(u, oracle_u(prob, periodic=True)) <= TOL_COMPLEX


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("nrhs,tpl", [(1, 1), (1, 2), (8, 1)])
def test_adjoint(dev, layout, nrhs, tpl):
    prob = problem(6000, nrhs, 70 + nrhs)
    gbar = wl.complex_normal((nrhs, prob.n), np.random.default_rng(71))
    plan = p2p.Plan("helmholtz", prob.n, LEVEL, prob.lo, prob.edge, nrhs=nrhs, layout=layout, adjoint=True,
                    device=dev)
    plan.set_tuning(tpl, 64, 0, 4)
    tp = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(tp)
    gq, gx = plan.helmholtz_adjoint(prob.k, tp, torch.from_numpy(gbar).to(dev), torch.from_numpy(prob.strength).to(dev),
                                    want_q=True, want_pos=True)
    gq2, _ = plan.helmholtz_adjoint(prob.k, tp, torch.from_numpy(gbar).to(dev), want_q=True, want_pos=False)
    torch.cuda.synchronize()
    oq, ox = oracle.helmholtz_adjoint(prob.pos, prob.strength, gbar, LEVEL, prob.lo, prob.edge, prob.k)
    assert rel_l2(gq.cpu().numpy(), oq) <= TOL_COMPLEX
    assert rel_l2(gq2.cpu().numpy(), oq) <= TOL_COMPLEX
    assert rel_l2(gx.cpu().numpy(), ox) <= TOL_REAL


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_batch_forward_and_adjoint(dev, layout):
    nrhs = 2
    probs = [problem(n, nrhs, 80 + i) for i, n in enumerate((3000, 8000, 5000))]
    b = p2p.Batch([(p.n, p.level, p.lo, p.edge) for p in probs], nrhs, K_FAST, pair=True, layout=layout, device=dev)
    pos = torch.from_numpy(np.concatenate([p.pos for p in probs])).to(dev)
    q = torch.from_numpy(np.concatenate([p.strength for p in probs], axis=1)).to(dev)
    y = wl.complex_normal((nrhs, b.N), np.random.default_rng(89))
    b.build(pos)
    u, g = b.run(pos, q, torch.from_numpy(y).to(dev))
    torch.cuda.synchronize()
    assert b.counters()["status"] == 0
    u, g = u.cpu().numpy(), g.cpu().numpy()
    for i, p in enumerate(probs):
        o0, o1 = b.offsets[i], b.offsets[i + 1]
        assert rel_l2(u[:, o0:o1], oracle_u(p)) <= TOL_COMPLEX
        og, _ = oracle.helmholtz_adjoint(p.pos, p.strength, y[:, o0:o1], p.level, p.lo, p.edge, p.k)
        assert rel_l2(g[:, o0:o1], og) <= TOL_COMPLEX


def test_just_above_the_switch_uses_the_accurate_routine(dev):
    """k * r_max = 32.04: the accurate sine/cosine, same tolerance."""
    prob = problem(6000, 1, 90, k=K_ABOVE)
    u = run(prob, dev, "redundant", 2, 64, 4)
    assert rel_l2(u, oracle_u(prob)) <= TOL_COMPLEX

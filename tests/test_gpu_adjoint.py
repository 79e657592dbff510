"""Adjoint kernels (through the C ABI and torch.autograd) against the FP64
oracle adjoints, and the differentiable Helmholtz loss on the 128^3 grid
checked by finite differences on 16 contrast entries."""
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


def random_points(n, seed):
    return np.random.default_rng(seed).random((n, 3), dtype=np.float32)


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("nrhs,group", [(1, 4), (3, 1), (8, 4)])
def test_helmholtz_adjoint_q_and_pos(dev, layout, nrhs, group):
    n, level = 12000, 4
    pos = random_points(n, 3 + nrhs)
    rng = np.random.default_rng(7)
    q = wl.complex_normal((nrhs, n), rng)
    gbar = wl.complex_normal((nrhs, n), rng)
    k = np.float32(2 * math.pi * 2.0)
    plan = p2p.Plan("helmholtz", n, level, (0, 0, 0), 1.0, nrhs=nrhs, layout=layout, adjoint=True, device=dev)
    plan.set_tuning(1, 64, 0, group)
    tp = torch.from_numpy(pos).to(dev)
    plan.tree_build(tp)
    gq, gx = plan.helmholtz_adjoint(k, tp, torch.from_numpy(gbar).to(dev), torch.from_numpy(q).to(dev),
                                    want_q=True, want_pos=True)
    # the q-only path (forward operator with -k)
    gq2, _ = plan.helmholtz_adjoint(k, tp, torch.from_numpy(gbar).to(dev), want_q=True, want_pos=False)
    torch.cuda.synchronize()
    oq, ox = oracle.helmholtz_adjoint(pos, q, gbar, level, (0, 0, 0), 1.0, k)
    assert rel_l2(gq.cpu().numpy(), oq) <= TOL_COMPLEX
    assert rel_l2(gq2.cpu().numpy(), oq) <= TOL_COMPLEX
    assert rel_l2(gx.cpu().numpy(), ox) <= TOL_REAL


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("tpl,group", [(1, 4), (2, 1)])
def test_gravity_adjoint(dev, layout, tpl, group):
    prob = wl.plummer_gravity(n=30000, level=5, eps=1e-3, seed=8)
    rng = np.random.default_rng(9)
    gphi = rng.standard_normal(prob.n).astype(np.float32)
    gacc = rng.standard_normal((prob.n, 3)).astype(np.float32)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, adjoint=True, device=dev)
    plan.set_tuning(tpl, 64, 0, group)
    tp = torch.from_numpy(prob.pos).to(dev)
    plan.tree_build(tp)
    gm, gx = plan.gravity_adjoint(prob.eps, tp, torch.from_numpy(prob.strength).to(dev),
                                  torch.from_numpy(gphi).to(dev), torch.from_numpy(gacc).to(dev))
    torch.cuda.synchronize()
    om, ox = oracle.gravity_adjoint(prob.pos, prob.strength, gphi, gacc, prob.level, prob.lo, prob.edge, prob.eps)
    assert rel_l2(gm.cpu().numpy(), om) <= TOL_REAL
    assert rel_l2(gx.cpu().numpy(), ox) <= TOL_REAL


def test_autograd_helmholtz_matches_oracle(dev):
    n, level, nrhs = 8000, 3, 2
    pos = random_points(n, 41)
    rng = np.random.default_rng(42)
    q = wl.complex_normal((nrhs, n), rng)
    y = wl.complex_normal((nrhs, n), rng)
    k = np.float32(2 * math.pi)
    plan = p2p.Plan("helmholtz", n, level, (0, 0, 0), 1.0, nrhs=nrhs, adjoint=True, device=dev)
    tp = torch.from_numpy(pos).to(dev).requires_grad_(True)
    tq = torch.from_numpy(q).to(dev).requires_grad_(True)
    u = p2p.helmholtz_p2p(tp, tq, plan, float(k))
    loss = torch.real(torch.sum(torch.conj(torch.from_numpy(y).to(dev)) * u))
    loss.backward()
    oq, ox = oracle.helmholtz_adjoint(pos, q, y, level, (0, 0, 0), 1.0, k)
    assert rel_l2(tq.grad.cpu().numpy(), oq) <= TOL_COMPLEX
    assert rel_l2(tp.grad.cpu().numpy(), ox) <= TOL_REAL


def test_autograd_gravity_matches_oracle(dev):
    prob = wl.uniform_gravity(n=8192, level=3, seed=5)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, adjoint=True, device=dev)
    tp = torch.from_numpy(prob.pos).to(dev).requires_grad_(True)
    tm = torch.from_numpy(prob.strength).to(dev).requires_grad_(True)
    phi, acc = p2p.gravity_p2p(tp, tm, plan, prob.eps)
    rng = np.random.default_rng(3)
    gphi = rng.standard_normal(prob.n).astype(np.float32)
    gacc = rng.standard_normal((prob.n, 3)).astype(np.float32)
    loss = (phi * torch.from_numpy(gphi).to(dev)).sum() + (acc * torch.from_numpy(gacc).to(dev)).sum()
    loss.backward()
    om, ox = oracle.gravity_adjoint(prob.pos, prob.strength, gphi, gacc, prob.level, prob.lo, prob.edge, prob.eps)
    assert rel_l2(tm.grad.cpu().numpy(), om) <= TOL_REAL
    assert rel_l2(tp.grad.cpu().numpy(), ox) <= TOL_REAL


def dbim_gradient(prob, dev):
    """GPU: L(chi) = ||P(chi u_inc) - P(chi2 u_inc)||^2 and dL/dchi by autograd."""
    k = prob.k
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=1, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    uinc = torch.from_numpy(prob.extra["uinc"]).to(dev)
    chi2 = torch.from_numpy(prob.extra["chi2"]).to(dev)
    with torch.no_grad():
        d = p2p.helmholtz_p2p(pos, (chi2 * uinc)[None], plan, k)
    chi = torch.from_numpy(prob.extra["chi"]).to(dev).requires_grad_(True)
    u = p2p.helmholtz_p2p(pos, (chi * uinc)[None], plan, k)
    loss = torch.sum(torch.abs(u - d) ** 2)
    loss.backward()
    return chi.grad.detach().cpu().numpy()


def test_dbim_gradient_64_vs_oracle(dev):
    prob = wl.diff_helmholtz(edge_points=64)
    g = dbim_gradient(prob, dev)
    q1 = (prob.extra["chi"] * prob.extra["uinc"]).astype(np.complex64)
    q2 = (prob.extra["chi2"] * prob.extra["uinc"]).astype(np.complex64)
    u1, _ = oracle.helmholtz(prob.pos, q1[None], prob.level, prob.lo, prob.edge, prob.k)
    u2, _ = oracle.helmholtz(prob.pos, q2[None], prob.level, prob.lo, prob.edge, prob.k)
    gbar = (2.0 * (u1 - u2)).astype(np.complex64)
    gq, _ = oracle.helmholtz_adjoint(prob.pos, q1[None], gbar, prob.level, prob.lo, prob.edge, prob.k)
    ref = np.conj(prob.extra["uinc"].astype(np.complex128)) * gq[0]
    assert rel_l2(g, ref) <= TOL_COMPLEX


def test_dbim_gradient_128_finite_differences(dev):
    """L is quadratic in (Re chi, Im chi): central differences are exact up to
    rounding.  A perturbation of chi_m changes u only on m's neighbourhood
    (column m of P), so each difference is evaluated there in FP64."""
    prob = wl.diff_helmholtz(edge_points=128)
    g = dbim_gradient(prob, dev)
    uinc = prob.extra["uinc"].astype(np.complex128)
    q1 = (prob.extra["chi"] * prob.extra["uinc"]).astype(np.complex64)
    q2 = (prob.extra["chi2"] * prob.extra["uinc"]).astype(np.complex64)
    u1, _ = oracle.helmholtz(prob.pos, q1[None], prob.level, prob.lo, prob.edge, prob.k)
    u2, _ = oracle.helmholtz(prob.pos, q2[None], prob.level, prob.lo, prob.edge, prob.k)
    r = (u1 - u2)[0]
    cells, _ = oracle.cells(prob.pos, prob.level, prob.lo, prob.edge)
    delta = 1e-3
    fd, got = [], []
    for m in prob.extra["fd_idx"]:
        near = np.nonzero(np.abs(cells - cells[m]).max(axis=1) <= 1)[0]
        em = np.zeros((1, prob.n), np.complex64)
        em[0, m] = 1.0
        col, _ = oracle.helmholtz(prob.pos, em, prob.level, prob.lo, prob.edge, prob.k, targets=near)
        col = col[0]
        val = []
        for e in (1.0, 1j):
            dv = e * uinc[m] * col
            lp = np.sum(np.abs(r[near] + delta * dv) ** 2)
            lm = np.sum(np.abs(r[near] - delta * dv) ** 2)
            val.append((lp - lm) / (2 * delta))
        fd.append(val[0] + 1j * val[1])
        got.append(g[m])
    assert rel_l2(np.array(got), np.array(fd)) <= TOL_COMPLEX

"""Invariants of the operator checked on the GPU with the library's FP64
device reductions (p2p_momentum_fp64, p2p_dot_fp64): the momentum of the
gravity near field vanishes, and the adjoints satisfy the inner-product
identity with the forward operators.  The operator computes in FP32; only
these global sums accumulate in FP64."""
import math

import numpy as np
import pytest
import torch

from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def gravity_outputs(prob, dev, layout="redundant", symmetric=False, periodic=False):
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, symmetric=symmetric,
                    periodic=periodic, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    m = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(pos)
    plan.restructure(pos, m)
    phi, acc = plan.gravity(prob.eps)
    assert plan.counters()["status"] == 0
    return m, phi, acc


@pytest.mark.parametrize("layout,symmetric,periodic", [
    ("redundant", False, False), ("indirect", False, False), ("pairtask", False, False),
    ("redundant", True, False), ("symmetric", False, False), ("redundant", False, True),
    ("indirect", True, True)])
def test_momentum_invariant_fp64(dev, layout, symmetric, periodic):
    prob = wl.plummer_gravity(n=60000, level=6, eps=1e-3, seed=5)
    m, _, acc = gravity_outputs(prob, dev, layout, symmetric, periodic)
    out = p2p.momentum_fp64(m, acc).cpu().numpy()
    # the device sums against the same sums taken on the host in float64
    f = acc.cpu().numpy().astype(np.float64) * prob.strength.astype(np.float64)[:, None]
    np.testing.assert_allclose(out[3:], np.abs(f).sum(axis=0), rtol=1e-12)
    np.testing.assert_allclose(out[:3], f.sum(axis=0), rtol=1e-9, atol=1e-12 * out[3:].max())
    assert np.abs(out[:3]).max() <= 1e-6 * out[3:].max()


def test_momentum_fp64_of_a_plain_array(dev):
    """The reduction itself on inputs with a known exact sum."""
    n = 100003
    m = torch.full((n,), 0.5, dtype=torch.float32, device=dev)
    acc = torch.arange(3 * n, dtype=torch.float32, device=dev).reshape(n, 3) % 7 - 3
    out = p2p.momentum_fp64(m, acc).cpu().numpy()
    ref = 0.5 * (np.arange(3 * n).reshape(n, 3) % 7 - 3).astype(np.float64)
    np.testing.assert_array_equal(out[:3], ref.sum(axis=0))
    np.testing.assert_array_equal(out[3:], np.abs(ref).sum(axis=0))


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
@pytest.mark.parametrize("nrhs,periodic", [(1, False), (3, False), (8, False), (1, True)])
def test_helmholtz_adjoint_inner_product_identity(dev, layout, nrhs, periodic):
    """Re<y, P q> = Re<P^H y, q>, both inner products reduced in FP64 on the device."""
    n, level = 12000, 4
    rng = np.random.default_rng(40 + nrhs)
    pos = rng.random((n, 3), dtype=np.float32)
    q = torch.from_numpy(wl.complex_normal((nrhs, n), rng)).to(dev)
    y = torch.from_numpy(wl.complex_normal((nrhs, n), rng)).to(dev)
    k = float(np.float32(2 * math.pi * 2.0))
    plan = p2p.Plan("helmholtz", n, level, (0, 0, 0), 1.0, nrhs=nrhs, layout=layout, periodic=periodic,
                    device=dev)
    tp = torch.from_numpy(pos).to(dev)
    plan.tree_build(tp)
    plan.restructure(tp, q)
    u = plan.helmholtz(k)
    gq, _ = plan.helmholtz_adjoint(k, tp, y, want_q=True, want_pos=False)
    lhs = float(p2p.dot_fp64(y, u))
    rhs = float(p2p.dot_fp64(gq, q))
    scale = math.sqrt(float(p2p.dot_fp64(y, y)) * float(p2p.dot_fp64(u, u)))
    assert abs(lhs - rhs) <= 1e-5 * scale
    # the device inner product equals the host's float64 sum of the same numbers
    host = float(np.sum(np.conj(y.cpu().numpy().astype(np.complex128)) * u.cpu().numpy().astype(np.complex128)).real)
    assert abs(lhs - host) <= 1e-12 * scale


@pytest.mark.parametrize("layout", ["indirect", "redundant"])
def test_gravity_adjoint_inner_product_identity(dev, layout):
    """phi and a are linear in the masses: <g_phi, phi(m)> + <g_a, a(m)> = <grad_m, m>,
    both sides reduced in FP64 on the device."""
    prob = wl.plummer_gravity(n=30000, level=5, eps=1e-3, seed=8)
    rng = np.random.default_rng(9)
    gphi = torch.from_numpy(rng.standard_normal(prob.n).astype(np.float32)).to(dev)
    gacc = torch.from_numpy(rng.standard_normal((prob.n, 3)).astype(np.float32)).to(dev)
    plan = p2p.Plan("gravity", prob.n, prob.level, prob.lo, prob.edge, layout=layout, adjoint=True, device=dev)
    tp = torch.from_numpy(prob.pos).to(dev)
    m = torch.from_numpy(prob.strength).to(dev)
    plan.tree_build(tp)
    plan.restructure(tp, m)
    phi, acc = plan.gravity(prob.eps)
    gm, _ = plan.gravity_adjoint(prob.eps, tp, m, gphi, gacc, want_mass=True, want_pos=False)
    lhs = float(p2p.dot_fp64(gphi, phi)) + float(p2p.dot_fp64(gacc, acc))
    rhs = float(p2p.dot_fp64(gm, m))
    scale = math.sqrt(float(p2p.dot_fp64(gphi, gphi)) * float(p2p.dot_fp64(phi, phi))) + \
        math.sqrt(float(p2p.dot_fp64(gacc, gacc)) * float(p2p.dot_fp64(acc, acc)))
    assert abs(lhs - rhs) <= 1e-5 * scale

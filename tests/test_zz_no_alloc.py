"""The workspace-free gravity entry point (p2p_gravity_noalloc).

It is meant for callers that cannot allocate device memory where they need
the operator; it must give the same results as the workspace-based entry
points.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

TOL_REAL = 1e-5
MAX_N = 8192
MAX_LEVEL = 4


def rel_l2(a, b):
    a, b = a.double().cpu().numpy().ravel(), b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def call_noalloc(pos, mass, prob, layout, phi, acc):
    lib = p2p.load()
    lo = (ctypes.c_float * 3)(*prob.lo)
    return lib.p2p_gravity_noalloc(ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(mass.data_ptr()), prob.n,
                                   prob.level, lo, float(prob.edge), float(prob.eps), p2p.LAYOUTS[layout],
                                   ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(acc.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.gpu
def test_noalloc_matches_workspace_path_two_calls(dev):
    # two different problems in a row: the second call must not see the first call's leftovers
    probs = [wl.uniform_gravity(n=MAX_N, level=3, seed=0), wl.plummer_gravity(n=5000, level=MAX_LEVEL, eps=1e-3, seed=3)]
    for layout in ("redundant", "indirect"):
        for prob in probs:
            pos = torch.from_numpy(prob.pos).to(dev)
            mass = torch.from_numpy(prob.strength).to(dev)
            phi = torch.full((prob.n,), float("nan"), dtype=torch.float32, device=dev)
            acc = torch.full((prob.n, 3), float("nan"), dtype=torch.float32, device=dev)
            assert call_noalloc(pos, mass, prob, layout, phi, acc) == 0
            ref_phi, ref_acc = p2p.gravity(pos, mass, prob.level, prob.lo, prob.edge, prob.eps, layout=layout)
            torch.cuda.synchronize()
            assert torch.isfinite(phi).all() and torch.isfinite(acc).all()
            assert rel_l2(phi, ref_phi) <= TOL_REAL
            assert rel_l2(acc, ref_acc) <= TOL_REAL


@pytest.mark.gpu
def test_noalloc_rejects_oversized_requests(dev):
    prob = wl.uniform_gravity(n=MAX_N + 1, level=3)
    pos = torch.from_numpy(prob.pos).to(dev)
    mass = torch.from_numpy(prob.strength).to(dev)
    phi = torch.empty(prob.n, dtype=torch.float32, device=dev)
    acc = torch.empty(prob.n, 3, dtype=torch.float32, device=dev)
    assert call_noalloc(pos, mass, prob, "redundant", phi, acc) == 5       # P2P_ERR_UNSUPPORTED
    small = wl.uniform_gravity(n=100, level=MAX_LEVEL + 1)
    assert call_noalloc(pos[:100], mass[:100], small, "redundant", phi, acc) == 5

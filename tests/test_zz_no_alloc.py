"""The workspace-free gravity entry point (p2p_gravity_noalloc).

It is meant for callers that cannot allocate device memory where they need
the operator (an allocator that forbids new device allocations, a plugin
handed only its input and output buffers).  It runs the plan set-up, layout
and kernels of the workspace entry points with the default tuning, so its
results must equal theirs bit for bit, and meet the FP64 oracle's tolerance.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

import oracle
from paper_2511_21535_gb300 import p2p
from paper_2511_21535_gb300 import workloads as wl

TOL_REAL = 1e-5
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "p2p_gb300.h")


def header_constant(name: str) -> int:
    m = re.search(r"#define\s+" + name + r"\s+\(?(\d+)\)?", open(HEADER).read())
    return int(m.group(1))


MAX_N = header_constant("P2P_NOALLOC_MAX_N")
MAX_LEVEL = header_constant("P2P_NOALLOC_MAX_LEVEL")
SCRATCH_BYTES = header_constant("P2P_NOALLOC_SCRATCH_BYTES")
ERR_UNSUPPORTED, ERR_DOMAIN = 5, 6


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def call_noalloc(pos, mass, prob, layout, phi, acc):
    lib = p2p.load()
    lo = (ctypes.c_float * 3)(*prob.lo)
    return lib.p2p_gravity_noalloc(ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(mass.data_ptr()), prob.n,
                                   prob.level, lo, float(prob.edge), float(prob.eps), p2p.LAYOUTS[layout],
                                   ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(acc.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def noalloc_status():
    flags = ctypes.c_uint()
    st = p2p.load().p2p_gravity_noalloc_status(ctypes.byref(flags),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, flags.value


def run_noalloc(prob, layout, dev):
    pos = torch.from_numpy(prob.pos).to(dev)
    mass = torch.from_numpy(prob.strength).to(dev)
    phi = torch.full((prob.n,), float("nan"), dtype=torch.float32, device=dev)
    acc = torch.full((prob.n, 3), float("nan"), dtype=torch.float32, device=dev)
    assert call_noalloc(pos, mass, prob, layout, phi, acc) == 0
    return pos, mass, phi, acc


def test_worst_case_layout_fits_the_scratch():
    """The scratch a call needs is the workspace of the equivalent plan: at the
    largest n, for every level up to the limit and both layouts, it fits
    (host only: plan creation queues no device work)."""
    lib = p2p.load()
    worst = 0
    for level in range(1, MAX_LEVEL + 1):
        for layout in ("indirect", "redundant"):
            h = ctypes.c_void_p()
            lo = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
            assert lib.p2p_plan_create(ctypes.byref(h), p2p.GRAVITY, MAX_N, level, lo, 1.0, 1,
                                       p2p.LAYOUTS[layout], 0) == 0
            nb = ctypes.c_size_t()
            assert lib.p2p_plan_workspace_bytes(h, ctypes.byref(nb)) == 0
            lib.p2p_plan_destroy(h)
            worst = max(worst, nb.value)
    assert 0 < worst <= SCRATCH_BYTES


@pytest.mark.gpu
def test_noalloc_matches_workspace_path_two_calls(dev):
    """Two different problems in a row, both layouts, the largest accepted size
    among them: the no-workspace call equals the workspace path bit for bit
    (the second call must not see the first call's leftovers)."""
    probs = [wl.uniform_gravity(n=MAX_N, level=MAX_LEVEL, seed=0),
             wl.plummer_gravity(n=5000, level=3, eps=1e-3, seed=3)]
    for layout in ("redundant", "indirect"):
        for prob in probs:
            pos, mass, phi, acc = run_noalloc(prob, layout, dev)
            ref_phi, ref_acc = p2p.gravity(pos, mass, prob.level, prob.lo, prob.edge, prob.eps, layout=layout)
            torch.cuda.synchronize()
            assert noalloc_status() == (0, 0)
            assert torch.equal(phi, ref_phi) and torch.equal(acc, ref_acc)


@pytest.mark.gpu
def test_noalloc_matches_the_oracle(dev):
    prob = wl.plummer_gravity(n=MAX_N, level=MAX_LEVEL, eps=1e-3, seed=5)
    _, _, phi, acc = run_noalloc(prob, "redundant", dev)
    torch.cuda.synchronize()
    ophi, oacc, _ = oracle.gravity(prob.pos, prob.strength, prob.level, prob.lo, prob.edge, prob.eps)
    assert rel_l2(phi.cpu().numpy(), ophi) <= TOL_REAL
    assert rel_l2(acc.cpu().numpy(), oacc) <= TOL_REAL


@pytest.mark.gpu
def test_noalloc_reports_device_errors(dev):
    """A NaN position is detected on the device: the call itself returns OK (it
    only queues work), the status call reports P2P_ERR_DOMAIN; a valid call
    afterwards reports OK again."""
    prob = wl.uniform_gravity(n=2000, level=3, seed=7)
    bad = prob.pos.copy()
    bad[11, 2] = np.nan
    bad_prob = wl.Problem(prob.name, bad, prob.strength, prob.level, prob.lo, prob.edge, "gravity", eps=prob.eps)
    run_noalloc(bad_prob, "redundant", dev)
    st, flags = noalloc_status()
    assert st == ERR_DOMAIN and flags & p2p.FLAG_DOMAIN
    run_noalloc(prob, "indirect", dev)
    assert noalloc_status() == (0, 0)


@pytest.mark.gpu
def test_noalloc_rejects_oversized_requests(dev):
    prob = wl.uniform_gravity(n=MAX_N + 1, level=3)
    pos = torch.from_numpy(prob.pos).to(dev)
    mass = torch.from_numpy(prob.strength).to(dev)
    phi = torch.empty(prob.n, dtype=torch.float32, device=dev)
    acc = torch.empty(prob.n, 3, dtype=torch.float32, device=dev)
    assert call_noalloc(pos, mass, prob, "redundant", phi, acc) == ERR_UNSUPPORTED
    small = wl.uniform_gravity(n=100, level=MAX_LEVEL + 1)
    assert call_noalloc(pos[:100], mass[:100], small, "redundant", phi, acc) == ERR_UNSUPPORTED

"""Randomized plans through the checked library variant (run as a child
process by test_gpu_checked.py, with P2P_GB300_VARIANT=checked).

Every case draws a kernel, layout, evaluation mode, boundary condition,
particle count, level, distribution and tuning from one seeded generator,
runs tree build, restructuring and the operator, and compares with the FP64
oracle.  Prints one JSON line per case: the library status, the device flags
(P2P_FLAG_BOUNDS = 0x10 means an index check failed) and the error.
"""
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_21535_gb300 import p2p  # noqa: E402
from paper_2511_21535_gb300 import workloads as wl  # noqa: E402


def rel_l2(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.max(np.abs(a)) if a.size else 0.0)


def draw(rng):
    kind = ["gravity", "helmholtz"][rng.integers(2)]
    mode = ["indirect", "redundant", "pairtask", "symmetric", "indirect+sym", "redundant+sym"][rng.integers(6)]
    level = int(rng.integers(1, 7))
    dist = ["uniform", "plummer", "one_box"][rng.integers(3)]
    # at most ~3e7 oracle pairs: n^2 * min(1, 27 / 8^level) uniform, about n^2 / 10 for the
    # Plummer core, n^2 in one box
    frac = {"uniform": min(1.0, 27.0 / 8 ** level), "plummer": min(1.0, max(0.1, 27.0 / 8 ** level)),
            "one_box": 1.0}[dist]
    nmax = int(min(40000, np.sqrt(3e7 / frac)))
    n = int(np.exp(rng.uniform(0.0, np.log(nmax))))
    periodic = bool(rng.integers(2)) and level >= 2 and dist == "uniform"
    sym = mode == "symmetric" or mode.endswith("+sym")
    # symmetric Helmholtz plans take one or two right-hand sides
    nrhs = 1 if kind == "gravity" else int(([1, 2] if sym else [1, 2, 3, 8])[rng.integers(2 if sym else 4)])
    tuning = None
    if rng.integers(2):
        # targets per lane: 1, 2 (4 for gravity); symmetric kernels take 2
        tpls = [2] if sym else [1, 2, 4]
        tuning = (int(tpls[rng.integers(len(tpls))]), int([32, 64][rng.integers(2)]), 0,
                  int([1, 2, 4][rng.integers(3)]))
    return dict(kind=kind, mode=mode, level=level, n=n, dist=dist, periodic=periodic, nrhs=nrhs, tuning=tuning)


def points(c, rng):
    n = c["n"]
    if c["dist"] == "uniform":
        return wl.uniform_points(n, rng)
    if c["dist"] == "plummer":
        return wl.plummer_points(n, 0.05, (0.5, 0.5, 0.5), rng)
    cell = 1.0 / (1 << c["level"])                 # everything inside one leaf box
    return (0.25 + rng.uniform(0.0, cell, size=(n, 3))).astype(np.float32)


def run_case(c, seed, dev):
    rng = np.random.default_rng(seed)
    pos = points(c, rng)
    lo, edge = (0.0, 0.0, 0.0), 1.0
    layout = c["mode"].split("+")[0]
    sym = c["mode"].endswith("+sym")
    try:
        plan = p2p.Plan(c["kind"], c["n"], c["level"], lo, edge, nrhs=c["nrhs"], layout=layout,
                        periodic=c["periodic"], symmetric=sym, device=dev)
        if c["tuning"]:
            plan.set_tuning(*c["tuning"])
    except p2p.P2PError as e:                       # a combination the library refuses by design
        return dict(refused=e.status)
    tpos = torch.from_numpy(pos).to(dev)
    if c["kind"] == "gravity":
        m = rng.uniform(0.5, 1.5, size=c["n"]).astype(np.float32)
        plan.tree_build(tpos)
        plan.restructure(tpos, torch.from_numpy(m).to(dev))
        try:
            phi, acc = plan.gravity(1e-3)
        except p2p.P2PError as e:
            return dict(refused=e.status)
        torch.cuda.synchronize()
        ophi, oacc, _ = oracle.gravity(pos, m, c["level"], lo, edge, 1e-3, periodic=c["periodic"])
        err = max(rel_l2(phi.cpu().numpy(), ophi), rel_l2(acc.cpu().numpy(), oacc))
        tol = 1e-5
    else:
        q = wl.complex_normal((c["nrhs"], c["n"]), rng)
        plan.tree_build(tpos)
        plan.restructure(tpos, torch.from_numpy(q).to(dev))
        try:
            u = plan.helmholtz(20.0)
        except p2p.P2PError as e:
            return dict(refused=e.status)
        torch.cuda.synchronize()
        ou, _ = oracle.helmholtz(pos, q, c["level"], lo, edge, 20.0, periodic=c["periodic"])
        err = rel_l2(u.cpu().numpy(), ou)
        tol = 2e-5
    ctr = plan.counters()
    return dict(status=ctr["status"], flags=ctr["flags"], err=err, tol=tol)


def main():
    cases, seed = int(sys.argv[1]), int(sys.argv[2])
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    assert p2p.load().p2p_build_checked() == 1, "the checked variant was not loaded"
    rng = np.random.default_rng(seed)
    for i in range(cases):
        c = draw(rng)
        res = run_case(c, seed * 1000 + i, dev)
        print(json.dumps(dict(case=c, **res)), flush=True)


if __name__ == "__main__":
    main()

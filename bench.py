"""Benchmark: near-field (P2P) pair interactions per second on one GB300.

One step = the whole hot path on one batch of synthetic input already in HBM:
tree build (Morton keys, radix sort, box CSR, E2 neighbour lists) ->
restructuring (box-ordered records, redundant per-box streams) -> P2P kernel
(outputs written in original order).  The step is captured once in a CUDA
graph and replayed (--no-graph launches it kernel by kernel); phase times come
from CUDA events the library records on the launching stream (external event
nodes inside the graph).

Default workload: the clustered gravity case, 4,194,304 particles (a Plummer
sphere of scale radius 0.05 plus a 10 % uniform background) on a level-7
octree with eps = 1e-4, redundant layout; the indirect layout on the same
workload is reported beside it (`indirect`, `layouts_compared`), and the
64^3 Helmholtz grid (both layouts, the symmetric evaluation, two batches in
flight) as the `grid_helmholtz_64` object.  The batched forward + adjoint of
64 uneven grids x 8 right-hand sides against per-instance launches is the
`batched` object, the differentiable 128^3 step the `adjoint` object.

`e2e` is the same step from pinned host buffers through the library's
host-buffer call (p2p_gravity_host / p2p_helmholtz_host): the positions' and
strengths' copies to the device and the results' copy back are inside the
timed region.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(the only other code path this script may run), on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_21535_gb300 import workloads as wl  # noqa: E402

METRIC = "P2P pair-interactions/s"


def kernel_name(kind: str, symmetric: bool, pattern: bool = False, tile2d: bool = False, nrhs: int = 1) -> str:
    """The dominant kernel of a step: Helmholtz runs k_helmholtz_pattern in pattern mode,
    k_helmsym for a symmetric evaluation, k_helmplanar for four or more right-hand sides,
    k_helmtile for one-sided plans of one or two right-hand sides with four targets per
    lane (the default), else k_helmholtz; gravity runs k_gravity_pk (packed, two or four
    targets per lane: tile2d) one-sided, else k_gravity."""
    if kind == "helmholtz":
        if pattern:
            return "k_helmholtz_pattern"
        if symmetric:
            return "k_helmsym"
        if nrhs >= 4:
            return "k_helmplanar"
        if tile2d:
            return "k_helmtile"
        return "k_helmholtz"
    return "k_gravity_pk" if (tile2d and not symmetric) else "k_gravity"


def traffic_records(entry):
    """The capture records of one kernel: a single record or a list of them
    (one per workload, layout or evaluation)."""
    if isinstance(entry, dict):
        return [entry]
    return list(entry) if entry else []


def kernel_traffic(kernel: str, workload: str, layout: str, n: int, symmetric: bool):
    """DRAM bytes per launch from the committed ncu capture of this kernel on
    this workload, layout and evaluation, if the kernel's sources are
    unchanged since that capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    try:
        entry = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    for rec in traffic_records(entry):
        if rec.get("workload") != workload or rec.get("layout") != layout:
            continue
        if bool(rec.get("symmetric", False)) != symmetric:
            continue
        if rec.get("n") is not None and rec["n"] != n:
            continue
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, "paper_2511_21535_gb300", "csrc", f), "rb").read())
        return rec["dram_bytes_per_launch"] if h.hexdigest()[:16] == rec["source_hash"] else None
    return None
L2_FLUSH_BYTES = 512 << 20     # > 129 MB L2
MUFU_PER_SM_CLK = 16           # nominal XU (MUFU) throughput per SM per clock
FP32_PER_SM_CLK = 128


def replica_throughput(units: float, ms: float, dist: bool, device=None):
    """Whole-job throughput of independent replicas (one per GPU): the units
    of all ranks over the slowest rank's time per step.  Returns (units/s,
    max ms, total units); every rank gets the same values."""
    if not dist:
        return units / (ms * 1e-3), ms, units
    import torch
    import torch.distributed as td
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_units = torch.tensor([float(units)], dtype=torch.float64, device=device)
    td.all_reduce(t_ms, op=td.ReduceOp.MAX)
    td.all_reduce(t_units, op=td.ReduceOp.SUM)
    td.barrier()
    ms_max, total = float(t_ms.item()), float(t_units.item())
    return total / (ms_max * 1e-3), ms_max, total


def make_problem(name: str, periodic: bool = False):
    prob = _make_problem(name)
    prob.extra["periodic"] = bool(periodic)
    return prob


def _make_problem(name: str):
    if name == "grid_helmholtz":
        return wl.grid_helmholtz()
    if name == "uniform_gravity":
        return wl.uniform_gravity()
    if name == "plummer_gravity":
        return wl.plummer_gravity()
    if name == "grid_helmholtz_128":
        return wl.grid_helmholtz(edge_points=128)
    if name == "plummer_gravity_1m":
        return wl.plummer_gravity(n=1 << 20, level=6)
    if name == "grid_helmholtz_r8":
        return wl.grid_helmholtz(nrhs=8)
    raise SystemExit(f"unknown workload {name}")


def workload_config(prob, layout, pattern=False, symmetric=False):
    cfg = {"workload": prob.name, "n": prob.n, "level": prob.level, "kernel": prob.kind, "layout": layout,
           "kernel_mode": "pattern table" if pattern else "direct",
           "evaluation": "symmetric (each pair of small box pairs once)" if symmetric else "one-sided",
           "boundary": "periodic" if prob.extra.get("periodic") else "open", "nrhs": prob.nrhs,
           "l2": "flushed between steps (512 MiB write)", "inputs": "seeded synthetic"}
    if prob.kind == "gravity":
        cfg["eps"] = prob.eps
    else:
        cfg["k"] = prob.k
        cfg["spacing"] = wl.SPACING
    return cfg


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons of the samples taken in
        [t0, t1] (host time of the timed region); if fewer than 3 fall inside,
        the 3 samples closest to the window's end are used and "window" says so."""
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        rows = []
        for ts, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        window = "timed"
        sel = [r for r in rows if t0 is None or (t0 - 0.15 <= r[0] <= t1 + 0.15)]
        if len(sel) < 3 and rows:
            window = "nearest to the timed region"
            sel = sorted(rows, key=lambda r: abs(r[0] - (t1 or r[0])))[:3]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = sorted({nm for r in sel for nm, v in zip(names, r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
                "reasons": reasons, "samples": len(sel), "window": window}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def roofline_of(prob, kern_ms: float, evals: int, pipes: dict, f_mhz: float, sms: int, pattern: bool = False):
    """Pipe roofline of the P2P kernel: pipe lanes per SM per clock (measured by
    p2p_measure_pipes) x SMs x sampled SM clock / operations per pair evaluation."""
    mufu_rate = min(pipes["mufu_rsqrt"], pipes["mufu_sin"])
    if prob.kind == "helmholtz" and pattern:
        # table lookups: one 8-byte shared load per lane and pair; 128 B/clk/SM of shared bandwidth
        pipe, per_pair, rate = "smem", 8.0, 128.0
    elif prob.kind == "helmholtz" and prob.nrhs <= 2:
        pipe, per_pair, rate = "mufu", 3.0, mufu_rate      # rsqrt, sin, cos per geometric pair
    elif prob.kind == "helmholtz":
        pipe, per_pair, rate = "fp32", 12.0 + 4.0 * prob.nrhs, pipes["fp32"]
    else:
        pipe, per_pair, rate = "fp32", 13.0, pipes["fp32"]
    peak = rate * sms * f_mhz * 1e6 / per_pair
    achieved = evals / (kern_ms * 1e-3)
    return {"bound": "alu", "pipe": pipe, "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": achieved / peak, "ops_per_pair": per_pair, "sm_mhz": f_mhz, "sms": sms,
            "evaluations_per_launch": evals,
            "peak_source": "pipe rates measured by p2p_measure_pipes x SMs x sampled SM clock"}


def measure_arm(prob, layout: str, args, dev, pipes: dict, clk, steps: int, warmup: int, symmetric: bool = False,
                pattern: bool = False, e2e: bool = True):
    """One layout of one workload: the whole step (tree, restructuring, P2P
    kernel with the update to original order) captured in one CUDA graph and
    replayed `steps` times (L2 flushed between steps), phase times from the
    plan's events, and the same step end to end from pinned host buffers
    through p2p_*_host.  Returns the arm's record (the plan is released)."""
    import torch
    from paper_2511_21535_gb300 import p2p

    plan = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    timing=True, periodic=bool(prob.extra.get("periodic")), symmetric=symmetric, host_io=e2e,
                    device=dev)
    if args.tpl:
        plan.set_tuning(args.tpl, args.tile, args.ctas, args.group)
    if pattern:
        plan.set_grid(wl.SPACING, wl.LEAF_EDGE_POINTS)
    pos = torch.from_numpy(prob.pos).to(dev)
    strength = torch.from_numpy(prob.strength).to(dev)
    out_a = torch.empty(prob.n, dtype=torch.float32, device=dev)
    out_b = torch.empty(prob.n, 3, dtype=torch.float32, device=dev)
    out_u = torch.empty(prob.nrhs, prob.n, dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.tree_build(pos)
        plan.restructure(pos, strength)
        if prob.kind == "gravity":
            plan.gravity(prob.eps, out_a, out_b)
        else:
            plan.helmholtz(prob.k, out_u)

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    cnt = plan.counters(check=True)
    geo_pairs = cnt["pairs"]
    pairs = geo_pairs * (prob.nrhs if prob.kind == "helmholtz" else 1)
    sym = symmetric or layout == "symmetric"
    evals = cnt.get("evals", geo_pairs) if sym else geo_pairs

    # capture the whole step (tree, restructuring, operator) in one CUDA graph
    run, graph, graph_note, launches_per_replay, graph_events = step, None, None, None, False
    if args.graph:
        try:
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                step()
            stream.wait_stream(side)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            l0 = p2p.launch_count()
            with torch.cuda.graph(graph):
                step()
            launches_per_replay = p2p.launch_count() - l0
            for _ in range(warmup):
                flush.zero_()
                graph.replay()
            torch.cuda.synchronize()
            run = graph.replay
            graph_note = "whole step captured in one CUDA graph"
            try:                       # phase events recorded by the replay itself
                plan.timing()
                graph_events = True
                graph_note += "; phase times from external event nodes of the replay"
            except Exception:
                graph_events = False
        except Exception as e:  # report and fall back to stream launches
            graph, run = None, step
            graph_note = f"graph capture failed: {type(e).__name__}: {e}"[:200]

    if dist_active():
        import torch.distributed as td
        td.barrier()
    torch.cuda.synchronize()
    launches0 = p2p.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    phases = {k: [] for k in p2p.PHASES}
    t_start = time.time()
    # the timed steps are enqueued back to back (no host wait inside the loop,
    # so host delays cannot idle the GPU between steps)
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    # phase times from further steps, each read when it has ended (the replay's
    # event nodes, or the same step launched on the stream where a replay
    # records none)
    for _ in range(min(steps, 50)):
        flush.zero_()
        run() if graph_events else step()
        for k, v in plan.timing().items():
            phases[k].append(v)
    torch.cuda.synchronize()
    launches = p2p.launch_count() - launches0
    if graph is not None:
        launches = launches_per_replay * steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    srt = sorted(step_ms)
    spread = {"min": srt[0], "median": srt[len(srt) // 2], "max": srt[-1]}
    csum = clk.summary(t_start, t_end)
    phases_ms = {k: (sum(v) / len(v) if v else None) for k, v in phases.items()}
    rec = {"layout": layout, "evaluation": "symmetric" if sym else "one-sided", "ms_per_step": ms,
           "step_ms_spread": spread,
           "pairs_per_step": pairs, "geometric_pairs": geo_pairs, "phases_ms": phases_ms,
           "kernel_ms": phases_ms["kernel"], "gpu_launches": launches, "graph": graph_note, "clocks": csum,
           "n_boxes": cnt["n_boxes"], "redundant_records": cnt["total_src"] if layout != "indirect" else 0}
    rec["evaluations_per_launch"] = evals

    if e2e:
        # end to end through the C ABI's host-buffer step (p2p_*_host) from pinned
        # host buffers: H2D of positions and strengths (the strengths' copy
        # overlapped with the tree build), full step, D2H of the results
        hpos = torch.from_numpy(prob.pos).pin_memory()
        hstr = torch.from_numpy(prob.strength).pin_memory()
        if prob.kind == "gravity":
            hout = (torch.empty(prob.n, dtype=torch.float32).pin_memory(),
                    torch.empty(prob.n, 3, dtype=torch.float32).pin_memory())
        else:
            hout = (torch.empty(prob.nrhs, prob.n, dtype=torch.complex64).pin_memory(),)

        def e2e_step():
            if prob.kind == "gravity":
                plan.gravity_host(prob.eps, hpos, hstr, hout[0], hout[1])
            else:
                plan.helmholtz_host(prob.k, hpos, hstr, hout[0])

        for _ in range(max(1, warmup)):
            flush.zero_()
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = []
        for i in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e_mean = sum(e2e_ms) / len(e2e_ms)
        rec["e2e"] = {"value": pairs / (e2e_mean * 1e-3), "unit": "pairs/s",
                      "h2d_bytes_per_step": prob.pos.nbytes + prob.strength.nbytes,
                      "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in hout), "ms_per_step": e2e_mean}
    rec["value"] = pairs / (ms * 1e-3)
    rec["unit"] = "pairs/s"
    del plan, pos, strength, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def kernel_of(prob, layout: str, args, symmetric: bool, pattern: bool):
    """The dominant kernel of an arm, by the library's default tuning."""
    if prob.kind == "helmholtz":
        tile2d = not symmetric and layout != "symmetric" and prob.nrhs <= 2 and args.tpl in (0, 4)
    else:
        tile2d = not symmetric and layout != "symmetric" and args.tpl in (0, 2, 4)
    return kernel_name(prob.kind, symmetric or layout == "symmetric", pattern, tile2d, prob.nrhs)


def arm_with_roofline(prob, layout, args, dev, pipes, clk, steps, warmup, symmetric=False, pattern=False):
    import torch
    rec = measure_arm(prob, layout, args, dev, pipes, clk, steps, warmup, symmetric, pattern)
    f_mhz = rec["clocks"]["sm_mhz"] or pipes["sm_mhz"] or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    kname = kernel_of(prob, layout, args, symmetric, pattern)
    roof = roofline_of(prob, rec["kernel_ms"], rec["evaluations_per_launch"], pipes, f_mhz, sms, pattern)
    roof["kernel"] = kname
    roof["traffic"] = (None if prob.extra.get("periodic") else
                       kernel_traffic(kname, prob.name, layout, prob.n, symmetric or layout == "symmetric"))
    roof["work_unit"] = ("pair evaluation (a mutual one serves two ordered pairs)"
                         if rec["evaluations_per_launch"] != rec["geometric_pairs"] else "ordered pair")
    rec["roofline"] = roof
    return rec


_DIST = {"on": False}


def dist_active() -> bool:
    return _DIST["on"]


def run_gpu(args, rank, world, local_rank):
    """The bench line: the selected workload and layout (default: the 4.2 M
    Plummer sphere, redundant layout), the other target-owned layout on the
    same workload beside it, and (for the default) the 64^3 Helmholtz grid
    with both layouts as a secondary object."""
    import torch
    from paper_2511_21535_gb300 import p2p

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    _DIST["on"] = world > 1
    prob = make_problem(args.workload, args.periodic)
    layout = args.layout
    # symmetric evaluation applies to the target-owned layouts in direct mode with <= 2 right-hand sides
    symmetric = (args.evaluation == "symmetric" and not args.pattern and layout in ("redundant", "indirect")
                 and (prob.kind == "gravity" or prob.nrhs <= 2))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_id = vis.split(",")[local_rank].strip() if vis else str(local_rank)
    clk = ClockSampler(smi_id).__enter__()
    time.sleep(0.5)
    pipes = p2p.measure_pipes()
    main = arm_with_roofline(prob, layout, args, dev, pipes, clk, args.steps, args.warmup, symmetric, args.pattern)
    value, ms, _ = replica_throughput(main["pairs_per_step"], main["ms_per_step"], world > 1, dev)
    e2e = dict(main["e2e"])
    e2e["value"], e2e["ms_per_step"], _ = replica_throughput(main["pairs_per_step"], e2e["ms_per_step"],
                                                             world > 1, dev)
    result = {
        "metric": METRIC,
        "value": value,
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(prob, layout, args.pattern, symmetric),
        "e2e": e2e,
        "roofline": dict(main["roofline"], pipe_rates_per_sm_clk={k: round(v, 3) for k, v in pipes.items()}),
        "phases_ms": main["phases_ms"],
        "step_ms_spread": main["step_ms_spread"],
        "pairs_per_step": main["pairs_per_step"],
        "gpu_launches": main["gpu_launches"],
        "graph": main["graph"],
        "clocks": main["clocks"],
    }
    if not args.no_arms and not args.pattern and layout in ("redundant", "indirect"):
        other = "indirect" if layout == "redundant" else "redundant"
        arm = arm_with_roofline(prob, other, args, dev, pipes, clk, args.steps, args.warmup, symmetric)
        result[other] = {k: arm[k] for k in ("value", "unit", "ms_per_step", "kernel_ms", "phases_ms", "e2e",
                                             "roofline", "gpu_launches", "clocks")}
        result["layouts_compared"] = {
            "workload": prob.name, "unit": "pairs/s",
            layout: {"step": value, "kernel": main["pairs_per_step"] / (main["kernel_ms"] * 1e-3),
                     "e2e": e2e["value"], "restructure_ms": main["phases_ms"]["restructure"]},
            other: {"step": arm["value"], "kernel": arm["pairs_per_step"] / (arm["kernel_ms"] * 1e-3),
                    "e2e": arm["e2e"]["value"], "restructure_ms": arm["phases_ms"]["restructure"]}}
    return result, prob, pipes, clk


def grid_secondary(args, dev, pipes, clk, steps: int):
    """The 64^3 Helmholtz grid (262,144 points at lambda/10, 4^3-point leaves,
    one right-hand side): redundant and indirect arms with their rooflines,
    the symmetric evaluation, and two batches in flight."""
    prob = make_problem("grid_helmholtz", args.periodic)
    out = {"workload": "grid_helmholtz_64", "config": workload_config(prob, "redundant")}
    for layout in ("redundant", "indirect"):
        rec = arm_with_roofline(prob, layout, args, dev, pipes, clk, steps, args.warmup)
        out[layout] = {k: rec[k] for k in ("value", "unit", "ms_per_step", "kernel_ms", "phases_ms", "e2e",
                                           "roofline", "gpu_launches", "clocks")}
    mufu_peak = out["redundant"]["roofline"]["peak"] * 1e9
    out["symmetric"] = evaluation_variant(prob, "redundant", dev, steps, mufu_peak)
    out["pipelined"] = pipelined_batches(prob, "redundant", dev, min(max(steps, 20), 400))
    return out


# ---------------------------------------------------------------------------
# secondary measurements of the default line
# ---------------------------------------------------------------------------

def timed_graph_steps(step, steps: int, flush, stream):
    """CUDA-graph replay of `step`, mean ms per replay over `steps` (L2 flushed between)."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(3):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:   # enqueued back to back, read at the end
        flush.zero_()
        a.record(stream)
        graph.replay()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def evaluation_variant(prob, layout: str, dev, steps: int, mufu_peak: float):
    """The same workload with symmetric evaluation (each pair of a small box pair once)."""
    import torch
    from paper_2511_21535_gb300 import p2p
    plan = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    timing=True, periodic=bool(prob.extra.get("periodic")), symmetric=True, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    strength = torch.from_numpy(prob.strength).to(dev)
    u = torch.empty(prob.nrhs, prob.n, dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        plan.tree_build(pos)
        plan.restructure(pos, strength)
        plan.helmholtz(prob.k, u)

    ms = timed_graph_steps(step, steps, flush, torch.cuda.current_stream())
    t = plan.timing()
    c = plan.counters(check=True)
    evals_per_s = c["evals"] / (t["kernel"] * 1e-3)
    return {"evaluation": "symmetric", "layout": layout, "value": c["pairs"] * prob.nrhs / (ms * 1e-3),
            "unit": "pairs/s", "ms_per_step": ms, "kernel_ms": t["kernel"],
            "phases_ms": t, "evaluations_per_launch": c["evals"],
            "roofline": {"pipe": "mufu", "achieved": evals_per_s / 1e9, "peak": mufu_peak / 1e9,
                         "unit": "G evaluations/s", "frac": evals_per_s / mufu_peak}}


PIPE_COPIES = 32   # rotating input copies: 32 x (positions + strengths) > L2


def pipelined_batches(prob, layout: str, dev, steps: int, ctas_per_sm: int = 3):
    """Throughput of a stream of independent batches with two in flight: two
    plans on two streams, each step a captured graph of the whole path (tree,
    restructuring, P2P) on one of PIPE_COPIES rotating input copies, so the
    collect phase of one batch runs while the other's P2P kernel does.  With
    fewer P2P CTAs per SM (ctas_per_sm) the collect kernels find room on the SMs."""
    import torch
    from paper_2511_21535_gb300 import p2p
    plans = []
    for _ in range(2):
        pl = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                      periodic=bool(prob.extra.get("periodic")), device=dev)
        if ctas_per_sm and prob.kind == "helmholtz" and prob.nrhs <= 2:
            pl.set_tuning(4, 64, ctas_per_sm, 4)   # the default tuning with fewer CTAs per SM
        plans.append(pl)
    pos0 = torch.from_numpy(prob.pos).to(dev)
    str0 = torch.from_numpy(prob.strength).to(dev)
    inputs = [(pos0.clone(), str0.clone()) for _ in range(PIPE_COPIES)]
    if prob.kind == "gravity":
        outs = [(torch.empty(prob.n, device=dev), torch.empty(prob.n, 3, device=dev)) for _ in range(2)]
    else:
        outs = [torch.empty(prob.nrhs, prob.n, dtype=torch.complex64, device=dev) for _ in range(2)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]

    def step(pl, inp, out):
        pl.tree_build(inp[0])
        pl.restructure(inp[0], inp[1])
        if prob.kind == "gravity":
            pl.gravity(prob.eps, out[0], out[1])
        else:
            pl.helmholtz(prob.k, out)

    for i in range(4):
        with torch.cuda.stream(streams[i % 2]):
            step(plans[i % 2], inputs[i], outs[i % 2])
    torch.cuda.synchronize()
    graphs = []
    for c in range(PIPE_COPIES):   # copy c runs on plan / stream c % 2
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(streams[c % 2]):
            with torch.cuda.graph(g, stream=streams[c % 2]):
                step(plans[c % 2], inputs[c], outs[c % 2])
        graphs.append(g)
    torch.cuda.synchronize()

    def run(n):
        main = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        for st in streams:
            st.wait_stream(main)
        for i in range(n):
            with torch.cuda.stream(streams[i % 2]):
                graphs[i % PIPE_COPIES].replay()
        for st in streams:
            main.wait_stream(st)
        b.record(main)
        b.synchronize()
        return a.elapsed_time(b) / n

    run(min(steps, 20))
    ms = run(steps)
    c = plans[0].counters(check=True)
    units = c["pairs"] * (prob.nrhs if prob.kind == "helmholtz" else 1)
    return {"value": units / (ms * 1e-3), "unit": "pairs/s", "ms_per_step": ms, "steps": steps,
            "batches_in_flight": 2, "streams": 2,
            "ctas_per_sm": ctas_per_sm if (prob.kind == "helmholtz" and prob.nrhs <= 2) else "auto",
            "inputs": f"{PIPE_COPIES} rotating input copies ({PIPE_COPIES * (prob.pos.nbytes + prob.strength.nbytes) >> 20} MiB > L2)"}


def dbim_forward_adjoint(dev, steps: int, pipes: dict, f_mhz: float, edge_points: int = 128):
    """Differentiable 128^3 configuration: L = ||P(chi u_inc) - d||^2 and dL/dchi through
    the autograd wrapper (forward P2P + hand-written adjoint P2P), per step; and the two
    P2P kernels' own times (forward u = P q, adjoint grad_q = conj(P) gbar) from the
    plan's events, for their roofline."""
    import torch
    from paper_2511_21535_gb300 import p2p
    prob = wl.diff_helmholtz(edge_points=edge_points)
    plan = p2p.Plan("helmholtz", prob.n, prob.level, prob.lo, prob.edge, nrhs=1, timing=True, device=dev)
    pos = torch.from_numpy(prob.pos).to(dev)
    uinc = torch.from_numpy(prob.extra["uinc"]).to(dev)
    with torch.no_grad():
        d = p2p.helmholtz_p2p(pos, (torch.from_numpy(prob.extra["chi2"]).to(dev) * uinc)[None], plan, prob.k)
    chi0 = torch.from_numpy(prob.extra["chi"]).to(dev)

    def step():
        chi = chi0.clone().requires_grad_(True)
        u = p2p.helmholtz_p2p(pos, (chi * uinc)[None], plan, prob.k)
        loss = torch.sum(torch.abs(u - d) ** 2)
        loss.backward()
        return chi.grad

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        g = step()
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    pairs = plan.counters(check=True)["pairs"]
    # the two kernels alone: forward on q = chi u_inc, adjoint on gbar = 2 (u - d)
    q = (chi0 * uinc)[None].contiguous()
    fwd, adj = [], []
    for _ in range(steps):
        plan.restructure(pos, q)
        u = plan.helmholtz(prob.k)
        fwd.append(plan.timing()["kernel"])
        plan.helmholtz_adjoint(prob.k, pos, (2.0 * (u - d)).contiguous(), want_q=True, want_pos=False)
        adj.append(plan.timing()["kernel"])
    kf, ka = sum(fwd) / len(fwd), sum(adj) / len(adj)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mufu = min(pipes["mufu_rsqrt"], pipes["mufu_sin"])
    peak = mufu * sms * f_mhz * 1e6 / 3.0
    achieved = 2 * pairs / ((kf + ka) * 1e-3)
    return {"workload": f"{edge_points}^3 grid, contrast sphere r = 0.3 of the extent, plane wave; "
                        "L = ||P(chi u_inc) - d||^2, dL/dchi by the adjoint kernel",
            "n": prob.n, "ms_per_step": ms, "pairs_per_step": 2 * pairs,
            "value": 2 * pairs / (ms * 1e-3), "unit": "pairs/s (forward + adjoint)",
            "kernel_ms": {"forward": kf, "adjoint": ka},
            "roofline": {"bound": "alu", "pipe": "mufu", "kernel": "k_helmtile (forward and adjoint)",
                         "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s", "frac": achieved / peak,
                         "ops_per_pair": 3.0, "sm_mhz": f_mhz, "sms": sms,
                         "peak_source": "MUFU lanes per SM per clock measured by p2p_measure_pipes x SMs x "
                                        "sampled SM clock"},
            "grad_finite": bool(torch.isfinite(g).all())}


# ---------------------------------------------------------------------------
# batched forward + adjoint (64 uneven grid instances x 8 RHS) vs plain launches
# ---------------------------------------------------------------------------

def batched_vs_plain(dev, steps: int, pipes: dict, f_mhz: float, layout: str = "auto"):
    """One CUDA-graph launch computing u = P q and g = conj(P) y for all 64
    instances, against per-instance plans doing restructure + forward +
    adjoint with their own launches; both compensated FP32, and the plain
    plans given the batch's autotuned layout and tuning, so that the ratio
    isolates batching and the graph launch."""
    import torch
    from paper_2511_21535_gb300 import p2p
    probs = wl.batched_helmholtz()
    nrhs = probs[0].nrhs
    k = probs[0].k
    rng = np.random.default_rng(123)
    batch = p2p.Batch([(p.n, p.level, p.lo, p.edge) for p in probs], nrhs, k, pair=True, layout=layout,
                      timing=True, device=dev)
    pos = torch.from_numpy(np.concatenate([p.pos for p in probs])).to(dev)
    q = torch.from_numpy(np.concatenate([p.strength for p in probs], axis=1)).to(dev)
    y = torch.from_numpy(wl.complex_normal((nrhs, batch.N), rng)).to(dev)
    t0 = time.perf_counter()
    batch.build(pos)
    build_s = time.perf_counter() - t0
    best = batch.autotune(pos, q, y)
    u, g = batch.capture(pos, q, y)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        batch.launch()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lb = p2p.launch_count()
    a.record(stream)
    for _ in range(steps):
        batch.launch()
    b.record(stream)
    b.synchronize()
    batched_ms = a.elapsed_time(b) / steps
    batched_kernels = (p2p.launch_count() - lb) // steps
    pairs = batch.counters()["pairs"]
    # the P2P kernel's share of a replay: phase events inside the graph
    kern, restr = [], []
    for _ in range(steps):
        batch.launch()
        t = batch.timing()
        kern.append(t["kernel"])
        restr.append(t["restructure"])
    kernel_ms = sum(kern) / len(kern)
    passes = -(-2 * nrhs // 8)                 # right-hand-side passes of at most 8 (forward and adjoint)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    per_pass = 12.0 + 4.0 * min(8, 2 * nrhs)
    peak = pipes["fp32"] * sms * f_mhz * 1e6 / per_pass
    achieved = pairs * passes / (kernel_ms * 1e-3)

    # plain: one plan per instance, three calls per product; timed with the
    # batch's autotuned tuning and with the plans' default tuning, the faster
    # of the two is the comparison (so the ratio isolates batching and the graph)
    def plain_arm(tuning):
        plans, per = [], []
        for i, pr in enumerate(probs):
            o0, o1 = batch.offsets[i], batch.offsets[i + 1]
            lay = tuning["layout"] if tuning else "indirect"
            pl = p2p.Plan("helmholtz", pr.n, pr.level, pr.lo, pr.edge, nrhs=nrhs, layout=lay, device=dev)
            if tuning:
                pl.set_tuning(tuning["targets_per_lane"], tuning["tile"], 0, tuning["warps_per_item"])
            pp = pos[o0:o1].contiguous()
            pl.tree_build(pp)
            per.append((pp, q[:, o0:o1].contiguous(), y[:, o0:o1].contiguous(),
                        torch.empty(nrhs, pr.n, dtype=torch.complex64, device=dev)))
            plans.append(pl)

        def plain_step():
            outs = []
            for pl, (pp, qi, yi, ui) in zip(plans, per):
                pl.restructure(pp, qi)
                pl.helmholtz(k, ui)
                gi, _ = pl.helmholtz_adjoint(k, pp, yi, want_q=True, want_pos=False)
                outs.append((ui, gi))
            return outs

        for _ in range(2):
            outs = plain_step()
        torch.cuda.synchronize()
        l0 = p2p.launch_count()
        a.record(stream)
        for _ in range(steps):
            outs = plain_step()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / steps, (p2p.launch_count() - l0) // steps, outs

    tuned_ms, plain_launches, outs_tuned = plain_arm(best)
    default_ms, _, outs_default = plain_arm(None)
    plain_ms = min(tuned_ms, default_ms)
    outs = outs_tuned if tuned_ms <= default_ms else outs_default
    # equal accuracy: both against each other (same per-pair arithmetic)
    uc = torch.cat([o[0] for o in outs], dim=1)
    gc = torch.cat([o[1] for o in outs], dim=1)
    diff_u = float(torch.linalg.vector_norm(u - uc) / torch.linalg.vector_norm(uc))
    diff_g = float(torch.linalg.vector_norm(g - gc) / torch.linalg.vector_norm(gc))
    return {"workload": "64 grid instances (edges 16-64, 4^3 leaves, lambda/10), 8 RHS, forward + adjoint",
            "n_total": batch.N, "geometric_pairs": pairs, "rhs_pairs_per_step": pairs * nrhs * 2,
            "batched_ms": batched_ms, "plain_ms": plain_ms, "speedup": plain_ms / batched_ms,
            "batched_pairs_per_s": pairs * nrhs * 2 / (batched_ms * 1e-3),
            "plain_pairs_per_s": pairs * nrhs * 2 / (plain_ms * 1e-3),
            "batched_graph_launches_per_step": 1, "batched_kernels_per_step": int(batched_kernels),
            "plain_kernels_per_step": int(plain_launches),
            "batched_phases_ms": {"restructure": sum(restr) / len(restr), "kernel": kernel_ms},
            "roofline": {"bound": "alu", "pipe": "fp32", "kernel": "k_helmplanar (8 right-hand sides per pass)",
                         "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G geometric pair-passes/s",
                         "frac": achieved / peak, "ops_per_pair_pass": per_pass, "passes": passes,
                         "sm_mhz": f_mhz, "sms": sms,
                         "peak_source": "FP32 lanes per SM per clock measured by p2p_measure_pipes x SMs x "
                                        "sampled SM clock"},
            "rel_l2_batched_vs_plain": {"u": diff_u, "g": diff_g}, "autotune": best,
            "plain_arm": {"plans": len(probs),
                          "calls_per_instance": "restructure, forward, adjoint (strengths only)",
                          "batch_tuning_ms": tuned_ms, "default_tuning_ms": default_ms,
                          "batch_tuning": {"layout": best["layout"], "targets_per_lane": best["targets_per_lane"],
                                           "tile": best["tile"], "warps_per_item": best["warps_per_item"]},
                          "default_tuning": "indirect layout, the plan defaults for 8 right-hand sides",
                          "compared": "the faster of the two"},
            "build_s": build_s}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_context(prob):
    """The oracle's tree of the whole workload, and the seconds its build took."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    ctx = oracle.Context(prob.pos, prob.level, prob.lo, prob.edge, periodic=bool(prob.extra.get("periodic")))
    return ctx, time.perf_counter() - t0


def oracle_sums(ctx, prob, tg) -> int:
    """The oracle's sums at targets tg; returns the pair interactions (per right-hand side)."""
    if prob.kind == "gravity":
        return ctx.gravity(prob.strength, prob.eps, targets=tg)[2]
    _, pairs = ctx.helmholtz(prob.strength, prob.k, targets=tg)
    return pairs * prob.nrhs


def oracle_target_count(ctx, prob, seconds: float, rng) -> int:
    """Random targets per call for about `seconds` of the oracle's sums."""
    nt = 256
    while True:
        tg = rng.choice(prob.n, min(nt, prob.n), replace=False)
        t0 = time.perf_counter()
        oracle_sums(ctx, prob, tg)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * seconds or nt >= prob.n:
            return max(64, min(prob.n, int(nt * seconds / max(dt, 1e-6))))
        nt = min(prob.n, int(nt * max(2.0, 0.5 * seconds / max(dt, 1e-3))))


def oracle_timed(ctx, tree_s, prob, seconds: float, seed: int, calls: int = 4):
    """The oracle's sums at random target samples for about `seconds` (split over
    `calls` calls), with the tree build charged in proportion to the targets
    sampled (tree seconds x targets / n): the throughput of the oracle's whole
    path on this workload, estimated from a bounded sample."""
    rng = np.random.default_rng(seed)
    nt = oracle_target_count(ctx, prob, seconds / calls, rng)
    pairs, t, targets = 0, 0.0, 0
    while t < seconds:
        tg = rng.choice(prob.n, nt, replace=False)
        t0 = time.perf_counter()
        pairs += oracle_sums(ctx, prob, tg)
        t += time.perf_counter() - t0
        targets += nt
    charged = t + tree_s * targets / prob.n
    return pairs, charged, targets, nt


def cpu_baseline(prob, seconds):
    """The oracle as it stands, on all host cores and on one core, on random
    target samples of the workload (about `seconds` of sums each)."""
    import oracle
    ctx, tree_s = oracle_context(prob)
    pairs, t, targets, nt = oracle_timed(ctx, tree_s, prob, seconds, 7)
    cores = oracle.num_threads()
    prev = oracle.set_num_threads(1)
    try:
        p1, t1, tg1, nt1 = oracle_timed(ctx, tree_s, prob, 0.5 * seconds, 8, calls=2)
    finally:
        oracle.set_num_threads(prev)
    sample = ("FP64 oracle sums at {tg} random targets ({calls} calls of {nt}; {p} pairs) of the full workload, "
              "plus its tree build of all {n} particles ({tree:.2f} s, charged x targets/n)")
    return {"value": pairs / t, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": sample.format(tg=targets, calls=targets // nt, nt=nt, p=pairs, n=prob.n, tree=tree_s),
            "single_core": {"value": p1 / t1, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                            "sample": sample.format(tg=tg1, calls=tg1 // nt1, nt=nt1, p=p1, n=prob.n, tree=tree_s)}}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, each step the
    oracle's sums at a random target sample of the workload sized so that the
    whole run takes about two minutes, with the tree build of the whole
    workload charged in proportion to the targets of the step."""
    if rank != 0:
        return None
    import oracle
    prob = make_problem(args.workload, args.periodic)
    ctx, tree_s = oracle_context(prob)
    rng = np.random.default_rng(1)
    per_step = min(4.0, max(0.5, 120.0 / (args.warmup + args.steps)))
    nt = oracle_target_count(ctx, prob, per_step, rng)
    samples = [rng.choice(prob.n, nt, replace=False) for _ in range(args.warmup + args.steps)]
    for tg in samples[:args.warmup]:
        oracle_sums(ctx, prob, tg)
    tot_pairs, tot_t = 0, 0.0
    for tg in samples[args.warmup:]:
        t0 = time.perf_counter()
        tot_pairs += oracle_sums(ctx, prob, tg)
        tot_t += time.perf_counter() - t0 + tree_s * nt / prob.n
    value = tot_pairs / tot_t
    ms = 1e3 * tot_t / max(1, args.steps)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(prob, args.layout),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: FP64 oracle sums at {nt} random targets of the workload, plus its "
                                   f"tree build of all {prob.n} particles ({tree_s:.2f} s) charged x {nt}/{prob.n}"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="plummer_gravity",
                    help="plummer_gravity (default: 4,194,304 particles, level 7), grid_helmholtz (64^3), "
                         "uniform_gravity (8,192), grid_helmholtz_128, plummer_gravity_1m, grid_helmholtz_r8")
    ap.add_argument("--layout", default="redundant", choices=["redundant", "indirect", "pairtask", "symmetric"])
    ap.add_argument("--tpl", type=int, default=0)
    ap.add_argument("--tile", type=int, default=64)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--group", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="launch the step's kernels on the stream instead of replaying one captured CUDA graph")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--pattern", action="store_true", help="tabulated-G kernel for grid workloads")
    ap.add_argument("--periodic", action="store_true", help="toroidal neighbourhoods (wrapped boxes)")
    ap.add_argument("--evaluation", default="one-sided", choices=["one-sided", "symmetric"],
                    help="one-sided: every ordered pair is evaluated (the paper's operator); symmetric: each pair "
                         "of box pairs with a box of <= 64 particles is evaluated once for both particles (pattern "
                         "mode, pair tasks and more than two right-hand sides stay one-sided).  The default line "
                         "also reports the symmetric evaluation of a Helmholtz workload")
    ap.add_argument("--batched-only", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-arms", action="store_true",
                    help="skip the other target-owned layout on the same workload")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 64^3 Helmholtz object (and, for a Helmholtz workload, the symmetric and "
                         "pipelined objects)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return

    import torch
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2511_21535_gb300 import build as cuda_build
    cuda_build.build()
    dev = torch.device("cuda", local_rank)
    if args.batched_only:
        from paper_2511_21535_gb300 import p2p
        pipes = p2p.measure_pipes()
        print(json.dumps(batched_vs_plain(dev, 10, pipes, pipes["sm_mhz"] or 2070.0)))
        return
    res, prob, pipes, clk = run_gpu(args, rank, world, local_rank)
    f_mhz = res["clocks"]["sm_mhz"] or pipes["sm_mhz"] or 2070.0
    try:
        if not args.no_secondary and prob.name != "grid_helmholtz" and not args.pattern:
            res["grid_helmholtz_64"] = grid_secondary(args, dev, pipes, clk, min(max(args.steps, 50), 300))
        elif (prob.kind == "helmholtz" and prob.nrhs <= 2 and args.evaluation == "one-sided" and not args.pattern
              and args.layout in ("redundant", "indirect") and not args.no_secondary):
            res["symmetric"] = evaluation_variant(prob, args.layout, dev, 100, res["roofline"]["peak"] * 1e9)
            res["pipelined"] = pipelined_batches(prob, args.layout, dev, min(max(args.steps, 20), 400))
        if not args.no_batched:
            res["batched"] = batched_vs_plain(dev, 10, pipes, f_mhz)
            res["adjoint"] = dbim_forward_adjoint(dev, 10, pipes, f_mhz)
    finally:
        clk.__exit__(None, None, None)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()

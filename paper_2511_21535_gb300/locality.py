"""The paper's speedup model (Section 3) applied to this library's layouts.

Propositions 1-4 and Theory 1 predict the speedup of a restructured P2P
operator from its components (Eq. 2: collect, transfer, compute, update),
each weighted by its share of the baseline's time (Eq. 4-6).  The compute
speedup is complexity x locality x kernel-launch (Eq. 9); locality comes
from Definition 1: per worker, D = non-adjacent memory blocks it reads and V
= the data volume, compared with the cache capacity C (Eq. 10 when the
restructured volume fits, Eq. 11 when it does not).  Collect and update
follow Conjecture 1 (Eq. 7: complexity ratio x volume ratio), transfer
Proposition 4 (Eq. 8: volume ratio).

Here the baseline is the indirect ("Indexing") layout and the restructured
versions are the redundant per-box streams and the pair tasks.  The counts
are exact for a given tree (no fitted functions):

  worker        one work item = one target box (and its neighbour ranges);
                a pair task for the pair-task layout
  D_indirect    maximal runs of consecutive box indices in b's neighbour list
                (consecutive boxes are adjacent in the box-ordered array)
  D_redundant   2: the box's stream and its targets in the box-ordered array
  D_pairtask    1: the task block holds targets and sources
  V             bytes the kernel reads over the whole operator (its footprint)

Definition 1 speaks of "a thread" while Table 5 counts whole-operator
volumes, so two readings are evaluated side by side:
  A (Table 5)   D per worker, V = the operator's footprint, C = L2;
  B (per worker) D and V both per worker (the bytes one work item streams),
                C = the on-chip memory of one SM (where a worker's tiles live).

Measured speedups come from CUDA events around the same phases.  The model
is meant to rank configurations (the paper reports it predicts about 1.8x
too high on average while following the trend), so the comparison reports
both the ratio and the rank agreement.

Run ``python -m paper_2511_21535_gb300.locality`` on a GPU for the sweep.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

LAYOUTS = ("indirect", "redundant", "pairtask")


# ---------------------------------------------------------------------------
# counts (host logic over the tree arrays)
# ---------------------------------------------------------------------------

def runs_per_box(nbr_start: np.ndarray, nbr_idx: np.ndarray) -> np.ndarray:
    """Maximal runs of consecutive indices in each box's (ascending) neighbour list."""
    ns = np.asarray(nbr_start, np.int64)
    ni = np.asarray(nbr_idx, np.int64)
    B = ns.shape[0] - 1
    if ni.size == 0:
        return np.zeros(B, np.int64)
    first = np.zeros(ni.size, bool)
    first[ns[:-1][np.diff(ns) > 0]] = True
    brk = np.ones(ni.size, bool)
    brk[1:] = ni[1:] != ni[:-1] + 1
    start = first | brk
    box_of = np.repeat(np.arange(B), np.diff(ns))
    return np.bincount(box_of, weights=start, minlength=B).astype(np.int64)


def tree_stats(box_start, nbr_start, nbr_idx, rec_bytes: int, out_bytes: int) -> dict:
    """Exact sizes of one tree: n, B, E, S = sum_b S_b, pairs, dispersions, volumes (bytes)."""
    bs = np.asarray(box_start, np.int64)
    ns = np.asarray(nbr_start, np.int64)
    ni = np.asarray(nbr_idx, np.int64)
    occ = np.diff(bs)
    B = occ.size
    n = int(bs[-1])
    E = int(ni.size)
    box_of = np.repeat(np.arange(B), np.diff(ns))
    S_b = np.bincount(box_of, weights=occ[ni], minlength=B).astype(np.int64)
    S = int(S_b.sum())
    work = occ * S_b                                   # pair work per box (incl. self pairs)
    runs = runs_per_box(ns, ni)
    wsum = float(work.sum()) if work.sum() else 1.0
    d_ind = float((runs * work).sum() / wsum)
    deg = np.diff(ns)
    # per-worker volumes (reading B), weighted by pair work like D
    vw_ind = float(((S_b * rec_bytes + 8 * deg) * work).sum() / wsum)
    vw_red = float((((S_b + occ) * rec_bytes) * work).sum() / wsum)
    if E:
        occ_b = occ[box_of]
        task_work = occ_b * occ[ni]
        tw = float(task_work.sum()) or 1.0
        vw_pt = float((((occ_b + occ[ni]) * rec_bytes) * task_work).sum() / tw)
    else:
        vw_pt = 0.0
    return {
        "n": n, "boxes": B, "entries": E, "S": S, "pairs": int(work.sum()) - n,
        "mean_occupancy": n / max(B, 1),
        # dispersion per worker, weighted by the worker's pair work
        "D": {"indirect": d_ind, "redundant": 2.0, "pairtask": 1.0},
        "D_indirect_unweighted": float(runs.mean()) if B else 0.0,
        "V_worker": {"indirect": vw_ind, "redundant": vw_red, "pairtask": vw_pt},
        # kernel footprint: what the operator reads
        "V": {"indirect": n * rec_bytes + 4 * (2 * (B + 1) + E),
              "redundant": S * rec_bytes + n * rec_bytes + 4 * 2 * (B + 1),
              "pairtask": 2 * S * rec_bytes + 4 * 3 * (E + 1)},
        # collect: elements written and bytes moved after the tree
        "collect_ops": {"indirect": n + E, "redundant": n + E + S, "pairtask": n + 3 * E + 2 * S},
        "collect_bytes": {"indirect": n * rec_bytes,
                          "redundant": n * rec_bytes + 2 * S * rec_bytes,
                          "pairtask": n * rec_bytes + 4 * S * rec_bytes + 12 * E},
        # update: results written in original order (fused scatter) or partials reduced
        "update_ops": {"indirect": n, "redundant": n, "pairtask": n + S},
        "update_bytes": {"indirect": n * out_bytes, "redundant": n * out_bytes,
                         "pairtask": n * out_bytes + 2 * S * out_bytes},
    }


# ---------------------------------------------------------------------------
# the model (Eq. 4-11)
# ---------------------------------------------------------------------------

def x_locality(D_base: float, D_rest: float, V_base: float, V_rest: float, cache_bytes: float) -> float:
    """Eq. 10 (restructured volume fits the cache) or Eq. 11 (it does not),
    with D' and V' the indexing-to-redundant ratios."""
    Dp = D_base / D_rest
    Vp = V_base / V_rest
    return Dp * Vp if V_rest <= cache_bytes else Vp / Dp


def amdahl(shares: dict, speedups: dict) -> float:
    """Eq. 5/6: 1 / (sum_i share_i / X_i + unmodified share)."""
    s = sum(shares.values())
    rest = max(0.0, 1.0 - s)
    return 1.0 / (sum(shares[k] / speedups[k] for k in shares) + rest)


def predict(st: dict, layout: str, shares: dict, cache_bytes: float, reading: str = "A") -> dict:
    """Predicted component and total speedups of `layout` over the indirect
    baseline; reading "A" (footprint vs L2) or "B" (per-worker volume vs the
    per-SM on-chip memory, passed as cache_bytes)."""
    b = "indirect"
    V = st["V"] if reading == "A" else st["V_worker"]
    x_loc = x_locality(st["D"][b], st["D"][layout], V[b], V[layout], cache_bytes)
    x = {
        # Eq. 7: complexity ratio x volume ratio
        "collect": (st["collect_ops"][b] / st["collect_ops"][layout]) *
                   (st["collect_bytes"][b] / st["collect_bytes"][layout]),
        # Eq. 8: host<->device volume is the same (restructuring runs on the device)
        "transfer": 1.0,
        # Eq. 9: same pair work, one persistent launch each, locality from Eq. 10/11
        "compute": 1.0 * x_loc * 1.0,
        "update": (st["update_ops"][b] / st["update_ops"][layout]) *
                  (st["update_bytes"][b] / st["update_bytes"][layout]),
    }
    return {"x_locality": x_loc, "x": x, "x_p2p": amdahl(shares, x),
            "fits_cache": V[layout] <= cache_bytes}


def spearman(a, b) -> float:
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if a.size < 2:
        return float("nan")
    ra = np.argsort(np.argsort(a)).astype(float)
    rb = np.argsort(np.argsort(b)).astype(float)
    ra -= ra.mean()
    rb -= rb.mean()
    den = math.sqrt(float((ra * ra).sum() * (rb * rb).sum()))
    return float((ra * rb).sum() / den) if den else float("nan")


# ---------------------------------------------------------------------------
# measurement sweep (GPU)
# ---------------------------------------------------------------------------

def _configs():
    from . import workloads as wl

    def uni(n, level, seed=0):
        return lambda: wl.uniform_gravity(n=n, level=level, eps=1e-3, seed=seed)

    def plum(n, level):
        return lambda: wl.plummer_gravity(n=n, level=level, eps=1e-4)

    def grid(e, leaf):
        def make():
            import numpy as np_
            rng = np_.random.default_rng(0)
            pos = wl.grid_points(e)
            q = wl.complex_normal((1, pos.shape[0]), rng)
            level, lo, edge = wl.grid_domain(e, leaf=leaf)
            return wl.Problem(f"grid_helmholtz_{e}_leaf{leaf}", pos, q, level, lo, edge, "helmholtz",
                              k=float(np_.float32(wl.WAVENUMBER)))
        return make

    return [
        ("uniform_1M_L4", uni(1 << 20, 4)), ("uniform_1M_L5", uni(1 << 20, 5)),
        ("uniform_1M_L6", uni(1 << 20, 6)), ("uniform_1M_L7", uni(1 << 20, 7)),
        ("plummer_1M_L5", plum(1 << 20, 5)), ("plummer_1M_L6", plum(1 << 20, 6)),
        ("plummer_1M_L7", plum(1 << 20, 7)),
        ("grid64_leaf2", grid(64, 2)), ("grid64_leaf4", grid(64, 4)), ("grid64_leaf8", grid(64, 8)),
    ]


def _measure(prob, layout, steps, warmup, dev):
    import torch

    from . import p2p
    plan = p2p.Plan(prob.kind, prob.n, prob.level, prob.lo, prob.edge, nrhs=prob.nrhs, layout=layout,
                    timing=True, device=dev)
    pos_h = torch.from_numpy(prob.pos).pin_memory()
    str_h = torch.from_numpy(prob.strength).pin_memory()
    pos = torch.empty_like(pos_h, device=dev)
    strength = torch.empty_like(str_h, device=dev)
    if prob.kind == "gravity":
        outs = [torch.empty(prob.n, device=dev), torch.empty(prob.n, 3, device=dev)]
    else:
        outs = [torch.empty(prob.nrhs, prob.n, dtype=torch.complex64, device=dev)]
    outs_h = [torch.empty_like(o, device="cpu").pin_memory() for o in outs]
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)   # 512 MiB > L2

    def device_step():
        plan.tree_build(pos)
        plan.restructure(pos, strength)
        if prob.kind == "gravity":
            plan.gravity(prob.eps, outs[0], outs[1])
        else:
            plan.helmholtz(prob.k, outs[0])

    pos.copy_(pos_h)
    strength.copy_(str_h)
    for _ in range(warmup):
        flush.zero_()
        device_step()
    torch.cuda.synchronize()
    ph = {k: 0.0 for k in p2p.PHASES}
    dev_ms = e2e_ms = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        device_step()
        b.record()
        b.synchronize()
        dev_ms += a.elapsed_time(b)
        for k, v in plan.timing().items():
            ph[k] += v
        flush.zero_()
        a.record()
        pos.copy_(pos_h, non_blocking=True)
        strength.copy_(str_h, non_blocking=True)
        device_step()
        for o, oh in zip(outs, outs_h):
            oh.copy_(o, non_blocking=True)
        b.record()
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    plan.counters(check=True)
    res = {k: v / steps for k, v in ph.items()}
    res["step"] = dev_ms / steps
    res["e2e"] = e2e_ms / steps
    arrays = None
    if layout == "indirect":
        c = plan.counters()
        B, E = c["n_boxes"], c["n_nbr"]
        arrays = (plan.array("box_start", B + 1).cpu().numpy(), plan.array("nbr_start", B + 1).cpu().numpy(),
                  plan.array("nbr_idx", E).cpu().numpy())
    del plan
    return res, arrays


def sweep(steps: int = 10, warmup: int = 3, names=None, device=None) -> dict:
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", 0)
    props = torch.cuda.get_device_properties(dev)
    cache = float(props.L2_cache_size)
    onchip = float(getattr(props, "shared_memory_per_multiprocessor", 228 * 1024))
    rows = []
    for name, make in _configs():
        if names and name not in names:
            continue
        prob = make()
        meas = {}
        arrays = None
        for layout in LAYOUTS:
            meas[layout], arr = _measure(prob, layout, steps, warmup, dev)
            arrays = arrays or arr
        rec_bytes = 16 if prob.kind == "gravity" else 16 * (1 + (prob.nrhs + 1) // 2)
        out_bytes = 16 if prob.kind == "gravity" else 8 * prob.nrhs
        st = tree_stats(*arrays, rec_bytes=rec_bytes, out_bytes=out_bytes)
        base = meas["indirect"]
        T = base["e2e"]
        shares = {"collect": (base["tree"] + base["restructure"]) / T,
                  "transfer": max(0.0, T - base["step"]) / T,
                  "compute": base["kernel"] / T,
                  "update": max(0.0, base["operator"] - base["kernel"]) / T}
        for layout in LAYOUTS[1:]:
            pr = predict(st, layout, shares, cache)
            pb = predict(st, layout, shares, onchip, reading="B")
            m = meas[layout]
            rows.append({
                "config": name, "layout": layout, "n": st["n"], "boxes": st["boxes"],
                "mean_occupancy": round(st["mean_occupancy"], 2),
                "D_indirect": round(st["D"]["indirect"], 3), "D_layout": st["D"][layout],
                "V_indirect_MB": round(st["V"]["indirect"] / 1e6, 2),
                "V_layout_MB": round(st["V"][layout] / 1e6, 2), "C_MB": round(cache / 1e6, 1),
                "fits_cache": pr["fits_cache"],
                "pred_x_compute": pr["x"]["compute"], "meas_x_kernel": base["kernel"] / m["kernel"],
                "pred_x_p2p": pr["x_p2p"], "meas_x_e2e": base["e2e"] / m["e2e"],
                "Vw_indirect_KB": round(st["V_worker"]["indirect"] / 1e3, 2),
                "Vw_layout_KB": round(st["V_worker"][layout] / 1e3, 2), "C_sm_KB": round(onchip / 1e3, 1),
                "B_fits": pb["fits_cache"], "predB_x_compute": pb["x"]["compute"], "predB_x_p2p": pb["x_p2p"],
                "shares": {k: round(v, 4) for k, v in shares.items()},
                "ms": {"indirect": {k: round(v, 4) for k, v in base.items()},
                       layout: {k: round(v, 4) for k, v in m.items()}},
            })
    summary = {}
    for layout in LAYOUTS[1:]:
        rs = [r for r in rows if r["layout"] == layout]
        if not rs:
            continue
        pk = [r["pred_x_compute"] for r in rs]
        mk = [r["meas_x_kernel"] for r in rs]
        pe = [r["pred_x_p2p"] for r in rs]
        me = [r["meas_x_e2e"] for r in rs]
        pkb = [r["predB_x_compute"] for r in rs]
        peb = [r["predB_x_p2p"] for r in rs]
        summary[layout] = {
            "spearman_kernel": spearman(pk, mk), "spearman_e2e": spearman(pe, me),
            "mean_pred_over_meas_kernel": float(np.mean(np.array(pk) / np.array(mk))),
            "mean_pred_over_meas_e2e": float(np.mean(np.array(pe) / np.array(me))),
            "B_spearman_kernel": spearman(pkb, mk), "B_spearman_e2e": spearman(peb, me),
            "B_mean_pred_over_meas_kernel": float(np.mean(np.array(pkb) / np.array(mk))),
            "B_mean_pred_over_meas_e2e": float(np.mean(np.array(peb) / np.array(me))),
        }
    return {"cache_bytes": cache, "rows": rows, "summary": summary}


def to_markdown(res: dict) -> str:
    lines = ["| config | layout | occ | D_ind | D | A: V_ind MB | A: V MB | A fits L2 | A: pred X_kernel "
             "| B: Vw_ind KB | B: Vw KB | B fits SM | B: pred X_kernel | meas X_kernel | A: pred X_e2e "
             "| B: pred X_e2e | meas X_e2e |",
             "|---|---|---|---|---|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for r in res["rows"]:
        lines.append(f"| {r['config']} | {r['layout']} | {r['mean_occupancy']} | {r['D_indirect']} | {r['D_layout']} "
                     f"| {r['V_indirect_MB']} | {r['V_layout_MB']} | {'yes' if r['fits_cache'] else 'no'} "
                     f"| {r['pred_x_compute']:.3f} | {r['Vw_indirect_KB']} | {r['Vw_layout_KB']} "
                     f"| {'yes' if r['B_fits'] else 'no'} | {r['predB_x_compute']:.3f} | {r['meas_x_kernel']:.3f} "
                     f"| {r['pred_x_p2p']:.3f} | {r['predB_x_p2p']:.3f} | {r['meas_x_e2e']:.3f} |")
    lines.append("")
    for layout, s in res["summary"].items():
        lines.append(f"- {layout}, reading A: Spearman(pred, meas) kernel {s['spearman_kernel']:.2f}, "
                     f"end-to-end {s['spearman_e2e']:.2f}; mean pred/meas kernel "
                     f"{s['mean_pred_over_meas_kernel']:.3f}, end-to-end {s['mean_pred_over_meas_e2e']:.3f}")
        lines.append(f"- {layout}, reading B: Spearman(pred, meas) kernel {s['B_spearman_kernel']:.2f}, "
                     f"end-to-end {s['B_spearman_e2e']:.2f}; mean pred/meas kernel "
                     f"{s['B_mean_pred_over_meas_kernel']:.3f}, end-to-end {s['B_mean_pred_over_meas_e2e']:.3f}")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description="locality-model check: predicted vs measured layout speedups")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--configs", nargs="*", default=None)
    ap.add_argument("--json", default=None, help="also write the full result as JSON here")
    args = ap.parse_args()
    res = sweep(args.steps, args.warmup, args.configs)
    if args.json:
        with open(args.json, "w") as f:
            json.dump(res, f, indent=1)
    print(to_markdown(res))


if __name__ == "__main__":
    main()

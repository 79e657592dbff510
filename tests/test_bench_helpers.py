"""Host logic of bench.py (no GPU): kernel naming, the DRAM-traffic lookup and its
staleness guard, the clock-sample summary, and the workload configs."""
import hashlib
import json
import os

import bench


def test_kernel_names():
    assert bench.kernel_name("helmholtz", False, tile2d=True) == "k_helmtile"
    assert bench.kernel_name("helmholtz", False) == "k_helmholtz"
    assert bench.kernel_name("helmholtz", False, tile2d=True, nrhs=8) == "k_helmplanar"
    assert bench.kernel_name("helmholtz", False, tile2d=False, nrhs=4) == "k_helmplanar"
    assert bench.kernel_name("helmholtz", True, tile2d=True) == "k_helmsym"
    assert bench.kernel_name("helmholtz", False, pattern=True, tile2d=True) == "k_helmholtz_pattern"
    assert bench.kernel_name("gravity", False, tile2d=True) == "k_gravity_pk"
    assert bench.kernel_name("gravity", True, tile2d=True) == "k_gravity"


def test_traffic_lookup_matches_workload_and_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2511_21535_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("one")
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256(b"one").hexdigest()[:16]
    rec = {"k_x": {"workload": "w", "layout": "redundant", "n": 10, "source_files": ["a.cuh"], "source_hash": h,
                   "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k_x", "w", "redundant", 10, False) == 123
    assert bench.kernel_traffic("k_x", "w", "indirect", 10, False) is None      # other layout
    assert bench.kernel_traffic("k_x", "w", "redundant", 11, False) is None     # other size
    assert bench.kernel_traffic("k_x", "w", "redundant", 10, True) is None      # other evaluation
    assert bench.kernel_traffic("k_y", "w", "redundant", 10, False) is None     # no record
    (csrc / "a.cuh").write_text("two")                                           # kernel changed since capture
    assert bench.kernel_traffic("k_x", "w", "redundant", 10, False) is None
    # one record per layout of the same kernel
    (csrc / "a.cuh").write_text("one")
    rec["k_x"] = [rec["k_x"], dict(rec["k_x"], layout="indirect", dram_bytes_per_launch=45)]
    (tmp_path / "profiles" / "kernel_traffic.json").write_text(json.dumps(rec))
    assert bench.kernel_traffic("k_x", "w", "redundant", 10, False) == 123
    assert bench.kernel_traffic("k_x", "w", "indirect", 10, False) == 45
    assert bench.kernel_traffic("k_x", "w", "pairtask", 10, False) is None


def test_committed_traffic_records_are_well_formed():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "kernel_traffic.json")))
    for name, entry in d.items():
        assert name.startswith("k_")
        keys = set()
        for rec in bench.traffic_records(entry):
            assert rec["dram_bytes_per_launch"] > 0
            assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]
            for f in rec["source_files"]:
                assert os.path.exists(os.path.join(bench.ROOT, "paper_2511_21535_gb300", "csrc", f))
            key = (rec["workload"], rec["layout"], bool(rec.get("symmetric", False)), rec.get("n"))
            assert key not in keys   # one record per workload, layout and evaluation
            keys.add(key)


def test_clock_summary():
    cs = bench.ClockSampler(0)
    row = "2026/01/01 00:00:00.000, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"
    cs.lines = [(10.0 + 0.1 * i, row.format(sm=2070 if i != 3 else 1800, cap="Active" if i == 4 else "Not Active"))
                for i in range(10)]
    s = cs.summary(10.0, 11.0)
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]
    assert s["window"] == "timed" and s["samples"] == 10
    far = cs.summary(100.0, 100.1)
    assert far["window"] == "nearest to the timed region" and far["samples"] == 3
    empty = bench.ClockSampler(0).summary(0.0, 1.0)
    assert empty["reasons"] == ["unsampled"]


def test_workload_configs_name_the_workloads():
    for name, kind in (("grid_helmholtz", "helmholtz"), ("uniform_gravity", "gravity"),
                       ("grid_helmholtz_r8", "helmholtz")):
        prob = bench.make_problem(name)
        cfg = bench.workload_config(prob, "redundant")
        assert cfg["kernel"] == kind and cfg["n"] == prob.n and cfg["layout"] == "redundant"
        assert "l2" in cfg and cfg["inputs"] == "seeded synthetic"

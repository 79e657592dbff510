"""Autotuner cache (host logic): keys, round trip, invalidation by kernel build."""
import json

from paper_2511_21535_gb300 import tune_cache as tc


def test_shape_class_quantises():
    a = tc.shape_class([4096, 13824, 262144], 8, True)
    b = tc.shape_class([4096, 13824, 262000], 8, True)
    assert a == b and a.startswith("i3-") and a.endswith("-r8-pair")
    assert tc.shape_class([4096] * 3, 8, True) != a
    assert tc.shape_class([4096, 13824, 262144], 8, False) != a
    assert tc.shape_class([4096, 13824, 262144], 4, True) != a


def test_round_trip_and_atomic_file(tmp_path):
    cache = tc.TuneCache(str(tmp_path / "sub" / "autotune.json"))
    key = tc.TuneCache.key("GPU X", "i2-n2^10-max2^9-r1-fwd")
    assert cache.get(key) is None
    val = {"layout": "indirect", "targets_per_lane": 2, "tile": 64, "warps_per_item": 1, "ms": 1.5}
    cache.put(key, val)
    assert cache.get(key) == val
    other = tc.TuneCache.key("GPU Y", "i2-n2^10-max2^9-r1-fwd")
    cache.put(other, dict(val, tile=32))
    assert cache.get(key) == val and cache.get(other)["tile"] == 32
    data = json.load(open(cache.path))
    assert set(data) == {key, other}
    assert not [p for p in (tmp_path / "sub").iterdir() if p.name.startswith(".autotune.")]


def test_kernel_build_is_part_of_the_key(monkeypatch, tmp_path):
    cache = tc.TuneCache(str(tmp_path / "a.json"))
    k1 = tc.TuneCache.key("GPU", "s")
    cache.put(k1, {"layout": "redundant", "targets_per_lane": 1, "tile": 64, "warps_per_item": 4, "ms": 1.0})
    monkeypatch.setattr(tc, "_version", "0123456789abcdef")
    k2 = tc.TuneCache.key("GPU", "s")
    assert k2 != k1 and cache.get(k2) is None
    assert len(tc.kernel_version()) == 16


def test_corrupt_file_reads_as_empty(tmp_path):
    p = tmp_path / "c.json"
    p.write_text("{not json")
    cache = tc.TuneCache(str(p))
    assert cache.get("x") is None
    cache.put("x", {"tile": 64})
    assert cache.get("x") == {"tile": 64}


def test_default_path_honours_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("P2P_GB300_TUNE_CACHE", str(tmp_path / "t.json"))
    assert tc.TuneCache().path == str(tmp_path / "t.json")

"""Host logic of the speedup model (Section 3, Eq. 4-11): counts against
brute force on trees the oracle builds, and the model's algebra on cases
with known answers."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_21535_gb300 import locality as lm
from paper_2511_21535_gb300 import workloads as wl


def brute_runs(nbr_start, nbr_idx):
    out = []
    for b in range(len(nbr_start) - 1):
        lst = list(nbr_idx[nbr_start[b]:nbr_start[b + 1]])
        r = 0
        for i, c in enumerate(lst):
            if i == 0 or c != lst[i - 1] + 1:
                r += 1
        out.append(r)
    return np.array(out)


@pytest.mark.parametrize("make", [lambda: wl.uniform_gravity(n=3000, level=3, seed=1),
                                  lambda: wl.grid_helmholtz(edge_points=16),
                                  lambda: wl.plummer_gravity(n=5000, level=4, eps=1e-3, seed=2)])
def test_runs_and_sizes_match_brute_force(make):
    prob = make()
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    runs = lm.runs_per_box(t["nbr_start"], t["nbr_idx"])
    np.testing.assert_array_equal(runs, brute_runs(t["nbr_start"], t["nbr_idx"]))
    st = lm.tree_stats(t["box_start"], t["nbr_start"], t["nbr_idx"], rec_bytes=16, out_bytes=16)
    assert st["n"] == prob.n and st["boxes"] == t["n_boxes"] and st["entries"] == t["n_nbr"]
    # S = sum_b S_b = sum_c n_c |N(c)| (the neighbour relation is symmetric)
    occ = np.diff(t["box_start"])
    assert st["S"] == int((occ * np.diff(t["nbr_start"])).sum())
    assert st["S"] == oracle.redundant(t, gather=False)["total"]
    assert st["pairs"] == oracle.pair_count(prob.pos, prob.level, prob.lo, prob.edge)
    assert 1.0 <= st["D"]["indirect"] <= 27.0


def test_full_grid_dispersion():
    # 16^3 lattice, 4^3 boxes: an interior box's 27 neighbours in Morton order
    # form at most 27 runs and at least 9 (x-pairs can merge)
    prob = wl.grid_helmholtz(edge_points=16)
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    runs = lm.runs_per_box(t["nbr_start"], t["nbr_idx"])
    assert runs.max() <= 27 and runs.min() >= 1
    assert lm.runs_per_box(np.array([0, 3]), np.array([4, 5, 6]))[0] == 1
    assert lm.runs_per_box(np.array([0, 3, 5]), np.array([1, 3, 4, 7, 9])).tolist() == [2, 2]


def test_locality_branches():
    # Eq. 10 when the restructured volume fits the cache, Eq. 11 otherwise
    assert lm.x_locality(8.0, 2.0, 1.0, 4.0, cache_bytes=10.0) == pytest.approx(4.0 * 0.25)
    assert lm.x_locality(8.0, 2.0, 1.0, 40.0, cache_bytes=10.0) == pytest.approx((1 / 40) / 4.0)


def test_amdahl_special_cases():
    shares = {"collect": 0.2, "transfer": 0.1, "compute": 0.6, "update": 0.1}
    one = {k: 1.0 for k in shares}
    assert lm.amdahl(shares, one) == pytest.approx(1.0)
    # only compute changes: Eq. 4
    x = dict(one, compute=3.0)
    assert lm.amdahl(shares, x) == pytest.approx(1.0 / (0.6 / 3.0 + 0.4))
    # the total lies between the smallest and largest component speedup
    x = {"collect": 0.5, "transfer": 1.0, "compute": 2.0, "update": 0.8}
    assert 0.5 <= lm.amdahl(shares, x) <= 2.0


def test_prediction_of_the_baseline_is_one():
    prob = wl.uniform_gravity(n=2000, level=3, seed=3)
    t = oracle.tree(prob.pos, prob.level, prob.lo, prob.edge)
    st = lm.tree_stats(t["box_start"], t["nbr_start"], t["nbr_idx"], rec_bytes=16, out_bytes=16)
    shares = {"collect": 0.3, "transfer": 0.2, "compute": 0.5, "update": 0.0}
    pr = lm.predict(st, "indirect", shares, cache_bytes=1e9)
    assert pr["x_p2p"] == pytest.approx(1.0)
    red = lm.predict(st, "redundant", shares, cache_bytes=1e9)
    # more data moved while collecting: the collect component cannot speed up
    assert red["x"]["collect"] < 1.0
    assert red["fits_cache"]


def test_spearman():
    assert lm.spearman([1, 2, 3, 4], [10, 20, 30, 40]) == pytest.approx(1.0)
    assert lm.spearman([1, 2, 3, 4], [4, 3, 2, 1]) == pytest.approx(-1.0)
    assert math.isnan(lm.spearman([1], [2]))

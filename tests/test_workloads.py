"""The synthetic inputs (seed 0) have the sizes the design notes and the bench
configs state: particle counts, boxes, occupancies and exact pair counts, the
latter counted by the oracle."""
import numpy as np

import oracle
from paper_2511_21535_gb300 import workloads as wl


def test_uniform_gravity_8192():
    p = wl.uniform_gravity()
    assert p.n == 8192 and p.level == 3 and np.isclose(p.eps, 1e-3)
    assert oracle.pair_count(p.pos, p.level, p.lo, p.edge) == 2_732_724
    assert p.strength.min() >= 0.5 and p.strength.max() < 1.5


def test_grid_helmholtz_64():
    p = wl.grid_helmholtz()
    assert p.n == 64 ** 3 and p.level == 4 and p.nrhs == 1
    assert np.isclose(p.k, 2 * np.pi)
    assert oracle.pair_count(p.pos, p.level, p.lo, p.edge) == 398_426_112


def test_plummer_gravity_4m():
    p = wl.plummer_gravity()
    assert p.n == 4_194_304 and p.level == 7
    inside = np.all((p.pos >= 0.0) & (p.pos < 1.0), axis=1)
    assert inside.all()
    t = oracle.tree(p.pos, p.level, p.lo, p.edge)
    assert t["n_boxes"] == 605_596
    assert int(np.diff(t["box_start"]).max()) == 3_336
    assert oracle.pair_count(p.pos, p.level, p.lo, p.edge) == 63_033_853_198


def test_batched_helmholtz_64_instances():
    probs = wl.batched_helmholtz()
    edges = [round(p.n ** (1 / 3)) for p in probs]
    assert len(probs) == 64 and sum(p.n for p in probs) == 5_981_696
    assert [edges.count(e) for e in (16, 24, 32, 48, 64)] == [14, 9, 11, 16, 14]
    assert all(p.nrhs == 8 for p in probs)
    assert sum(oracle.pair_count(p.pos, p.level, p.lo, p.edge) for p in probs) == 8_839_576_064

"""Pins for the FP64 oracle: checks against facts that do not come from the
oracle itself (hand-derived closed forms, brute-force O(N^2) sums written
independently here, counting identities, invariants of the operator).

CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2511_21535_gb300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


# ---------------------------------------------------------------------------
# helpers written independently of the oracle (brute force)
# ---------------------------------------------------------------------------

def brute_cells_unit(pos, level):
    """Cells in the unit cube: floor(x * 2^L) is exact for a power of two."""
    c = np.floor(pos.astype(np.float64) * (1 << level)).astype(np.int64)
    return np.minimum(c, (1 << level) - 1)


def brute_mask(cells):
    """near[i, j] = boxes of i and j at Chebyshev distance <= 1."""
    d = np.abs(cells[:, None, :] - cells[None, :, :]).max(axis=2)
    return d <= 1


def brute_gravity(pos, mass, cells, eps):
    x = pos.astype(np.float64)
    d = x[None, :, :] - x[:, None, :]                    # d[i, j] = x_j - x_i
    r2 = (d ** 2).sum(axis=2) + float(eps) ** 2
    w = brute_mask(cells)
    np.fill_diagonal(w, False)
    m = np.where(w, mass.astype(np.float64)[None, :], 0.0)
    inv = 1.0 / np.sqrt(np.where(w, r2, 1.0))
    phi = -(m * inv).sum(axis=1)
    acc = ((m * inv ** 3)[:, :, None] * d).sum(axis=1)
    return phi, acc


def brute_helmholtz(pos, q, cells, k):
    x = pos.astype(np.float64)
    d = x[None, :, :] - x[:, None, :]
    r = np.sqrt((d ** 2).sum(axis=2))
    w = brute_mask(cells)
    np.fill_diagonal(w, False)
    rs = np.where(w, r, 1.0)
    g = np.where(w, np.exp(1j * float(k) * rs) / (4.0 * math.pi * rs), 0.0)
    return (g @ q.astype(np.complex128).T).T


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# Morton keys and boxing
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLDEN["morton"]["cases"])
def test_morton_hand_values(case):
    cx, cy, cz = case["cell"]
    assert oracle.morton(cx, cy, cz, case["level"]) == case["key"]
    assert oracle.unmorton(case["key"], case["level"]) == (cx, cy, cz)


def test_cells_unit_cube_exact():
    rng = np.random.default_rng(5)
    pos = rng.random((20000, 3), dtype=np.float32)
    for level in (1, 3, 7, 10):
        cell, key = oracle.cells(pos, level, (0, 0, 0), 1.0)
        np.testing.assert_array_equal(cell, brute_cells_unit(pos, level))


def test_cells_domain_edges():
    # the upper face belongs to the last cell; outside points are rejected
    cell, _ = oracle.cells(np.array([[1.0, 0.0, 0.999999]], np.float32), 2, (0, 0, 0), 1.0)
    assert cell.tolist() == [[3, 0, 3]]
    for bad in ([-1e-7, 0.5, 0.5], [0.5, 1.0000001, 0.5], [np.nan, 0.5, 0.5], [0.5, 0.5, np.inf]):
        with pytest.raises(RuntimeError):
            oracle.cells(np.array([bad], np.float32), 2, (0, 0, 0), 1.0)


def test_cells_grid_domain_centres():
    # grid points sit half a spacing inside their leaf box: box = index // 4
    for e in (16, 24, 64):
        level, lo, edge = wl.grid_domain(e)
        pos = wl.grid_points(e)
        cell, _ = oracle.cells(pos, level, lo, edge)
        idx = np.arange(e ** 3)
        ix, iy, iz = idx % e, (idx // e) % e, idx // (e * e)
        np.testing.assert_array_equal(cell, np.stack([ix // 4, iy // 4, iz // 4], axis=1))


# ---------------------------------------------------------------------------
# tree structure
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,level", [(1, 2), (7, 1), (500, 2), (3000, 3), (2000, 5)])
def test_tree_bruteforce(n, level):
    rng = np.random.default_rng(n + level)
    pos = rng.random((n, 3), dtype=np.float32)
    t = oracle.tree(pos, level, (0, 0, 0), 1.0)
    cells = brute_cells_unit(pos, level)
    keys = np.array([oracle.morton(*c, level) for c in cells], np.int64)
    perm = t["perm"]
    assert sorted(perm.tolist()) == list(range(n))
    sk = keys[perm]
    assert np.all(np.diff(sk) >= 0)
    ties = np.diff(sk) == 0
    assert np.all(np.diff(perm)[ties] > 0)                  # stable: ties by original index
    ub = np.unique(keys)
    np.testing.assert_array_equal(t["box_key"], ub)
    np.testing.assert_array_equal(np.diff(t["box_start"]), np.array([np.sum(keys == k) for k in ub]))
    bc = np.array([oracle.unmorton(int(k), level) for k in ub])
    near = np.abs(bc[:, None, :] - bc[None, :, :]).max(axis=2) <= 1
    for b in range(len(ub)):
        lst = t["nbr_idx"][t["nbr_start"][b]:t["nbr_start"][b + 1]]
        assert lst.tolist() == np.nonzero(near[b])[0].tolist()   # exactly the E2 set, ascending


def test_regular_grid_neighbour_counts():
    for case in GOLDEN["grid_counts"]["cases"][:2]:
        e, B = case["edge_points"], case["boxes_per_edge"]
        level, lo, edge = wl.grid_domain(e)
        t = oracle.tree(wl.grid_points(e), level, lo, edge)
        cnt = np.diff(t["nbr_start"])
        assert t["n_boxes"] == B ** 3
        assert t["n_nbr"] == case["n_nbr"] == (3 * B - 2) ** 3
        vals, mult = np.unique(cnt, return_counts=True)
        expect = {8: 8, 12: 12 * (B - 2), 18: 6 * (B - 2) ** 2, 27: (B - 2) ** 3}
        assert dict(zip(vals.tolist(), mult.tolist())) == {k: v for k, v in expect.items() if v}
        assert np.all(np.diff(t["box_start"]) == 64)


def test_pair_count_closed_forms():
    for case in GOLDEN["grid_counts"]["cases"]:
        e = case["edge_points"]
        level, lo, edge = wl.grid_domain(e)
        assert oracle.pair_count(wl.grid_points(e), level, lo, edge) == case["pairs"]


def test_redundant_identities():
    p = wl.uniform_gravity(n=3000, level=3)
    t = oracle.tree(p.pos, p.level, p.lo, p.edge)
    r = oracle.redundant(t)
    bs, ns, ni = t["box_start"], t["nbr_start"], t["nbr_idx"]
    occ = np.diff(bs)
    deg = np.diff(ns)
    S = np.array([occ[ni[ns[b]:ns[b + 1]]].sum() for b in range(t["n_boxes"])])
    assert r["total"] == S.sum() == (occ * deg).sum()             # sum S_b = sum_c n_c |N(c)|
    np.testing.assert_array_equal(np.diff(r["red_start"]), S)
    # each sorted source appears |N(box)| times
    box_of_sorted = np.repeat(np.arange(t["n_boxes"]), occ)
    np.testing.assert_array_equal(np.bincount(r["gather_idx"], minlength=3000), deg[box_of_sorted])
    # the self segment holds the box's own particles in order
    for b in range(t["n_boxes"]):
        s0 = r["red_start"][b] + r["red_self"][b]
        np.testing.assert_array_equal(r["gather_idx"][s0:s0 + occ[b]], np.arange(bs[b], bs[b + 1]))
    # pairs = sum n_b S_b - n
    assert oracle.pair_count(p.pos, p.level, p.lo, p.edge) == int((occ * S).sum()) - 3000


def decode_morton(keys, level):
    """Cells of Morton keys, de-interleaved bit by bit (x from key bit 3b, y 3b+1, z 3b+2)."""
    keys = np.asarray(keys, np.int64)
    c = np.zeros((keys.size, 3), np.int64)
    for b in range(level):
        for a in range(3):
            c[:, a] |= ((keys >> (3 * b + a)) & 1) << b
    return c


@pytest.mark.parametrize("n,level,seed", [(3000, 3, 1), (4000, 4, 2)])
def test_redundant_stream_order_bruteforce(n, level, seed):
    """The redundant stream of each target box, rebuilt from the box keys alone:
    the sorted particles of every box at Chebyshev cell distance <= 1 (found by
    testing all box pairs), boxes in ascending Morton key, each box's particles
    in sorted order; red_self is the offset of the box's own block.  Uneven
    occupancies (a clustered sphere) so that a wrong neighbour order changes
    the stream."""
    p = wl.plummer_gravity(n=n, level=level, eps=1e-3, seed=seed)
    t = oracle.tree(p.pos, p.level, p.lo, p.edge)
    r = oracle.redundant(t)
    keys, bs = t["box_key"].astype(np.int64), t["box_start"]
    assert np.all(np.diff(keys) > 0)
    cell = decode_morton(keys, level)
    occ = np.diff(bs)
    assert len(np.unique(occ)) > 3
    pos = 0
    for b in range(t["n_boxes"]):
        near = np.nonzero(np.abs(cell - cell[b]).max(axis=1) <= 1)[0]     # ascending index = ascending key
        expect = np.concatenate([np.arange(bs[c], bs[c + 1]) for c in near])
        assert r["red_start"][b] == pos
        np.testing.assert_array_equal(r["gather_idx"][pos:pos + expect.size], expect)
        own = int(np.nonzero(near == b)[0][0])
        assert r["red_self"][b] == occ[near[:own]].sum()
        pos += expect.size
    assert r["total"] == pos == r["red_start"][-1]


def f32_cells(pos, level, lo, edge):
    """The boxing rule in numpy float32 (each operation rounded to float32):
    s = 2^L / edge, u = (x - lo) * s, cell = min(floor(u), 2^L - 1)."""
    f = np.float32
    s = f(f(1 << level) / f(edge))
    u = (np.asarray(pos, f) - np.asarray(lo, f)) * s
    assert u.dtype == np.float32
    return np.minimum(np.floor(u).astype(np.int64), (1 << level) - 1), u


def test_cells_offset_domain_near_faces():
    """A shifted domain with a non-dyadic edge (lo != 0, edge = 2.7): points on
    and within a few float32 ulps of every cell face, plus random points; the
    oracle's cells equal the float32 rule evaluated by numpy, and the points
    sit close enough to the faces that evaluating the same rule in float64
    would box some of them differently."""
    level, edge = 5, 2.7
    lo = np.array([-0.37, 1.25, 3.1], np.float32)
    side = 1 << level
    f = np.float32
    pts = []
    for a in range(3):
        faces = lo[a].astype(np.float64) + np.arange(side + 1) * (float(f(edge)) / side)
        x = faces.astype(np.float32)
        for k in range(-3, 4):
            y = x.copy()
            for _ in range(abs(k)):
                y = np.nextafter(y, np.float32(np.inf if k > 0 else -np.inf))
            pts.append((a, y))
    rng = np.random.default_rng(17)
    base = (lo + rng.random((1, 3), dtype=np.float32) * f(edge)).astype(np.float32)
    rows = []
    for a, y in pts:
        blk = np.repeat(base, y.size, axis=0)
        blk[:, a] = y
        rows.append(blk)
    rows.append((lo + rng.random((5000, 3), dtype=np.float32) * f(edge * 0.999)).astype(np.float32))
    pos = np.concatenate(rows)
    ref, u = f32_cells(pos, level, lo, edge)
    ok = np.all((u >= 0) & (u <= side), axis=1)
    assert ok.sum() > 5000 and (~ok).sum() > 0
    cell, key = oracle.cells(pos[ok], level, lo, edge)
    np.testing.assert_array_equal(cell, ref[ok])
    np.testing.assert_array_equal(decode_morton(key, level), ref[ok])
    u64 = (pos[ok].astype(np.float64) - lo.astype(np.float64)) * (side / float(f(edge)))
    c64 = np.minimum(np.floor(u64).astype(np.int64), side - 1)
    assert np.any(c64 != ref[ok])
    for bad in pos[~ok][:20]:
        with pytest.raises(RuntimeError):
            oracle.cells(bad[None], level, lo, edge)


def test_oracle_calls_are_reentrant():
    """Open and periodic calls running at the same time in two host threads
    (ctypes releases the interpreter lock) give the results of sequential calls."""
    import threading
    p = wl.uniform_gravity(n=6000, level=3, seed=12)
    seq_open = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps)
    seq_per = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps, periodic=True)
    out = {}

    def work(name, periodic):
        res = []
        for _ in range(4):
            res.append(oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps, periodic=periodic))
        out[name] = res

    th = [threading.Thread(target=work, args=("open", False)), threading.Thread(target=work, args=("per", True))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for name, ref in (("open", seq_open), ("per", seq_per)):
        for res in out[name]:
            np.testing.assert_array_equal(res[0], ref[0])
            np.testing.assert_array_equal(res[1], ref[1])
            assert res[2] == ref[2]
    assert seq_per[2] > seq_open[2]


# ---------------------------------------------------------------------------
# sums
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,level,eps", [(400, 1, 1e-3), (1500, 2, 1e-3), (2000, 3, 0.0)])
def test_gravity_vs_bruteforce(n, level, eps):
    rng = np.random.default_rng(11 + n)
    pos = rng.random((n, 3), dtype=np.float32)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    phi, acc, pairs = oracle.gravity(pos, mass, level, (0, 0, 0), 1.0, eps)
    bphi, bacc = brute_gravity(pos, mass, brute_cells_unit(pos, level), np.float32(eps))
    assert rel_l2(phi, bphi) < 1e-13
    assert rel_l2(acc, bacc) < 1e-13
    w = brute_mask(brute_cells_unit(pos, level))
    assert pairs == int(w.sum()) - n


@pytest.mark.parametrize("n,level,nrhs", [(500, 1, 1), (1800, 2, 3), (2000, 3, 2)])
def test_helmholtz_vs_bruteforce(n, level, nrhs):
    rng = np.random.default_rng(3 + n)
    pos = rng.random((n, 3), dtype=np.float32)
    q = wl.complex_normal((nrhs, n), rng)
    k = np.float32(2 * math.pi * 3.0)
    u, _ = oracle.helmholtz(pos, q, level, (0, 0, 0), 1.0, k)
    bu = brute_helmholtz(pos, q, brute_cells_unit(pos, level), k)
    assert rel_l2(u, bu) < 1e-13


def test_targets_subset_matches_full():
    p = wl.uniform_gravity(n=4000, level=3)
    phi, acc, _ = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps)
    tg = np.array([0, 17, 3999, 1234, 17])
    phi2, acc2, _ = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps, targets=tg)
    np.testing.assert_array_equal(phi2, phi[tg])
    np.testing.assert_array_equal(acc2, acc[tg])


def test_gravity_single_pair_closed_form():
    g = GOLDEN["gravity_pair"]
    pos = np.array(g["pos"], np.float32)
    phi, acc, pairs = oracle.gravity(pos, np.array(g["mass"], np.float32), g["level"],
                                     (0, 0, 0), 1.0, np.float32(g["eps"]))
    np.testing.assert_allclose(phi, g["phi"], rtol=1e-15)
    np.testing.assert_allclose(acc, g["acc"], rtol=1e-15, atol=0)
    assert pairs == 2


def test_helmholtz_single_pair_closed_form():
    g = GOLDEN["helmholtz_pair"]
    pos = np.array(g["pos"], np.float32)
    q = np.array([[complex(*g["q"][0]), complex(*g["q"][1])]], np.complex64)
    k = np.float32(g["k_over_pi"] * math.pi)
    u, _ = oracle.helmholtz(pos, q, g["level"], (0, 0, 0), 1.0, k)
    # k is float32, so the phase is pi/5 to ~1e-7
    np.testing.assert_allclose(u[0, 0], complex(*g["u1"]), rtol=0, atol=2e-7)
    np.testing.assert_allclose(u[0, 1], complex(*g["u2"]), rtol=0, atol=2e-7)


def test_far_pair_contributes_nothing():
    # boxes 0 and 2 along x at level 2 are not neighbours
    pos = np.array([[0.1, 0.1, 0.1], [0.6, 0.1, 0.1]], np.float32)
    phi, acc, pairs = oracle.gravity(pos, np.ones(2, np.float32), 2, (0, 0, 0), 1.0, 1e-3)
    assert pairs == 0 and np.all(phi == 0) and np.all(acc == 0)
    u, pairs = oracle.helmholtz(pos, np.ones((1, 2), np.complex64), 2, (0, 0, 0), 1.0, 1.0)
    assert pairs == 0 and np.all(u == 0)


def test_helmholtz_k0_is_laplace():
    # k = 0: u = sum q/(4 pi r) = -phi/(4 pi) for gravity with eps = 0 and m = q
    p = wl.uniform_gravity(n=3000, level=3)
    u, _ = oracle.helmholtz(p.pos, p.strength.astype(np.complex64)[None, :], p.level, p.lo, p.edge, 0.0)
    phi, _, _ = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, 0.0)
    assert rel_l2(u[0].real, -phi / (4 * math.pi)) < 1e-14
    assert np.all(u[0].imag == 0)


def test_momentum_invariant():
    # neighbour relation symmetric + odd force: sum_i m_i a_i = 0
    for p in (wl.uniform_gravity(n=6000, level=3), wl.plummer_gravity(n=20000, level=4, eps=1e-3)):
        _, acc, _ = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps)
        f = p.strength.astype(np.float64)[:, None] * acc
        assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()


def test_reciprocity_and_linearity():
    # G(r) = G(-r) and a symmetric neighbour relation: P^T = P (bilinear)
    p = wl.grid_helmholtz(edge_points=16, nrhs=2, seed=4)
    a, b = p.strength[0], p.strength[1]
    ua, _ = oracle.helmholtz(p.pos, a[None], p.level, p.lo, p.edge, p.k)
    ub, _ = oracle.helmholtz(p.pos, b[None], p.level, p.lo, p.edge, p.k)
    lhs = np.sum(b.astype(np.complex128) * ua[0])
    rhs = np.sum(a.astype(np.complex128) * ub[0])
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # multi-RHS equals stacked single-RHS results
    uab, _ = oracle.helmholtz(p.pos, p.strength, p.level, p.lo, p.edge, p.k)
    np.testing.assert_array_equal(uab[0], ua[0])
    np.testing.assert_array_equal(uab[1], ub[0])
    # linearity (sources exactly representable so the combination is exact in complex64)
    c = (a.astype(np.complex128) * 2.0 - b.astype(np.complex128)).astype(np.complex64)
    uc, _ = oracle.helmholtz(p.pos, c[None], p.level, p.lo, p.edge, p.k)
    lin = 2.0 * ua[0] - ub[0]
    assert rel_l2(uc[0], lin) < 1e-6   # c is rounded to complex64


def test_grid_translation_invariance():
    # equal unit sources on a regular grid: all interior boxes see the same pattern
    e = 24
    level, lo, edge = wl.grid_domain(e)
    pos = wl.grid_points(e)
    q = np.ones((1, e ** 3), np.complex64)
    u, _ = oracle.helmholtz(pos, q, level, lo, edge, np.float32(2 * math.pi))
    u = u[0].reshape(e, e, e)                     # [iz, iy, ix]
    a = u[4:8, 4:8, 4:8]
    for (z, y, x) in ((8, 8, 8), (4, 12, 8), (12, 4, 16)):
        np.testing.assert_allclose(u[z:z + 4, y:y + 4, x:x + 4], a, rtol=1e-6, atol=0)


# ---------------------------------------------------------------------------
# adjoints: pinned by finite differences of the forward sums and by the
# dot-product identity (not by re-deriving the adjoint formulas)
# ---------------------------------------------------------------------------

def lattice_points(n, level, seed, min_sep=0.04):
    """Points on a 2^-16 lattice, at least min_sep apart and away from box faces,
    so that +-2^-17 perturbations are exact in float32 and keep the tree."""
    rng = np.random.default_rng(seed)
    side = 1 << level
    pts = []
    while len(pts) < n:
        p = rng.uniform(0.05, 0.95, 3)
        cellpos = p * side - np.floor(p * side)
        if np.any(cellpos < 0.01) or np.any(cellpos > 0.99):
            continue
        if pts and np.min(np.linalg.norm(np.array(pts) - p, axis=1)) < min_sep:
            continue
        pts.append(p)
    return (np.round(np.array(pts) * 65536.0) / 65536.0).astype(np.float32)


FD_DELTA = np.float32(2.0 ** -17)


def test_helmholtz_adjoint_dot_product():
    p = wl.grid_helmholtz(edge_points=16, nrhs=2, seed=11)
    rng = np.random.default_rng(12)
    y = wl.complex_normal((2, p.n), rng)
    u, _ = oracle.helmholtz(p.pos, p.strength, p.level, p.lo, p.edge, p.k)
    gq, _ = oracle.helmholtz_adjoint(p.pos, p.strength, y, p.level, p.lo, p.edge, p.k)
    lhs = np.real(np.vdot(y.astype(np.complex128), u))       # Re <y, P q>
    rhs = np.real(np.vdot(gq, p.strength.astype(np.complex128)))   # Re <P^H y, q>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_helmholtz_adjoint_finite_differences(nrhs):
    level, n = 2, 120
    pos = lattice_points(n, level, 21 + nrhs)
    rng = np.random.default_rng(5)
    q = wl.complex_normal((nrhs, n), rng)
    y = wl.complex_normal((nrhs, n), rng)
    k = np.float32(2 * math.pi * 2.0)
    gq, gx = oracle.helmholtz_adjoint(pos, q, y, level, (0, 0, 0), 1.0, k)

    def loss(pp, qq):
        u, _ = oracle.helmholtz(pp, qq, level, (0, 0, 0), 1.0, k)
        return float(np.real(np.sum(np.conj(y.astype(np.complex128)) * u)))

    for i in (0, 7, 55, 119):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += FD_DELTA
            pm[i, a] -= FD_DELTA
            fd = (loss(pp, q) - loss(pm, q)) / (2 * float(FD_DELTA))
            assert abs(fd - gx[i, a]) <= 1e-5 * max(1.0, np.abs(gx).max()), (i, a, fd, gx[i, a])
    # L is linear in q: central differences in Re/Im q are exact up to rounding
    for i in (3, 90):
        for r in range(nrhs):
            for unit in (1.0, 1j):
                qp, qm = q.copy(), q.copy()
                qp[r, i] += np.complex64(0.5 * unit)
                qm[r, i] -= np.complex64(0.5 * unit)
                step = complex(qp[r, i]) - complex(qm[r, i])       # the float32-rounded step
                step = step.real if unit == 1.0 else step.imag
                fd = (loss(pos, qp) - loss(pos, qm)) / step
                ref = gq[r, i].real if unit == 1.0 else gq[r, i].imag
                assert abs(fd - ref) <= 1e-10 * max(1.0, abs(ref))


def test_gravity_adjoint_finite_differences():
    level, n = 2, 150
    pos = lattice_points(n, level, 31)
    rng = np.random.default_rng(6)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    gphi = rng.standard_normal(n).astype(np.float32)
    gacc = rng.standard_normal((n, 3)).astype(np.float32)
    eps = np.float32(0.02)
    gm, gx = oracle.gravity_adjoint(pos, mass, gphi, gacc, level, (0, 0, 0), 1.0, eps)

    def loss(pp, mm):
        phi, acc, _ = oracle.gravity(pp, mm, level, (0, 0, 0), 1.0, eps)
        return float(np.sum(gphi.astype(np.float64) * phi) + np.sum(gacc.astype(np.float64) * acc))

    for i in (0, 9, 77, 149):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += FD_DELTA
            pm[i, a] -= FD_DELTA
            fd = (loss(pp, mass) - loss(pm, mass)) / (2 * float(FD_DELTA))
            assert abs(fd - gx[i, a]) <= 1e-5 * max(1.0, np.abs(gx).max()), (i, a, fd, gx[i, a])
        # linear in m: exact central difference with an exactly representable step
        mp, mm_ = mass.copy(), mass.copy()
        mp[i] += np.float32(0.25)
        mm_[i] -= np.float32(0.25)
        fd = (loss(pos, mp) - loss(pos, mm_)) / 0.5
        assert abs(fd - gm[i]) <= 1e-9 * max(1.0, abs(gm[i]))


# ---------------------------------------------------------------------------
# periodic (toroidal) neighbours
# ---------------------------------------------------------------------------

def brute_periodic(pos, level, edge=1.0):
    """(mask[i, j], image shift of x_j [i, j, 3]) from wrapped cell offsets."""
    side = 1 << level
    cells = brute_cells_unit(pos, level)
    d = cells[None, :, :] - cells[:, None, :]                 # cell_j - cell_i
    dw = np.mod(d + 1, side) - 1                              # wrapped offset
    mask = np.all(np.abs(dw) <= 1, axis=2)
    shift = (dw - d) * (edge / side)
    return mask, shift


def test_periodic_tree_bruteforce():
    level, n = 3, 1500
    pos = np.random.default_rng(41).random((n, 3), dtype=np.float32)
    t = oracle.tree(pos, level, (0, 0, 0), 1.0, periodic=True)
    bc = np.array([oracle.unmorton(int(k), level) for k in t["box_key"]])
    side = 1 << level
    for b in range(t["n_boxes"]):
        lst = t["nbr_idx"][t["nbr_start"][b]:t["nbr_start"][b + 1]]
        img = t["nbr_img"][t["nbr_start"][b]:t["nbr_start"][b + 1]]
        d = bc - bc[b]
        dw = np.mod(d + 1, side) - 1
        near = np.nonzero(np.all(np.abs(dw) <= 1, axis=1))[0]
        assert lst.tolist() == near.tolist()
        o = (dw - d)[lst] // side                                # image multiplier per axis
        np.testing.assert_array_equal(img, (o[:, 0] + 1) + 3 * (o[:, 1] + 1) + 9 * (o[:, 2] + 1))


@pytest.mark.parametrize("level", [2, 3])
def test_periodic_sums_vs_bruteforce(level):
    n = 1200
    rng = np.random.default_rng(43 + level)
    pos = rng.random((n, 3), dtype=np.float32)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    q = wl.complex_normal((2, n), rng)
    eps = np.float32(1e-3)
    mask, shift = brute_periodic(pos, level)
    np.fill_diagonal(mask, False)
    x = pos.astype(np.float64)
    d = x[None, :, :] + shift - x[:, None, :]
    r2 = (d ** 2).sum(axis=2)
    h = np.where(mask, r2 + float(eps) ** 2, 1.0)
    m = np.where(mask, mass.astype(np.float64)[None, :], 0.0)
    bphi = -(m / np.sqrt(h)).sum(axis=1)
    bacc = ((m / h ** 1.5)[:, :, None] * d).sum(axis=1)
    phi, acc, pairs = oracle.gravity(pos, mass, level, (0, 0, 0), 1.0, eps, periodic=True)
    assert rel_l2(phi, bphi) < 1e-13 and rel_l2(acc, bacc) < 1e-13
    assert pairs == int(mask.sum())
    k = np.float32(2 * math.pi * 2)
    r = np.sqrt(np.where(mask, r2, 1.0))
    g = np.where(mask, np.exp(1j * float(k) * r) / (4 * math.pi * r), 0.0)
    bu = (g @ q.astype(np.complex128).T).T
    u, _ = oracle.helmholtz(pos, q, level, (0, 0, 0), 1.0, k, periodic=True)
    assert rel_l2(u, bu) < 1e-13


def test_periodic_pair_across_the_boundary():
    # x = 1/64 and 63/64 at level 2: neighbours only through the wrap, distance 1/32
    pos = np.array([[1 / 64, 0.5, 0.5], [63 / 64, 0.5, 0.5]], np.float32)
    eps = np.float32(0.0)
    phi, acc, pairs = oracle.gravity(pos, np.ones(2, np.float32), 2, (0, 0, 0), 1.0, eps, periodic=True)
    assert pairs == 2
    np.testing.assert_allclose(phi, [-32.0, -32.0], rtol=1e-15)
    np.testing.assert_allclose(acc[:, 0], [-1024.0, 1024.0], rtol=1e-15)   # attraction through the wrap
    phi0, _, pairs0 = oracle.gravity(pos, np.ones(2, np.float32), 2, (0, 0, 0), 1.0, eps)
    assert pairs0 == 0 and np.all(phi0 == 0)


def test_periodic_translation_by_a_box():
    level = 3
    rng = np.random.default_rng(47)
    pos = (np.round(rng.random((2000, 3)) * 2 ** 20) / 2 ** 20).astype(np.float32) % np.float32(1.0)
    mass = rng.uniform(0.5, 1.5, 2000).astype(np.float32)
    eps = np.float32(1e-3)
    phi, acc, _ = oracle.gravity(pos, mass, level, (0, 0, 0), 1.0, eps, periodic=True)
    moved = ((pos.astype(np.float64) + np.array([1 / 8, 3 / 8, 5 / 8])) % 1.0).astype(np.float32)
    phi2, acc2, _ = oracle.gravity(moved, mass, level, (0, 0, 0), 1.0, eps, periodic=True)
    assert rel_l2(phi2, phi) < 1e-14 and rel_l2(acc2, acc) < 1e-14
    f = mass.astype(np.float64)[:, None] * acc
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()


@pytest.mark.parametrize("periodic", [False, True])
def test_context_sums_equal_one_call_sums(periodic):
    """A tree context kept across calls gives the one-call results bit for bit
    (the same tree and the same loops), at any target sample."""
    p = wl.uniform_gravity(n=5000, level=3, seed=21)
    ctx = oracle.Context(p.pos, p.level, p.lo, p.edge, periodic=periodic)
    tg = np.random.default_rng(2).choice(p.n, 700, replace=False)
    for targets in (None, tg):
        a = oracle.gravity(p.pos, p.strength, p.level, p.lo, p.edge, p.eps, targets=targets, periodic=periodic)
        b = ctx.gravity(p.strength, p.eps, targets=targets)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        assert a[2] == b[2]
        q = wl.complex_normal((2, p.n), np.random.default_rng(3))
        u1, n1 = oracle.helmholtz(p.pos, q, p.level, p.lo, p.edge, 9.0, targets=targets, periodic=periodic)
        u2, n2 = ctx.helmholtz(q, 9.0, targets=targets)
        np.testing.assert_array_equal(u1, u2)
        assert n1 == n2

"""ctypes binding of the plain-C FP64 oracle (test infrastructure only).

``build()`` compiles ``p2p_oracle.c`` with gcc (-O2, OpenMP, no FP
contraction so the float32 boxing rule is evaluated exactly as written).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p2p_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libp2p_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its source."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        F = ctypes.c_float
        lib.orc_num_threads.restype = I
        lib.orc_set_num_threads.restype = I
        lib.orc_set_num_threads.argtypes = [I]
        lib.orc_morton.restype = ctypes.c_uint32
        lib.orc_morton.argtypes = [ctypes.c_int32] * 3 + [I]
        lib.orc_unmorton.argtypes = [ctypes.c_uint32, I, P, P, P]
        lib.orc_cells.argtypes = [P, I64, I, P, F, P, P]
        lib.orc_tree.argtypes = [P, I64, I, P, F, P, P, P, P, P, P, P]
        lib.orc_redundant.argtypes = [P, ctypes.c_int32, P, P, P, P, P, P]
        lib.orc_gravity.argtypes = [P, P, I64, I, P, F, F, P, I64, P, P, P]
        lib.orc_helmholtz.argtypes = [P, P, I, I64, I, P, F, F, P, I64, P, P]
        lib.orc_pair_count.argtypes = [P, I64, I, P, F, P]
        lib.orc_helmholtz_adjoint.argtypes = [P, P, P, I, I64, I, P, F, F, P, P]
        lib.orc_tree_periodic.argtypes = [P, I64, I, P, F, P, P, P, P, P, P, P, P]
        lib.orc_gravity_periodic.argtypes = [P, P, I64, I, P, F, F, P, I64, P, P, P]
        lib.orc_helmholtz_periodic.argtypes = [P, P, I, I64, I, P, F, F, P, I64, P, P]
        lib.orc_gravity_adjoint.argtypes = [P, P, P, P, I64, I, P, F, F, P, P]
        lib.orc_context_new.restype = P
        lib.orc_context_new.argtypes = [P, I64, I, P, F, I, ctypes.POINTER(I)]
        lib.orc_context_free.argtypes = [P]
        lib.orc_gravity_ctx.argtypes = [P, P, P, F, P, I64, P, P, P]
        lib.orc_helmholtz_ctx.argtypes = [P, P, P, I, F, P, I64, P, P]
        lib.orc_gravity_ctx.restype = I
        lib.orc_helmholtz_ctx.restype = I
        for f in ("orc_cells", "orc_tree", "orc_redundant", "orc_gravity", "orc_helmholtz",
                  "orc_pair_count", "orc_helmholtz_adjoint", "orc_gravity_adjoint", "orc_tree_periodic",
                  "orc_gravity_periodic", "orc_helmholtz_periodic"):
            getattr(lib, f).restype = I
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _lo(lo):
    return np.ascontiguousarray(np.asarray(lo, np.float32).reshape(3))


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def num_threads() -> int:
    return int(load().orc_num_threads())


def set_num_threads(t: int) -> int:
    """Threads of the oracle's parallel loops on the calling thread from now on; returns the previous count."""
    return int(load().orc_set_num_threads(int(t)))


def morton(cx: int, cy: int, cz: int, level: int) -> int:
    return int(load().orc_morton(cx, cy, cz, level))


def unmorton(key: int, level: int):
    x, y, z = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    load().orc_unmorton(key, level, ctypes.byref(x), ctypes.byref(y), ctypes.byref(z))
    return x.value, y.value, z.value


def cells(pos, level, lo, edge):
    pos = np.ascontiguousarray(pos, np.float32)
    n = pos.shape[0]
    cell = np.zeros((n, 3), np.int32)
    key = np.zeros(n, np.uint32)
    lo = _lo(lo)
    _check(load().orc_cells(_p(pos), n, level, _p(lo), float(edge), _p(cell), _p(key)), "cells")
    return cell, key


def tree(pos, level, lo, edge, periodic: bool = False):
    """dict with perm, box_key, box_start, nbr_start, nbr_idx (exact sizes); periodic
    trees also carry nbr_img (image code (ox+1) + 3(oy+1) + 9(oz+1) per entry)."""
    pos = np.ascontiguousarray(pos, np.float32)
    n = pos.shape[0]
    perm = np.zeros(n, np.int32)
    box_key = np.zeros(n, np.uint32)
    box_start = np.zeros(n + 1, np.int32)
    nbr_start = np.zeros(n + 1, np.int32)
    nbr_idx = np.zeros(27 * n, np.int32)
    nbr_img = np.zeros(27 * n, np.int32)
    nb = ctypes.c_int32()
    ne = ctypes.c_int64()
    lo = _lo(lo)
    if periodic:
        _check(load().orc_tree_periodic(_p(pos), n, level, _p(lo), float(edge), _p(perm), _p(box_key),
                                        _p(box_start), ctypes.byref(nb), _p(nbr_start), _p(nbr_idx), _p(nbr_img),
                                        ctypes.byref(ne)), "tree_periodic")
    else:
        _check(load().orc_tree(_p(pos), n, level, _p(lo), float(edge), _p(perm), _p(box_key),
                               _p(box_start), ctypes.byref(nb), _p(nbr_start), _p(nbr_idx),
                               ctypes.byref(ne)), "tree")
    B, E = nb.value, ne.value
    out = {"perm": perm, "box_key": box_key[:B].copy(), "box_start": box_start[:B + 1].copy(),
           "nbr_start": nbr_start[:B + 1].copy(), "nbr_idx": nbr_idx[:E].copy(),
           "n_boxes": B, "n_nbr": E}
    if periodic:
        out["nbr_img"] = nbr_img[:E].copy()
    return out


def redundant(t, gather: bool = True):
    """red_start, red_self and (optionally) gather_idx for a tree dict."""
    B = t["n_boxes"]
    bs, ns, ni = (np.ascontiguousarray(t[k], np.int32) for k in ("box_start", "nbr_start", "nbr_idx"))
    occ = np.diff(bs).astype(np.int64)
    total_cap = int(sum(occ[ni[ns[b]:ns[b + 1]]].sum() for b in range(B))) if B < 4096 else None
    if total_cap is None:
        seg = np.repeat(np.arange(B), np.diff(ns))
        total_cap = int(np.bincount(seg, weights=occ[ni], minlength=B).sum())
    red_start = np.zeros(B + 1, np.int32)
    red_self = np.zeros(B, np.int32)
    gidx = np.zeros(max(total_cap, 1), np.uint32) if gather else None
    tot = ctypes.c_int64()
    _check(load().orc_redundant(_p(bs), B, _p(ns), _p(ni), _p(red_start), _p(red_self),
                                _p(gidx), ctypes.byref(tot)), "redundant")
    out = {"red_start": red_start, "red_self": red_self, "total": tot.value}
    if gather:
        out["gather_idx"] = gidx[:tot.value].copy()
    return out


def gravity(pos, mass, level, lo, edge, eps, targets=None, periodic: bool = False):
    """(phi[nt], acc[nt,3], pairs) in float64 at `targets` (original indices; None = all)."""
    pos = np.ascontiguousarray(pos, np.float32)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[0]
    tg = None if targets is None else np.ascontiguousarray(targets, np.int64)
    nt = n if tg is None else tg.shape[0]
    phi = np.zeros(nt, np.float64)
    acc = np.zeros((nt, 3), np.float64)
    pairs = ctypes.c_int64()
    lo = _lo(lo)
    fn = load().orc_gravity_periodic if periodic else load().orc_gravity
    _check(fn(_p(pos), _p(mass), n, level, _p(lo), float(edge), float(eps),
              _p(tg), nt, _p(phi), _p(acc), ctypes.byref(pairs)), "gravity")
    return phi, acc, pairs.value


def helmholtz(pos, q, level, lo, edge, k, targets=None, periodic: bool = False):
    """(u[nrhs, nt] complex128, pairs) at `targets` (original indices; None = all).

    q: complex64 [nrhs, n] (or [n] for one right-hand side)."""
    pos = np.ascontiguousarray(pos, np.float32)
    q = np.asarray(q)
    if q.ndim == 1:
        q = q[None, :]
    q = np.ascontiguousarray(q, np.complex64)
    nrhs, n = q.shape
    tg = None if targets is None else np.ascontiguousarray(targets, np.int64)
    nt = n if tg is None else tg.shape[0]
    u = np.zeros((nrhs, nt, 2), np.float64)
    pairs = ctypes.c_int64()
    lo = _lo(lo)
    fn = load().orc_helmholtz_periodic if periodic else load().orc_helmholtz
    _check(fn(_p(pos), _p(q.view(np.float32)), nrhs, n, level, _p(lo),
              float(edge), float(k), _p(tg), nt, _p(u), ctypes.byref(pairs)),
           "helmholtz")
    return u[..., 0] + 1j * u[..., 1], pairs.value


class Context:
    """The oracle's tree of one workload, kept across calls so that sums at
    several target samples share one tree build (the benchmark's CPU baseline
    times the two apart).  Same results as gravity() / helmholtz()."""

    def __init__(self, pos, level, lo, edge, periodic: bool = False):
        self.pos = np.ascontiguousarray(pos, np.float32)
        self.n = self.pos.shape[0]
        st = ctypes.c_int()
        self._h = load().orc_context_new(_p(self.pos), self.n, level, _p(_lo(lo)), float(edge),
                                         1 if periodic else 0, ctypes.byref(st))
        _check(st.value, "context")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_context_free(h)
            self._h = None

    def gravity(self, mass, eps, targets=None):
        mass = np.ascontiguousarray(mass, np.float32)
        tg = None if targets is None else np.ascontiguousarray(targets, np.int64)
        nt = self.n if tg is None else tg.shape[0]
        phi = np.zeros(nt, np.float64)
        acc = np.zeros((nt, 3), np.float64)
        pairs = ctypes.c_int64()
        _check(load().orc_gravity_ctx(self._h, _p(self.pos), _p(mass), float(eps), _p(tg), nt, _p(phi), _p(acc),
                                      ctypes.byref(pairs)), "gravity_ctx")
        return phi, acc, pairs.value

    def helmholtz(self, q, k, targets=None):
        q = np.asarray(q)
        if q.ndim == 1:
            q = q[None, :]
        q = np.ascontiguousarray(q, np.complex64)
        nrhs = q.shape[0]
        tg = None if targets is None else np.ascontiguousarray(targets, np.int64)
        nt = self.n if tg is None else tg.shape[0]
        u = np.zeros((nrhs, nt, 2), np.float64)
        pairs = ctypes.c_int64()
        _check(load().orc_helmholtz_ctx(self._h, _p(self.pos), _p(q.view(np.float32)), nrhs, float(k), _p(tg), nt,
                                        _p(u), ctypes.byref(pairs)), "helmholtz_ctx")
        return u[..., 0] + 1j * u[..., 1], pairs.value


def pair_count(pos, level, lo, edge) -> int:
    pos = np.ascontiguousarray(pos, np.float32)
    p = ctypes.c_int64()
    lo = _lo(lo)
    _check(load().orc_pair_count(_p(pos), pos.shape[0], level, _p(lo), float(edge),
                                 ctypes.byref(p)), "pair_count")
    return p.value


def helmholtz_adjoint(pos, q, gbar, level, lo, edge, k):
    """(grad_q [nrhs, n] complex128, grad_x [n, 3] float64) for gbar = dL/du [nrhs, n]."""
    pos = np.ascontiguousarray(pos, np.float32)
    q = np.ascontiguousarray(np.atleast_2d(q), np.complex64)
    gbar = np.ascontiguousarray(np.atleast_2d(gbar), np.complex64)
    nrhs, n = q.shape
    gq = np.zeros((nrhs, n, 2), np.float64)
    gx = np.zeros((n, 3), np.float64)
    lo = _lo(lo)
    _check(load().orc_helmholtz_adjoint(_p(pos), _p(q.view(np.float32)), _p(gbar.view(np.float32)), nrhs, n, level,
                                        _p(lo), float(edge), float(k), _p(gq), _p(gx)), "helmholtz_adjoint")
    return gq[..., 0] + 1j * gq[..., 1], gx


def gravity_adjoint(pos, mass, gphi, gacc, level, lo, edge, eps):
    """(grad_m [n] float64, grad_x [n, 3] float64) for gphi = dL/dphi, gacc = dL/da."""
    pos = np.ascontiguousarray(pos, np.float32)
    mass = np.ascontiguousarray(mass, np.float32)
    gphi = np.ascontiguousarray(gphi, np.float32)
    gacc = np.ascontiguousarray(gacc, np.float32)
    n = pos.shape[0]
    gm = np.zeros(n, np.float64)
    gx = np.zeros((n, 3), np.float64)
    lo = _lo(lo)
    _check(load().orc_gravity_adjoint(_p(pos), _p(mass), _p(gphi), _p(gacc), n, level, _p(lo), float(edge),
                                      float(eps), _p(gm), _p(gx)), "gravity_adjoint")
    return gm, gx

"""Thin Python binding of the C ABI in ``include/p2p_gb300.h``.

Argument marshalling only: every step of the operator runs in the CUDA
library.  PyTorch provides device memory (the workspace and the outputs) and
the stream (the current torch stream).  If the compiled library is missing
the first call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

GRAVITY, HELMHOLTZ = 0, 1
LAYOUTS = {"indirect": 0, "redundant": 1, "auto": 2, "pairtask": 3, "symmetric": 4}
PLAN_GATHER_MAP, PLAN_PLAIN_FP32, PLAN_TIMING, PLAN_ADJOINT, PLAN_PERIODIC = 0x1, 0x2, 0x4, 0x8, 0x10
PLAN_SYMMETRIC = 0x20
PLAN_HOST_IO = 0x40
FLAG_DOMAIN, FLAG_TIMEOUT, FLAG_CAPACITY, FLAG_LATTICE = 0x1, 0x2, 0x4, 0x8

ARRAYS = {"perm": (0, torch.int32), "box_key": (1, torch.int32), "box_start": (2, torch.int32),
          "nbr_start": (3, torch.int32), "nbr_idx": (4, torch.int32), "red_start": (5, torch.int32),
          "red_self": (6, torch.int32), "gather_idx": (7, torch.int32), "sorted_key": (8, torch.int32),
          "nbr_img": (9, torch.int32), "ent_box": (10, torch.int32), "pt_start": (11, torch.int32),
          "part_start": (12, torch.int32), "task_kind": (13, torch.int32), "mirror": (14, torch.int32),
          "bslot": (15, torch.int32)}
COUNTERS = ("n_boxes", "n_nbr", "flags", "total_src", "pairs", "n_items", "evals")
PHASES = ("tree", "restructure", "kernel", "operator")

EXPORTS = ("p2p_status_string", "p2p_abi_version", "p2p_plan_create", "p2p_plan_destroy",
           "p2p_plan_workspace_bytes", "p2p_plan_set_tuning", "p2p_tree_build", "p2p_tree_import",
           "p2p_restructure", "p2p_gravity", "p2p_helmholtz", "p2p_plan_array", "p2p_read_counters",
           "p2p_plan_timing", "p2p_launch_count", "p2p_gravity_noalloc",
           "p2p_measure_pipes", "p2p_helmholtz_adjoint", "p2p_gravity_adjoint",
           "p2p_batch_create", "p2p_batch_destroy", "p2p_batch_workspace_bytes", "p2p_batch_build",
           "p2p_batch_set_tuning", "p2p_batch_run", "p2p_batch_autotune", "p2p_batch_capture",
           "p2p_batch_launch", "p2p_batch_counters", "p2p_selftest_bounded_wait",
           "p2p_plan_set_grid", "p2p_build_checked", "p2p_fail_host_allocs", "p2p_gravity_host",
           "p2p_helmholtz_host", "p2p_batch_timing", "p2p_gravity_noalloc_status", "p2p_momentum_fp64",
           "p2p_dot_fp64")


class P2PError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


_lib = None


def library_path() -> str:
    """The release library, or the checked variant when the environment sets
    P2P_GB300_VARIANT=checked before the first load."""
    variant = os.environ.get("P2P_GB300_VARIANT", "release")
    if variant not in _build.VARIANTS:
        raise ValueError(f"P2P_GB300_VARIANT={variant!r}: expected one of {sorted(_build.VARIANTS)}")
    return _build.VARIANTS[variant][0]


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the compiled library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build(variants=(os.environ.get("P2P_GB300_VARIANT", "release"),))
        else:
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, I64, F, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_uint
    SZ = ctypes.c_size_t
    sig = {
        "p2p_status_string": (ctypes.c_char_p, [I]),
        "p2p_abi_version": (I, []),
        "p2p_plan_create": (I, [ctypes.POINTER(P), I, I64, I, P, F, I, I, U]),
        "p2p_plan_destroy": (I, [P]),
        "p2p_plan_workspace_bytes": (I, [P, ctypes.POINTER(SZ)]),
        "p2p_plan_set_tuning": (I, [P, I, I, I, I]),
        "p2p_tree_build": (I, [P, P, P, SZ, P]),
        "p2p_tree_import": (I, [P, P, P, ctypes.c_int32, P, P, ctypes.c_int32, P, SZ, P]),
        "p2p_restructure": (I, [P, P, P, P, SZ, P]),
        "p2p_gravity": (I, [P, F, P, P, P, SZ, P]),
        "p2p_helmholtz": (I, [P, F, P, P, SZ, P]),
        "p2p_plan_array": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "p2p_read_counters": (I, [P, P, ctypes.POINTER(I64), P]),
        "p2p_plan_timing": (I, [P, ctypes.POINTER(F)]),
        "p2p_launch_count": (I64, []),
        "p2p_gravity_noalloc": (I, [P, P, I64, I, P, F, F, I, P, P, P]),
        "p2p_measure_pipes": (I, [ctypes.POINTER(ctypes.c_double), P]),
        "p2p_helmholtz_adjoint": (I, [P, F, P, P, P, P, P, P, SZ, P]),
        "p2p_gravity_adjoint": (I, [P, F, P, P, P, P, P, P, P, SZ, P]),
        "p2p_batch_create": (I, [ctypes.POINTER(P), I, I, P, P, P, P, I, I, I, U]),
        "p2p_batch_destroy": (I, [P]),
        "p2p_batch_workspace_bytes": (I, [P, ctypes.POINTER(SZ)]),
        "p2p_batch_build": (I, [P, P, P, SZ, P]),
        "p2p_batch_set_tuning": (I, [P, I, I, I, I, I]),
        "p2p_batch_run": (I, [P, F, P, P, P, P, P, P, SZ, P]),
        "p2p_batch_autotune": (I, [P, F, P, P, P, P, P, P, SZ, P, ctypes.POINTER(I), ctypes.POINTER(F)]),
        "p2p_batch_capture": (I, [P, F, P, P, P, P, P, P, SZ]),
        "p2p_batch_launch": (I, [P, P]),
        "p2p_batch_counters": (I, [P, P, ctypes.POINTER(I64), P]),
        "p2p_batch_timing": (I, [P, ctypes.POINTER(F)]),
        "p2p_gravity_noalloc_status": (I, [ctypes.POINTER(U), P]),
        "p2p_momentum_fp64": (I, [P, P, I64, P, P]),
        "p2p_dot_fp64": (I, [P, P, I64, P, P]),
        "p2p_selftest_bounded_wait": (I, [ctypes.c_uint64, P, P]),
        "p2p_plan_set_grid": (I, [P, F, I]),
        "p2p_build_checked": (I, []),
        "p2p_fail_host_allocs": (I, [I]),
        "p2p_gravity_host": (I, [P, F, P, P, P, P, P, SZ, P]),
        "p2p_helmholtz_host": (I, [P, F, P, P, P, P, SZ, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().p2p_status_string(int(status)).decode()
    except ImportError:
        return "library not loaded"


def launch_count() -> int:
    return int(load().p2p_launch_count())


def measure_pipes(stream=None) -> dict:
    """FP32 (scalar and packed two-wide) and MUFU lane-ops per SM per clock, and the SM
    clock (MHz), measured on the device."""
    out = (ctypes.c_double * 5)()
    _check(load().p2p_measure_pipes(out, _stream(stream)), "p2p_measure_pipes")
    return {"fp32": out[0], "mufu_rsqrt": out[1], "mufu_sin": out[2], "sm_mhz": out[3], "fp32x2": out[4]}


def selftest_bounded_wait(limit_ns: int = 2_000_000, device=None, stream=None) -> int:
    """Run a wait that nothing completes with the given limit; returns the status
    (P2P_ERR_TIMEOUT = 4 is the expected outcome)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    return int(load().p2p_selftest_bounded_wait(int(limit_ns), _ptr(flags), _stream(stream)))


def _check(st: int, what: str):
    if st != 0:
        raise P2PError(st, what)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """One problem shape (n, level, domain, kernel, layout) and its workspace.

    kind: "gravity" (softened 1/r: potential and acceleration) or "helmholtz"
    (e^{ikr}/(4 pi r) on complex sources, nrhs right-hand sides).  n particles
    in the cube [lo, lo + edge)^3, uniform octree of 2^level boxes per edge.
    layout: "redundant" (per-box contiguous source streams, the paper's data
    redundancy), "indirect" (per-neighbour ranges of the box-ordered records),
    "pairtask" (one task per (box, neighbour) with partial results reduced
    afterwards) or "symmetric" (pair tasks evaluated once for both particles).
    Flags: gather_map (keep the restructuring's source index map), plain_fp32
    (no compensated sums), timing (CUDA-event phase timers, see timing()),
    adjoint (room for the adjoint records), periodic (toroidal boundaries),
    symmetric (each pair of a small box pair evaluated once on a target-owned
    layout), host_io (device copies of inputs and outputs for the *_host calls).

    The workspace is one torch uint8 tensor on the plan's device (allocated
    here unless given); every intermediate array of the pipeline lives inside
    it.  Calls are asynchronous on the current (or given) stream; device-side
    errors are reported by counters().
    """

    def __init__(self, kind: str, n: int, level: int, lo, edge: float, nrhs: int = 1,
                 layout: str = "redundant", gather_map: bool = False, plain_fp32: bool = False,
                 timing: bool = False, adjoint: bool = False, periodic: bool = False, symmetric: bool = False,
                 host_io: bool = False, device=None, workspace: torch.Tensor | None = None):
        lib = load()
        self.kind = kind
        self.n = int(n)
        self.nrhs = int(nrhs)
        self.level = int(level)
        self.layout = layout
        self.periodic = bool(periodic)
        self.symmetric = bool(symmetric)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        flags = (PLAN_GATHER_MAP if gather_map else 0) | (PLAN_PLAIN_FP32 if plain_fp32 else 0) | \
                (PLAN_TIMING if timing else 0) | (PLAN_ADJOINT if adjoint else 0) | \
                (PLAN_PERIODIC if periodic else 0) | (PLAN_SYMMETRIC if symmetric else 0) | \
                (PLAN_HOST_IO if host_io else 0)
        lo_arr = (ctypes.c_float * 3)(*[float(v) for v in lo])
        h = ctypes.c_void_p()
        kid = {"gravity": GRAVITY, "helmholtz": HELMHOLTZ}[kind]
        _check(lib.p2p_plan_create(ctypes.byref(h), kid, self.n, self.level, lo_arr, float(edge),
                                   self.nrhs, LAYOUTS[layout], flags), "p2p_plan_create")
        self._h = h
        nb = ctypes.c_size_t()
        _check(lib.p2p_plan_workspace_bytes(h, ctypes.byref(nb)), "p2p_plan_workspace_bytes")
        self.ws_bytes = int(nb.value)
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        elif workspace.numel() < self.ws_bytes:
            raise ValueError("workspace too small")
        self.ws = workspace

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.p2p_plan_destroy(h)
            self._h = None

    # -- knobs --------------------------------------------------------------
    def set_tuning(self, targets_per_lane: int, tile: int, ctas_per_sm: int = 0, warps_per_item: int = 4):
        """Targets per lane (1, 2, 4), source records per shared-memory stage (32, 48, 64,
        128), CTAs per SM (0: as many as fit), warps cooperating on one work item (1, 2, 4)."""
        _check(load().p2p_plan_set_tuning(self._h, targets_per_lane, tile, ctas_per_sm, warps_per_item),
               "p2p_plan_set_tuning")

    def set_grid(self, h: float, points_per_box: int):
        """Pattern mode for particles on a regular lattice (0 points disables)."""
        _check(load().p2p_plan_set_grid(self._h, float(h), int(points_per_box)), "p2p_plan_set_grid")

    # -- pipeline -----------------------------------------------------------
    def _wsp(self):
        return ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel())

    def tree_build(self, pos: torch.Tensor, stream=None):
        _need(pos, torch.float32, (self.n, 3), self.device)
        w, b = self._wsp()
        _check(load().p2p_tree_build(self._h, _ptr(pos), w, b, _stream(stream)), "p2p_tree_build")

    def tree_import(self, perm, box_start, nbr_start, nbr_idx, stream=None):
        nb = int(box_start.numel()) - 1
        ne = int(nbr_idx.numel())
        for t in (perm, box_start, nbr_start, nbr_idx):
            _need(t, torch.int32, None, self.device)
        w, b = self._wsp()
        _check(load().p2p_tree_import(self._h, _ptr(perm), _ptr(box_start), nb, _ptr(nbr_start), _ptr(nbr_idx),
                                      ne, w, b, _stream(stream)), "p2p_tree_import")

    def restructure(self, pos: torch.Tensor, strength: torch.Tensor, stream=None):
        _need(pos, torch.float32, (self.n, 3), self.device)
        if self.kind == "gravity":
            _need(strength, torch.float32, (self.n,), self.device)
        else:
            _need(strength, torch.complex64, (self.nrhs, self.n), self.device)
        w, b = self._wsp()
        _check(load().p2p_restructure(self._h, _ptr(pos), _ptr(strength), w, b, _stream(stream)),
               "p2p_restructure")

    def gravity(self, eps: float, phi=None, acc=None, stream=None):
        if phi is None:
            phi = torch.empty(self.n, dtype=torch.float32, device=self.device)
        if acc is None:
            acc = torch.empty(self.n, 3, dtype=torch.float32, device=self.device)
        _need(phi, torch.float32, (self.n,), self.device)
        _need(acc, torch.float32, (self.n, 3), self.device)
        w, b = self._wsp()
        _check(load().p2p_gravity(self._h, float(eps), _ptr(phi), _ptr(acc), w, b, _stream(stream)), "p2p_gravity")
        return phi, acc

    def helmholtz(self, k: float, u=None, stream=None):
        if u is None:
            u = torch.empty(self.nrhs, self.n, dtype=torch.complex64, device=self.device)
        _need(u, torch.complex64, (self.nrhs, self.n), self.device)
        w, b = self._wsp()
        _check(load().p2p_helmholtz(self._h, float(k), _ptr(u), w, b, _stream(stream)), "p2p_helmholtz")
        return u

    def helmholtz_adjoint(self, k: float, pos, gbar, q=None, want_q: bool = True, want_pos: bool = False,
                          stream=None):
        """(grad_q [nrhs, n] complex64 or None, grad_pos [n, 3] float32 or None) for gbar = dL/du."""
        _need(pos, torch.float32, (self.n, 3), self.device)
        _need(gbar, torch.complex64, (self.nrhs, self.n), self.device)
        gq = torch.empty(self.nrhs, self.n, dtype=torch.complex64, device=self.device) if want_q else None
        gx = torch.empty(self.n, 3, dtype=torch.float32, device=self.device) if want_pos else None
        if want_pos:
            _need(q, torch.complex64, (self.nrhs, self.n), self.device)
        w, b = self._wsp()
        _check(load().p2p_helmholtz_adjoint(self._h, float(k), _ptr(pos), _ptr(q if want_pos else None), _ptr(gbar),
                                            _ptr(gq), _ptr(gx), w, b, _stream(stream)), "p2p_helmholtz_adjoint")
        return gq, gx

    def gravity_adjoint(self, eps: float, pos, mass, grad_phi, grad_acc, want_mass: bool = True,
                        want_pos: bool = True, stream=None):
        """(grad_mass [n] or None, grad_pos [n, 3] or None) for grad_phi = dL/dphi, grad_acc = dL/da."""
        _need(pos, torch.float32, (self.n, 3), self.device)
        _need(mass, torch.float32, (self.n,), self.device)
        _need(grad_phi, torch.float32, (self.n,), self.device)
        _need(grad_acc, torch.float32, (self.n, 3), self.device)
        gm = torch.empty(self.n, dtype=torch.float32, device=self.device) if want_mass else None
        gx = torch.empty(self.n, 3, dtype=torch.float32, device=self.device) if want_pos else None
        w, b = self._wsp()
        _check(load().p2p_gravity_adjoint(self._h, float(eps), _ptr(pos), _ptr(mass), _ptr(grad_phi),
                                          _ptr(grad_acc), _ptr(gm), _ptr(gx), w, b, _stream(stream)),
               "p2p_gravity_adjoint")
        return gm, gx

    # -- one step from host buffers (host_io plans) ---------------------------
    def gravity_host(self, eps: float, pos, mass, phi, acc, stream=None):
        """Host tensors in and out (pinned for asynchronous copies): positions [n, 3],
        masses [n] -> phi [n], acc [n, 3].  Asynchronous on the stream."""
        cpu = torch.device("cpu")
        _need(pos, torch.float32, (self.n, 3), cpu)
        _need(mass, torch.float32, (self.n,), cpu)
        _need(phi, torch.float32, (self.n,), cpu)
        _need(acc, torch.float32, (self.n, 3), cpu)
        w, b = self._wsp()
        _check(load().p2p_gravity_host(self._h, float(eps), _ptr(pos), _ptr(mass), _ptr(phi), _ptr(acc), w, b,
                                       _stream(stream)), "p2p_gravity_host")

    def helmholtz_host(self, k: float, pos, q, u, stream=None):
        """Host tensors in and out (pinned for asynchronous copies): positions [n, 3],
        q [nrhs, n] complex64 -> u [nrhs, n].  Asynchronous on the stream."""
        cpu = torch.device("cpu")
        _need(pos, torch.float32, (self.n, 3), cpu)
        _need(q, torch.complex64, (self.nrhs, self.n), cpu)
        _need(u, torch.complex64, (self.nrhs, self.n), cpu)
        w, b = self._wsp()
        _check(load().p2p_helmholtz_host(self._h, float(k), _ptr(pos), _ptr(q), _ptr(u), w, b, _stream(stream)),
               "p2p_helmholtz_host")

    # -- inspection ---------------------------------------------------------
    def counters(self, stream=None, check: bool = False) -> dict:
        out = (ctypes.c_int64 * len(COUNTERS))()
        st = load().p2p_read_counters(self._h, ctypes.c_void_p(self.ws.data_ptr()), out, _stream(stream))
        res = {k: int(v) for k, v in zip(COUNTERS, out)}
        res["status"] = int(st)
        if check:
            _check(st, "p2p_read_counters")
        return res

    def array(self, name: str, length: int | None = None) -> torch.Tensor:
        """A view of a workspace array (first `length` elements)."""
        which, dtype = ARRAYS[name]
        off, cap = ctypes.c_int64(), ctypes.c_int64()
        _check(load().p2p_plan_array(self._h, which, ctypes.byref(off), ctypes.byref(cap)), "p2p_plan_array")
        length = int(cap.value) if length is None else int(length)
        nbytes = length * 4
        return self.ws[off.value: off.value + nbytes].view(dtype)

    def timing(self) -> dict:
        out = (ctypes.c_float * len(PHASES))()
        _check(load().p2p_plan_timing(self._h, out), "p2p_plan_timing")
        return {k: float(v) for k, v in zip(PHASES, out)}


def momentum_fp64(mass, acc, stream=None) -> torch.Tensor:
    """Device FP64 sums (sum_i m_i a_i [3], sum_i |m_i a_i| [3]) of the gravity outputs: float64 [6]."""
    _need(mass, torch.float32, None, mass.device)
    _need(acc, torch.float32, (mass.numel(), 3), mass.device)
    out = torch.empty(6, dtype=torch.float64, device=mass.device)
    _check(load().p2p_momentum_fp64(_ptr(mass), _ptr(acc), mass.numel(), _ptr(out), _stream(stream)),
           "p2p_momentum_fp64")
    return out


def dot_fp64(x, y, stream=None) -> torch.Tensor:
    """Device FP64 sum of x_i y_i over the float32 (or complex64: Re sum conj(x) y) values: float64 [1]."""
    xf = torch.view_as_real(x) if x.is_complex() else x
    yf = torch.view_as_real(y) if y.is_complex() else y
    if xf.dtype != torch.float32 or yf.dtype != torch.float32 or xf.numel() != yf.numel():
        raise ValueError("dot_fp64 needs float32 or complex64 tensors of the same size")
    xf, yf = xf.contiguous(), yf.contiguous()
    out = torch.empty(1, dtype=torch.float64, device=xf.device)
    _check(load().p2p_dot_fp64(_ptr(xf), _ptr(yf), xf.numel(), _ptr(out), _stream(stream)), "p2p_dot_fp64")
    return out


def _need(t, dtype, shape, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.device != device:
        raise ValueError(f"expected a tensor on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")


# ---------------------------------------------------------------------------
# one-call conveniences: tree -> restructure -> operator
# ---------------------------------------------------------------------------

def gravity(pos, mass, level, lo, edge, eps, layout="redundant", plan: Plan | None = None,
            periodic: bool = False):
    """Softened-gravity near field (phi [n], acc [n,3]) in original particle order."""
    plan = plan or Plan("gravity", pos.shape[0], level, lo, edge, layout=layout, periodic=periodic,
                        device=pos.device)
    plan.tree_build(pos)
    plan.restructure(pos, mass)
    return plan.gravity(eps)


def helmholtz(pos, q, level, lo, edge, k, layout="redundant", plan: Plan | None = None,
              periodic: bool = False):
    """Helmholtz near field u [nrhs, n] (complex64) in original particle order."""
    if q.dim() == 1:
        q = q.unsqueeze(0)
    plan = plan or Plan("helmholtz", pos.shape[0], level, lo, edge, nrhs=q.shape[0], layout=layout,
                        periodic=periodic,
                        device=pos.device)
    plan.tree_build(pos)
    plan.restructure(pos, q.contiguous())
    return plan.helmholtz(k)


# ---------------------------------------------------------------------------
# differentiable operators (hand-written adjoint kernels behind autograd)
# ---------------------------------------------------------------------------

class _HelmholtzFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, q, plan, k):
        plan.tree_build(pos)
        plan.restructure(pos, q)
        u = plan.helmholtz(k)
        ctx.save_for_backward(pos, q)
        ctx.plan, ctx.k = plan, k
        return u

    @staticmethod
    def backward(ctx, grad_u):
        pos, q = ctx.saved_tensors
        want_pos, want_q = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_pos or want_q):
            return None, None, None, None
        plan = ctx.plan
        plan.tree_build(pos)          # the plan may have served other calls since the forward
        gq, gx = plan.helmholtz_adjoint(ctx.k, pos, grad_u.contiguous(), q, want_q=want_q, want_pos=want_pos)
        return gx, gq, None, None


class _GravityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, mass, plan, eps):
        plan.tree_build(pos)
        plan.restructure(pos, mass)
        phi, acc = plan.gravity(eps)
        ctx.save_for_backward(pos, mass)
        ctx.plan, ctx.eps = plan, eps
        return phi, acc

    @staticmethod
    def backward(ctx, grad_phi, grad_acc):
        pos, mass = ctx.saved_tensors
        want_pos, want_m = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_pos or want_m):
            return None, None, None, None
        if grad_phi is None:
            grad_phi = torch.zeros_like(mass)
        if grad_acc is None:
            grad_acc = torch.zeros_like(pos)
        plan = ctx.plan
        plan.tree_build(pos)
        gm, gx = plan.gravity_adjoint(ctx.eps, pos, mass, grad_phi.contiguous(), grad_acc.contiguous(),
                                      want_mass=want_m, want_pos=want_pos)
        return gx, gm, None, None


def helmholtz_p2p(pos, q, plan: Plan, k: float):
    """Differentiable Helmholtz near field u = P(pos) q; gradients flow to q and pos
    through the adjoint kernels.  The plan must be created with adjoint=True for
    position gradients."""
    return _HelmholtzFn.apply(pos, q, plan, k)


def gravity_p2p(pos, mass, plan: Plan, eps: float):
    """Differentiable softened gravity (phi, acc); gradients flow to mass and pos.
    The plan must be created with adjoint=True."""
    return _GravityFn.apply(pos, mass, plan, eps)


# ---------------------------------------------------------------------------
# batched instances: one persistent launch (optionally one CUDA graph)
# ---------------------------------------------------------------------------

class Batch:
    """Many Helmholtz instances with concatenated data; see p2p_batch_* in the header.

    instances: sequence of (n, level, lo, edge).  pair=True computes u = P q and
    g = conj(P) y in the same launch.
    """

    def __init__(self, instances, nrhs: int, k: float, pair: bool = False, layout: str = "auto",
                 plain_fp32: bool = False, timing: bool = False, device=None):
        lib = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nrhs, self.k, self.pair = int(nrhs), float(k), bool(pair)
        I = len(instances)
        n = (ctypes.c_int64 * I)(*[int(x[0]) for x in instances])
        lv = (ctypes.c_int * I)(*[int(x[1]) for x in instances])
        lo = (ctypes.c_float * (3 * I))(*[float(v) for x in instances for v in x[2]])
        ed = (ctypes.c_float * I)(*[float(x[3]) for x in instances])
        self.sizes = [int(x[0]) for x in instances]
        self.offsets = [0]
        for s_ in self.sizes:
            self.offsets.append(self.offsets[-1] + s_)
        self.N = self.offsets[-1]
        h = ctypes.c_void_p()
        _check(lib.p2p_batch_create(ctypes.byref(h), HELMHOLTZ, I, n, lv, lo, ed, self.nrhs, 1 if pair else 0,
                                    LAYOUTS[layout], (PLAN_PLAIN_FP32 if plain_fp32 else 0) |
                                    (PLAN_TIMING if timing else 0)), "p2p_batch_create")
        self._h = h
        nb = ctypes.c_size_t()
        _check(lib.p2p_batch_workspace_bytes(h, ctypes.byref(nb)), "p2p_batch_workspace_bytes")
        self.ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self._bufs = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.p2p_batch_destroy(h)
            self._h = None

    def _w(self):
        return ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel())

    def build(self, pos, stream=None):
        _need(pos, torch.float32, (self.N, 3), self.device)
        w, b = self._w()
        _check(load().p2p_batch_build(self._h, _ptr(pos), w, b, _stream(stream)), "p2p_batch_build")

    def _args(self, pos, q, y, u, g):
        _need(pos, torch.float32, (self.N, 3), self.device)
        _need(q, torch.complex64, (self.nrhs, self.N), self.device)
        if u is None:
            u = torch.empty(self.nrhs, self.N, dtype=torch.complex64, device=self.device)
        if self.pair:
            _need(y, torch.complex64, (self.nrhs, self.N), self.device)
            if g is None:
                g = torch.empty(self.nrhs, self.N, dtype=torch.complex64, device=self.device)
        return u, g

    def run(self, pos, q, y=None, u=None, g=None, stream=None):
        u, g = self._args(pos, q, y, u, g)
        w, b = self._w()
        _check(load().p2p_batch_run(self._h, self.k, _ptr(pos), _ptr(q), _ptr(y), _ptr(u), _ptr(g), w, b,
                                    _stream(stream)), "p2p_batch_run")
        return (u, g) if self.pair else u

    def set_tuning(self, layout: str, targets_per_lane: int, tile: int, warps_per_item: int, ctas_per_sm: int = 0):
        _check(load().p2p_batch_set_tuning(self._h, LAYOUTS[layout], targets_per_lane, tile, ctas_per_sm,
                                           warps_per_item), "p2p_batch_set_tuning")

    def autotune(self, pos, q, y=None, u=None, g=None, stream=None, cache=None) -> dict:
        """Time the tuning space on these buffers and keep the fastest choice.
        cache: a tune_cache.TuneCache (or True for the default file): a stored
        choice for this GPU, batch shape class and kernel build is applied
        without timing, and a new choice is stored."""
        from . import tune_cache as _tc
        if cache is True:
            cache = _tc.TuneCache()
        key = None
        if cache:
            key = _tc.TuneCache.key(torch.cuda.get_device_name(self.device),
                                    _tc.shape_class(self.sizes, self.nrhs, self.pair))
            hit = cache.get(key)
            if hit is not None:
                self.set_tuning(hit["layout"], hit["targets_per_lane"], hit["tile"], hit["warps_per_item"])
                return dict(hit, cached=True)
        res = self._autotune(pos, q, y, u, g, stream)
        if cache:
            cache.put(key, res)
        return dict(res, cached=False)

    def _autotune(self, pos, q, y, u, g, stream) -> dict:
        u, g = self._args(pos, q, y, u, g)
        best = (ctypes.c_int * 5)()
        ms = ctypes.c_float()
        w, b = self._w()
        _check(load().p2p_batch_autotune(self._h, self.k, _ptr(pos), _ptr(q), _ptr(y), _ptr(u), _ptr(g), w, b,
                                         _stream(stream), best, ctypes.byref(ms)), "p2p_batch_autotune")
        inv = {v: k_ for k_, v in LAYOUTS.items()}
        return {"layout": inv[best[0]], "targets_per_lane": best[1], "tile": best[2], "warps_per_item": best[4],
                "ms": ms.value}

    def capture(self, pos, q, y=None, u=None, g=None):
        """Capture run() on these buffers into a CUDA graph; returns the outputs it writes."""
        u, g = self._args(pos, q, y, u, g)
        self._bufs = (pos, q, y, u, g)     # the graph keeps using these addresses
        w, b = self._w()
        _check(load().p2p_batch_capture(self._h, self.k, _ptr(pos), _ptr(q), _ptr(y), _ptr(u), _ptr(g), w, b),
               "p2p_batch_capture")
        return (u, g) if self.pair else u

    def launch(self, stream=None):
        _check(load().p2p_batch_launch(self._h, _stream(stream)), "p2p_batch_launch")

    def timing(self) -> dict:
        """Milliseconds of the last run's phases (batches created with timing=True);
        "tree" is -1 (trees are built once by build())."""
        out = (ctypes.c_float * len(PHASES))()
        _check(load().p2p_batch_timing(self._h, out), "p2p_batch_timing")
        return {k_: float(v) for k_, v in zip(PHASES, out)}

    def counters(self, stream=None) -> dict:
        out = (ctypes.c_int64 * len(COUNTERS))()
        st = load().p2p_batch_counters(self._h, ctypes.c_void_p(self.ws.data_ptr()), out, _stream(stream))
        res = {k_: int(v) for k_, v in zip(COUNTERS, out)}
        res["status"] = int(st)
        return res

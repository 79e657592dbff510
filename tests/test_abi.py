"""The C ABI library loads and exports every entry point declared in
include/*.h; host-side argument checks (no GPU work)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2511_21535_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(p2p_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = cuda_build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("p2p_plan_create", "p2p_tree_build", "p2p_restructure", "p2p_gravity",
                     "p2p_helmholtz", "p2p_read_counters"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_export():
    from paper_2511_21535_gb300 import p2p
    assert set(declared_functions()) <= set(p2p.EXPORTS)


def _create(lib, kind=0, n=1000, level=3, lo=(0.0, 0.0, 0.0), edge=1.0, nrhs=1, layout=1, flags=0):
    h = ctypes.c_void_p()
    lo_arr = (ctypes.c_float * 3)(*lo)
    lib.p2p_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_uint]
    st = lib.p2p_plan_create(ctypes.byref(h), kind, n, level, ctypes.cast(lo_arr, ctypes.c_void_p), edge, nrhs,
                             layout, flags)
    return st, h


def test_plan_argument_checks(lib):
    bad = [dict(n=0), dict(n=(1 << 26) + 1), dict(level=0), dict(level=11), dict(edge=0.0), dict(edge=-1.0),
           dict(kind=2), dict(layout=5), dict(layout=2), dict(layout=4, kind=1, nrhs=3), dict(nrhs=2), dict(kind=1, nrhs=0), dict(kind=1, nrhs=17),
           dict(layout=3, n=(1 << 25) + 1), dict(layout=3, flags=0x8), dict(flags=0x10, level=1),
           dict(flags=0x100), dict(lo=(float("nan"), 0.0, 0.0))]
    for kw in bad:
        st, h = _create(lib, **kw)
        assert st == 1, kw
        assert not h.value
    st, h = _create(lib)
    assert st == 0 and h.value
    lib.p2p_plan_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    nb = ctypes.c_size_t()
    assert lib.p2p_plan_workspace_bytes(h, ctypes.byref(nb)) == 0
    assert nb.value > 27 * 1000 * 16          # holds the redundant streams
    st, hp = _create(lib, layout=3)
    assert st == 0 and hp.value
    nbp = ctypes.c_size_t()
    assert lib.p2p_plan_workspace_bytes(hp, ctypes.byref(nbp)) == 0
    assert nbp.value > nb.value + 27 * 1000 * 16   # task stream (54 n records) and partial results
    lib.p2p_plan_set_tuning.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
    assert lib.p2p_plan_set_tuning(h, 3, 64, 0, 1) == 1
    assert lib.p2p_plan_set_tuning(h, 2, 40, 0, 1) == 1
    assert lib.p2p_plan_set_tuning(h, 2, 256, 0, 1) == 1
    assert lib.p2p_plan_set_tuning(h, 2, 48, 0, 1) == 0
    assert lib.p2p_plan_set_tuning(h, 2, 64, 0, 3) == 1
    assert lib.p2p_plan_set_tuning(h, 4, 32, 2, 4) == 0
    # operator before the tree: state error is checked before any device work
    lib.p2p_gravity.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert lib.p2p_gravity(h, 1e-3, 256, 256, 0, 0, None) == 7      # no workspace
    lib.p2p_plan_destroy.argtypes = [ctypes.c_void_p]
    assert lib.p2p_plan_destroy(h) == 0
    assert lib.p2p_plan_destroy(hp) == 0
    assert lib.p2p_plan_destroy(None) == 0


def test_host_io_plan(lib):
    """P2P_PLAN_HOST_IO: the workspace holds device copies of the inputs and outputs
    (12 n + 4 n + 16 n bytes for gravity); the host entry points refuse plans
    without it before any device work."""
    lib.p2p_plan_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    st, h0 = _create(lib, n=10000)
    st1, h1 = _create(lib, n=10000, flags=0x40)
    assert st == 0 and st1 == 0 and h1.value
    b0, b1 = ctypes.c_size_t(), ctypes.c_size_t()
    lib.p2p_plan_workspace_bytes(h0, ctypes.byref(b0))
    lib.p2p_plan_workspace_bytes(h1, ctypes.byref(b1))
    assert b1.value - b0.value >= 32 * 10000
    P = ctypes.c_void_p
    lib.p2p_gravity_host.argtypes = [P, ctypes.c_float, P, P, P, P, P, ctypes.c_size_t, P]
    buf = (ctypes.c_float * 8)()
    ptr = ctypes.cast(buf, P)
    assert lib.p2p_gravity_host(h0, 1e-3, ptr, ptr, ptr, ptr, ptr, b0.value, None) == 5
    assert lib.p2p_gravity_host(h1, 1e-3, None, ptr, ptr, ptr, ptr, b1.value, None) == 1
    lib.p2p_plan_destroy.argtypes = [P]
    lib.p2p_plan_destroy(h0)


def test_workspace_layout_scales(lib):
    lib.p2p_plan_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    sizes = {}
    for layout in (0, 1):
        st, h = _create(lib, n=100000, level=5, layout=layout)
        nb = ctypes.c_size_t()
        lib.p2p_plan_workspace_bytes(h, ctypes.byref(nb))
        sizes[layout] = nb.value
        lib.p2p_plan_destroy(h)
    # the redundant layout reserves 27 n records (16 B) beyond the indirect one
    assert sizes[1] - sizes[0] >= 27 * 100000 * 16


def test_status_strings(lib):
    lib.p2p_status_string.restype = ctypes.c_char_p
    for s in range(10):
        assert lib.p2p_status_string(s)
    assert lib.p2p_abi_version() == 1


def test_injected_host_allocation_failure(lib):
    """Plan and batch creation report P2P_ERR_OOM (3) when their host
    allocation fails, leave *out null, and work again once the injection is used up."""
    assert lib.p2p_build_checked() == 0
    assert lib.p2p_fail_host_allocs(1) == 0
    st, h = _create(lib)
    assert st == 3 and not h.value
    st, h = _create(lib)
    assert st == 0 and h.value
    lib.p2p_plan_destroy(h)
    I64, I, F = ctypes.c_int64, ctypes.c_int, ctypes.c_float
    n, lv, lo, ed = (I64 * 2)(500, 700), (I * 2)(2, 3), (F * 6)(*([0.0] * 6)), (F * 2)(1.0, 1.0)
    lib.p2p_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I, I] + [ctypes.c_void_p] * 4 + [I, I, I,
                                                                                                       ctypes.c_uint]
    lib.p2p_batch_destroy.argtypes = [ctypes.c_void_p]
    args = lambda b: (ctypes.byref(b), 1, 2, ctypes.cast(n, ctypes.c_void_p), ctypes.cast(lv, ctypes.c_void_p),
                      ctypes.cast(lo, ctypes.c_void_p), ctypes.cast(ed, ctypes.c_void_p), 1, 0, 1, 0)
    lib.p2p_fail_host_allocs(1)
    b = ctypes.c_void_p()
    assert lib.p2p_batch_create(*args(b)) == 3 and not b.value
    assert lib.p2p_batch_create(*args(b)) == 0 and b.value
    assert lib.p2p_batch_destroy(b) == 0
    lib.p2p_fail_host_allocs(2)
    lib.p2p_fail_host_allocs(0)                  # clears
    st, h = _create(lib)
    assert st == 0 and h.value
    lib.p2p_plan_destroy(h)


def test_checked_variant_exports_the_same_symbols():
    path = cuda_build.build(variants=("checked",))
    chk = ctypes.CDLL(path)
    assert chk.p2p_build_checked() == 1
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing

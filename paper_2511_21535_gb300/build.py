"""Build the CUDA library in-tree for sm_103a (GB300).

Each .cu file is compiled to an object in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a), then linked into
``paper_2511_21535_gb300/_lib/libp2p_gb300.so``.  A second variant,
``libp2p_gb300_checked.so``, is the same sources with ``-DP2P_CHECKED``: its
kernels check every work item's ranges, slots and indices against the plan's
capacities and record P2P_FLAG_BOUNDS instead of touching memory out of range
(the tests run randomized plans through it).  Rebuilds only when a source or
header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libp2p_gb300.so")
VARIANTS = {"release": (LIB, "obj", []),
            "checked": (os.path.join(OUT_DIR, "libp2p_gb300_checked.so"), "obj_checked", ["-DP2P_CHECKED"])}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-v"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date(variant: str = "release") -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, obj: str, extra: list, verbose: bool) -> str:
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr if verbose else ""


def _link(lib: str, objs: list) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          variants: tuple = ("release",)) -> str:
    """Compile every CUDA source for each requested variant (one shared pool of
    nvcc processes) and link the libraries; return the first library's path."""
    todo = [v for v in variants if force or not up_to_date(v)]
    srcs = _sources()
    units = []
    for v in todo:
        lib, sub, extra = VARIANTS[v]
        obj_dir = os.path.join(OUT_DIR, sub)
        os.makedirs(obj_dir, exist_ok=True)
        units += [(s, os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o"), extra) for s in srcs]
    if units:
        jobs = jobs or min(len(units), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            logs = list(ex.map(lambda u: _compile(u[0], u[1], u[2], verbose), units))
        if verbose:
            for u, log in zip(units, logs):
                print(f"== {os.path.basename(u[1])}\n{log}")
        for v in todo:
            lib, sub, _ = VARIANTS[v]
            _link(lib, [os.path.join(OUT_DIR, sub, os.path.basename(s)[:-3] + ".o") for s in srcs])
    return VARIANTS[variants[0]][0]


def build_all(force: bool = False, verbose: bool = False) -> str:
    """The release library and its checked variant."""
    return build(force=force, verbose=verbose, variants=tuple(VARIANTS))


if __name__ == "__main__":
    import sys
    print(build_all(force="--force" in sys.argv, verbose="-v" in sys.argv))

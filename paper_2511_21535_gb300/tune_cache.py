"""Persistent cache of the batch autotuner's choices.

The autotuner (``p2p_batch_autotune``) times every layout / targets-per-lane
/ tile / warps-per-item combination on the caller's data, which costs a few
hundred launches.  Its choice depends on the GPU, on the shape of the batch
and on the kernels, so the cache keys an entry by the device name, a shape
class (instance count, total and largest instance size rounded to powers of
two, right-hand sides, forward+adjoint pairing) and a hash of the CUDA
sources; an entry written by other kernels is never used.  Entries live in
one JSON file (``$P2P_GB300_TUNE_CACHE``, else
``~/.cache/p2p_gb300/autotune.json``), rewritten atomically.
"""
from __future__ import annotations

import glob
import hashlib
import json
import math
import os
import tempfile

_CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
_version = None


def kernel_version() -> str:
    """Hash of every CUDA source and header of the library (16 hex digits)."""
    global _version
    if _version is None:
        h = hashlib.sha256()
        for f in sorted(glob.glob(os.path.join(_CSRC, "*.cu")) + glob.glob(os.path.join(_CSRC, "*.cuh"))):
            h.update(os.path.basename(f).encode())
            h.update(open(f, "rb").read())
        _version = h.hexdigest()[:16]
    return _version


def shape_class(sizes, nrhs: int, pair: bool) -> str:
    """Batches in one class share a tuning: instance count, total and largest
    instance size (nearest power of two), right-hand sides, pairing."""
    total, largest = int(sum(sizes)), int(max(sizes))
    return (f"i{len(sizes)}-n2^{round(math.log2(max(total, 1)))}-max2^{round(math.log2(max(largest, 1)))}"
            f"-r{int(nrhs)}-{'pair' if pair else 'fwd'}")


def default_path() -> str:
    return os.environ.get("P2P_GB300_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "p2p_gb300",
                                                                  "autotune.json")


class TuneCache:
    def __init__(self, path: str | None = None):
        self.path = path or default_path()

    @staticmethod
    def key(device_name: str, shape: str) -> str:
        return f"{device_name}|{shape}|{kernel_version()}"

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                data = json.load(f)
            return data if isinstance(data, dict) else {}
        except (OSError, ValueError):
            return {}

    def get(self, key: str):
        entry = self._load().get(key)
        return dict(entry) if isinstance(entry, dict) else None

    def put(self, key: str, value: dict) -> None:
        data = self._load()
        data[key] = dict(value)
        d = os.path.dirname(self.path) or "."
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".autotune.", dir=d)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise

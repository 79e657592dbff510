"""Seeded synthetic inputs for the near-field (P2P) operator.

This module only draws random numbers and lays out sample grids.  It holds
none of the operator's arithmetic (no boxing, no kernels), so both the CUDA
path and the FP64 oracle can be fed from it without sharing method code.

The paper's workloads are a uniform 2-D EM mesh (DBIM-MLFMA, Section 5.1) and
clustered stellar particles (PhotoNs-2.0, Section 5.2, dataset not public).
They are stood in for by five synthetic configurations:

  uniform_gravity     8,192 points uniform in [0,1)^3, masses U(0.5,1.5),
                      level 3, Plummer eps 1e-3
  grid_helmholtz      64^3 grid at spacing lambda/10, k = 2*pi, 4^3 leaf
                      boxes, complex64 sources N(0,1), one right-hand side
  plummer_gravity     4,194,304 points: Plummer sphere (a = 0.05, centre
                      (0.5,0.5,0.5), truncated to the unit cube) plus 10 %
                      uniform background, level 7, eps 1e-4
  batched_helmholtz   64 grids with edges drawn from {16,24,32,48,64}, 8 RHS
  diff_helmholtz      128^3 grid, contrast chi in a centred sphere, plane wave

Every array is float32 (complex64 for complex data), C-contiguous, in
"original" particle order.  Grid point (ix, iy, iz) has index
ix + E*(iy + E*iz) and sits at ((ix+1/2)h, (iy+1/2)h, (iz+1/2)h).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WAVELENGTH = 1.0
SPACING = 0.1                       # lambda / 10
WAVENUMBER = 2.0 * math.pi / WAVELENGTH
LEAF_EDGE_POINTS = 4                # 4^3 points per leaf box


@dataclasses.dataclass
class Problem:
    """One P2P instance: particles plus the boxing domain and kernel constant."""
    name: str
    pos: np.ndarray                 # float32 [n, 3]
    strength: np.ndarray            # float32 [n] (mass) or complex64 [nrhs, n]
    level: int
    lo: tuple                       # boxing domain lower corner (float32 values)
    edge: float                     # boxing domain edge length (float32 value)
    kind: str                       # "gravity" | "helmholtz"
    eps: float = 0.0                # Plummer softening (gravity)
    k: float = 0.0                  # wavenumber (helmholtz)
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nrhs(self) -> int:
        return 1 if self.kind == "gravity" else int(self.strength.shape[0])


# ----------------------------------------------------------------------------
# primitive generators
# ----------------------------------------------------------------------------

def uniform_points(n: int, rng: np.random.Generator) -> np.ndarray:
    """n points uniform in [0,1)^3, drawn directly as float32."""
    return rng.random((n, 3), dtype=np.float32)


def plummer_points(n: int, a: float, centre, rng: np.random.Generator) -> np.ndarray:
    """n points of a Plummer sphere of scale radius a, kept only inside [0,1)^3.

    Radius by inverse-CDF sampling of the Plummer cumulative mass
    M(<r)/M = r^3 / (r^2 + a^2)^{3/2}:  r = a / sqrt(X^{-2/3} - 1), X ~ U(0,1);
    isotropic direction.  Points outside the unit cube (after rounding to
    float32) are redrawn.
    """
    c = np.asarray(centre, np.float64)
    out = np.empty((n, 3), np.float32)
    filled = 0
    while filled < n:
        m = n - filled
        x = rng.random(m)
        x = np.clip(x, 1e-300, None)
        r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        cos_t = rng.uniform(-1.0, 1.0, m)
        phi = rng.uniform(0.0, 2.0 * math.pi, m)
        sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
        p = np.stack([r * sin_t * np.cos(phi), r * sin_t * np.sin(phi), r * cos_t], axis=1) + c
        p32 = p.astype(np.float32)
        ok = np.all((p32 >= np.float32(0.0)) & (p32 < np.float32(1.0)), axis=1)
        p32 = p32[ok]
        out[filled:filled + p32.shape[0]] = p32
        filled += p32.shape[0]
    return out


def grid_points(edge_points: int, h: float = SPACING) -> np.ndarray:
    """Regular grid of edge_points^3 points at ((i+1/2)h, ...), index ix + E*(iy + E*iz)."""
    e = int(edge_points)
    i = (np.arange(e, dtype=np.float64) + 0.5) * h
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)


def grid_domain(edge_points: int, h: float = SPACING, leaf: int = LEAF_EDGE_POINTS):
    """Octree level and boxing domain for a grid with `leaf`^3-point leaf boxes.

    The root box is the smallest power-of-two multiple of the leaf box that
    covers the grid, anchored at the origin; leaf boxes beyond the grid stay
    empty.  Returns (level, lo, edge) with edge a float32 value.
    """
    boxes = -(-int(edge_points) // leaf)
    level = max(1, int(math.ceil(math.log2(boxes))))
    edge = float(np.float32((1 << level) * leaf * h))
    return level, (0.0, 0.0, 0.0), edge


def complex_normal(shape, rng: np.random.Generator) -> np.ndarray:
    """complex64 array with real and imaginary parts i.i.d. N(0,1)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(np.complex64)


# ----------------------------------------------------------------------------
# the five configurations
# ----------------------------------------------------------------------------

def uniform_gravity(n: int = 8192, level: int = 3, eps: float = 1e-3, seed: int = 0) -> Problem:
    rng = np.random.default_rng(seed)
    pos = uniform_points(n, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return Problem("uniform_gravity", pos, mass, level, (0.0, 0.0, 0.0), 1.0, "gravity",
                   eps=float(np.float32(eps)))


def grid_helmholtz(edge_points: int = 64, nrhs: int = 1, seed: int = 0,
                   k: float = WAVENUMBER) -> Problem:
    rng = np.random.default_rng(seed)
    pos = grid_points(edge_points)
    q = complex_normal((nrhs, pos.shape[0]), rng)
    level, lo, edge = grid_domain(edge_points)
    return Problem(f"grid_helmholtz_{edge_points}", pos, q, level, lo, edge, "helmholtz",
                   k=float(np.float32(k)), extra={"edge_points": edge_points})


def plummer_gravity(n: int = 4_194_304, background: float = 0.10, a: float = 0.05,
                    level: int = 7, eps: float = 1e-4, seed: int = 0) -> Problem:
    rng = np.random.default_rng(seed)
    n_bg = int(n * background)
    n_pl = n - n_bg
    pl = plummer_points(n_pl, a, (0.5, 0.5, 0.5), rng)
    bg = uniform_points(n_bg, rng)
    pos = np.ascontiguousarray(np.concatenate([pl, bg], axis=0))
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return Problem("plummer_gravity", pos, mass, level, (0.0, 0.0, 0.0), 1.0, "gravity",
                   eps=float(np.float32(eps)))


BATCH_EDGES = (16, 24, 32, 48, 64)


def batched_helmholtz(instances: int = 64, nrhs: int = 8, seed: int = 0,
                      edges=BATCH_EDGES) -> list:
    """`instances` grid problems, edges drawn uniformly from `edges`, nrhs RHS each."""
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(edges), instances)
    out = []
    for i, p in enumerate(picks):
        e = int(edges[int(p)])
        pos = grid_points(e)
        q = complex_normal((nrhs, pos.shape[0]), rng)
        level, lo, edge = grid_domain(e)
        out.append(Problem(f"batch_{i}_{e}", pos, q, level, lo, edge, "helmholtz",
                           k=float(np.float32(WAVENUMBER)), extra={"edge_points": e}))
    return out


def contrast_sphere(edge_points: int, radius_frac: float, rng: np.random.Generator) -> np.ndarray:
    """complex64 contrast: Re, Im i.i.d. 0.1*U(0,1) inside the centred sphere of
    radius radius_frac * (grid extent), 0 outside."""
    pos = grid_points(edge_points).astype(np.float64)
    extent = edge_points * SPACING
    c = 0.5 * extent
    inside = np.sum((pos - c) ** 2, axis=1) <= (radius_frac * extent) ** 2
    n = pos.shape[0]
    re = 0.1 * rng.random(n)
    im = 0.1 * rng.random(n)
    chi = np.where(inside, re + 1j * im, 0.0).astype(np.complex64)
    return chi


def plane_wave(pos: np.ndarray, k: float) -> np.ndarray:
    """Incident field exp(i k x) along +x, complex64 (input data, evaluated in FP64)."""
    x = pos[:, 0].astype(np.float64)
    return np.exp(1j * float(k) * x).astype(np.complex64)


def diff_helmholtz(edge_points: int = 128, seed: int = 0, data_seed: int = 1,
                   fd_seed: int = 2, fd_entries: int = 16) -> Problem:
    """Differentiable configuration: chi (seed), the data contrast chi2 (data_seed),
    plane-wave incident field, and `fd_entries` random inside-sphere indices (fd_seed)."""
    pos = grid_points(edge_points)
    k = float(np.float32(WAVENUMBER))
    chi = contrast_sphere(edge_points, 0.3, np.random.default_rng(seed))
    chi2 = contrast_sphere(edge_points, 0.3, np.random.default_rng(data_seed))
    uinc = plane_wave(pos, k)
    inside = np.nonzero(chi != 0)[0]
    fd_idx = np.random.default_rng(fd_seed).choice(inside, fd_entries, replace=False)
    level, lo, edge = grid_domain(edge_points)
    # strength holds the contrast; the operator's source is chi * u_inc, formed by the method
    return Problem(f"diff_helmholtz_{edge_points}", pos, chi[None, :].copy(), level, lo, edge,
                   "helmholtz", k=k,
                   extra={"chi": chi, "chi2": chi2, "uinc": uinc, "fd_idx": np.sort(fd_idx),
                          "edge_points": edge_points})


CONFIGS = {
    "uniform_gravity": uniform_gravity,
    "grid_helmholtz": grid_helmholtz,
    "plummer_gravity": plummer_gravity,
    "batched_helmholtz": batched_helmholtz,
    "diff_helmholtz": diff_helmholtz,
}

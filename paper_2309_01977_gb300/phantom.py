"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the projector or of OSEM: it draws shapes,
scales an activity map to a requested count level given a forward projection
computed by the caller, and draws Poisson counts.  Everything is numpy with a
PCG64 generator seeded explicitly.

Phantom recipe (the paper's clinical and SIMIND data are not available; these
shapes stand in for them with the paper's acquisition sizes, Sec. 3.1 and the
appendix: 128 transaxial bins, 4.8 mm pixels, 60/96/120 projections):
  - water cylinder along z, radius 0.4*n, length 0.8*nz, activity 1;
  - five axis-aligned ellipsoids, full axis lengths U[5, 20] * n/64 voxels,
    centres uniform inside the cylinder shrunk by the largest semi-axis,
    activity U[0.5, 5], each overwriting what is under it, in order;
  - mu = 0.15 /cm inside the cylinder, one more seeded ellipsoid of bone at
    0.25 /cm, 0 outside.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Tuple

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One acquisition/reconstruction configuration."""

    name: str
    n: int
    nz: int
    n_angles: int
    n_iters: int
    n_subsets: int
    counts: float
    seed: int
    voxel_cm: float = 0.48
    sigma0: float = 0.5
    slope: float = 0.03
    nsigma: float = 3.0
    scatter_frac: float = 0.05


# The configurations the library is exercised on (sizes of the paper's SPECT
# acquisitions: 60, 96 and 120 projections of 128 x 128 bins at 4.8 mm).
WORKLOADS = {
    "osem64": Workload("osem64", 64, 64, 64, 2, 8, 2e6, 1),
    "osem128": Workload("osem128", 128, 128, 120, 4, 8, 1e7, 2),
    "serve64": Workload("serve64", 64, 64, 60, 2, 8, 1e6, 1000),
    "serve96": Workload("serve96", 96, 96, 96, 2, 8, 1e6, 1000),
    "serve128": Workload("serve128", 128, 128, 120, 2, 8, 1e6, 1000),
    "grad192": Workload("grad192", 192, 192, 128, 1, 1, 1e7, 5),
}


def _grid(n: int, nz: int):
    c = 0.5 * (n - 1)
    cz = 0.5 * (nz - 1)
    x = np.arange(n, dtype=np.float64)[:, None, None] - c
    y = np.arange(n, dtype=np.float64)[None, :, None] - c
    z = np.arange(nz, dtype=np.float64)[None, None, :] - cz
    return x, y, z


def _ellipsoid(rng, n, nz, radius, half_len, scale):
    axes = rng.uniform(5.0, 20.0, size=3) * scale          # full axis lengths (voxels)
    semi = 0.5 * axes
    big = semi.max()
    # centre uniform inside the cylinder shrunk by the largest semi-axis
    r_in = max(radius - big, 0.0)
    while True:
        cx, cy = rng.uniform(-r_in, r_in, size=2)
        if cx * cx + cy * cy <= r_in * r_in:
            break
    zl = max(half_len - big, 0.0)
    cz = rng.uniform(-zl, zl)
    return (cx, cy, cz), semi


def make_phantom(n: int, nz: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """Activity f (arbitrary units, before count scaling) and mu (1/cm), both [n][n][nz] float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y, z = _grid(n, nz)
    radius = 0.4 * n
    half_len = 0.4 * nz
    scale = n / 64.0
    cyl = (x * x + y * y <= radius * radius) & (np.abs(z) <= half_len)
    f = np.where(cyl, 1.0, 0.0)
    for _ in range(5):
        (cx, cy, cz), semi = _ellipsoid(rng, n, nz, radius, half_len, scale)
        act = rng.uniform(0.5, 5.0)
        inside = ((x - cx) / semi[0]) ** 2 + ((y - cy) / semi[1]) ** 2 + ((z - cz) / semi[2]) ** 2 <= 1.0
        f = np.where(inside, act, f)
    mu = np.where(cyl, 0.15, 0.0)
    (cx, cy, cz), semi = _ellipsoid(rng, n, nz, radius, half_len, scale)
    bone = ((x - cx) / semi[0]) ** 2 + ((y - cy) / semi[1]) ** 2 + ((z - cz) / semi[2]) ** 2 <= 1.0
    mu = np.where(bone, 0.25, mu)
    return f.astype(np.float64), mu.astype(np.float64)


def make_counts(f_raw: np.ndarray, hf_raw: np.ndarray, counts: float, scatter_frac: float, seed: int):
    """Scale the activity so that sum(H f_true) == counts, then draw y ~ Poisson(H f_true + s).

    hf_raw is the caller's forward projection of f_raw (all angles).  The
    scatter term s is a constant equal to scatter_frac times the mean bin of
    H f_true.  Returns (f_true, y, s, ybar) with y as float64 counts.
    """
    total = float(np.sum(hf_raw, dtype=np.float64))
    if not total > 0.0:
        raise ValueError("forward projection of the phantom is empty")
    scale = counts / total
    f_true = f_raw * scale
    hf = np.asarray(hf_raw, dtype=np.float64) * scale
    s = scatter_frac * float(hf.mean())
    ybar = hf + s
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    y = rng.poisson(ybar).astype(np.float64)
    return f_true, y, s, ybar


def random_volume(shape, seed: int, low: float = 0.0, high: float = 1.0) -> np.ndarray:
    """Uniform random test volume (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(low, high, size=shape)

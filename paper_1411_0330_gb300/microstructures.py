"""Seeded synthetic microstructures (geometry only).

This module produces phase maps, sphere packings and per-voxel scale fields
with the shapes and statistics of the workloads of Sec. 5 of Brisard &
Legoll (arXiv:1411.0330): a periodic unit cell Q = (0,1)^d split into N^d
voxels, spherical inclusions voxelised by the centre rule (a voxel belongs to
an inclusion when its centre lies inside it, Sec. 5).  It holds none of the
method's arithmetic; both the CUDA path and the oracle receive its outputs as
plain arrays.

Array conventions: phase maps are uint8 arrays of shape (N2, N1, N0) in 3D or
(N1, N0) in 2D (numpy C order, so axis 0 of the paper's beta is the fastest).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["square_inclusion", "laminate", "rsa_spheres", "hard_sphere_mc", "voxelize_spheres",
           "sphere_microstructure", "scale_field", "random_field", "sphere_volume"]


def square_inclusion(n: int = 32, side: float = 0.5) -> np.ndarray:
    """2D cell with a centred square inclusion (phase 1) of the given side."""
    c = (np.arange(n) + 0.5) / n
    inside = np.abs(c - 0.5) <= side / 2 + 1e-12
    return (inside[:, None] & inside[None, :]).astype(np.uint8)


def laminate(shape, axis: int, widths) -> np.ndarray:
    """Layered cell: phase id varies along `axis` (0 = fastest axis) only.

    widths: sequence of (phase, number of voxels) repeated until the axis is
    filled exactly.
    """
    shape = tuple(shape)
    n_ax = shape[len(shape) - 1 - axis]
    prof = []
    while len(prof) < n_ax:
        for ph, w in widths:
            prof.extend([ph] * w)
    prof = np.asarray(prof[:n_ax], dtype=np.uint8)
    bshape = [1] * len(shape)
    bshape[len(shape) - 1 - axis] = n_ax
    return np.broadcast_to(prof.reshape(bshape), shape).copy()


def sphere_volume(r: float) -> float:
    return 4.0 / 3.0 * math.pi * r ** 3


def _min_image(d: np.ndarray) -> np.ndarray:
    return d - np.round(d)


def rsa_spheres(radius: float, fraction: float, seed: int, max_tries: int = 2_000_000,
                gap: float = 0.0) -> np.ndarray:
    """Random sequential addition of non-overlapping spheres in the periodic unit cube.

    Returns centres (k, 3) in unit-cell coordinates, with k = round(fraction /
    sphere_volume(radius)) or fewer if the packing jams first.
    """
    rng = np.random.default_rng(seed)
    target = int(round(fraction / sphere_volume(radius)))
    cen = np.empty((target, 3))
    k = 0
    dmin2 = (2 * radius + gap) ** 2
    tries = 0
    while k < target and tries < max_tries:
        batch = rng.random((256, 3))
        for c in batch:
            tries += 1
            if k == 0 or np.min(np.sum(_min_image(cen[:k] - c) ** 2, axis=1)) >= dmin2:
                cen[k] = c
                k += 1
                if k == target:
                    break
    return cen[:k].copy()


def hard_sphere_mc(radius: float, count: int, seed: int, sweeps: int = 30) -> np.ndarray:
    """Hard-sphere Monte Carlo in the periodic unit cube (the kind of packing of Sec. 5).

    Start from `count` random sites of a face-centred cubic lattice fine
    enough not to overlap, then apply `sweeps` rounds of random displacement
    moves, each rejected if it creates an overlap.
    """
    rng = np.random.default_rng(seed)
    m = max(1, math.ceil((count / 4) ** (1 / 3)))
    while (1.0 / m) / math.sqrt(2.0) < 2 * radius and m > 1:
        m -= 1
    if 4 * m ** 3 < count or (1.0 / m) / math.sqrt(2.0) < 2 * radius:
        raise ValueError("fraction too high for this radius")
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    sites = ((g[:, None, :] + base[None, :, :]).reshape(-1, 3) + 0.25) / m
    cen = sites[rng.permutation(len(sites))[:count]].copy() % 1.0
    dmin2 = (2 * radius) ** 2
    step = radius
    for _ in range(sweeps):
        acc = 0
        for i in rng.permutation(count):
            trial = (cen[i] + rng.uniform(-step, step, 3)) % 1.0
            d2 = np.sum(_min_image(cen - trial) ** 2, axis=1)
            d2[i] = np.inf
            if np.min(d2) >= dmin2:
                cen[i] = trial
                acc += 1
        rate = acc / count
        step *= 1.2 if rate > 0.5 else 0.8
        step = min(max(step, 1e-4), 0.5)
    return cen


def voxelize_spheres(n, centres: np.ndarray, radius: float, phase_in: int = 1) -> np.ndarray:
    """Centre rule on an n^3 grid (or n = (n0, n1, n2)): a voxel is inside when the
    periodic minimum-image distance from its centre to a sphere centre is <= radius."""
    n0, n1, n2 = (n, n, n) if np.isscalar(n) else tuple(n)
    out = np.zeros((n2, n1, n0), dtype=np.uint8)
    ns = np.array([n0, n1, n2])
    for c in centres:
        lo = np.floor((c - radius) * ns - 0.5).astype(int) - 1
        hi = np.ceil((c + radius) * ns - 0.5).astype(int) + 1
        ax = [np.arange(lo[i], hi[i] + 1) for i in range(3)]
        d = [_min_image((ax[i] + 0.5) / ns[i] - c[i]) ** 2 for i in range(3)]
        inside = (d[2][:, None, None] + d[1][None, :, None] + d[0][None, None, :]) <= radius ** 2 + 1e-15
        iz, iy, ix = np.nonzero(inside)
        out[ax[2][iz] % n2, ax[1][iy] % n1, ax[0][ix] % n0] = phase_in
    return out


def sphere_microstructure(n: int, radius_vox: float, fraction: float, seed: int, method: str = "auto"):
    """Two-phase sphere packing on an n^3 grid.  Returns (phase map, centres, radius)."""
    r = radius_vox / n
    if method == "auto":
        method = "rsa" if fraction <= 0.3 else "mc"
    if method == "rsa":
        cen = rsa_spheres(r, fraction, seed)
    else:
        cen = hard_sphere_mc(r, int(round(fraction / sphere_volume(r))), seed)
    return voxelize_spheres(n, cen, r), cen, r


def sphere_fractions(n, centres: np.ndarray, radius: float, sub: int = 4) -> np.ndarray:
    """Volume fraction of the union of spheres in each voxel of an n^3 grid,
    estimated on a regular sub^3 lattice of points per voxel (point in a sphere:
    periodic minimum-image distance <= radius).  float32, shape (n, n, n)."""
    fine = voxelize_spheres(n * sub, centres, radius).astype(np.float32)
    return fine.reshape(n, sub, n, sub, n, sub).mean(axis=(1, 3, 5)).astype(np.float32)


def scale_field(shape, seed: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Per-voxel stiffness scale s ~ U(lo, hi), float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(shape)).astype(np.float32)


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard normal test field."""
    return np.random.default_rng(seed).standard_normal(tuple(shape)).astype(dtype)

"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it draws particles, charges
and multipole vectors from fixed seeds and bins particles into the integer
cells of a uniform-depth octree.  Both the tests (for the CPU oracle and for
the CUDA path) and the benchmark draw their inputs from here.

The paper's workloads are particles scattered at random on sphere and
spheroid surfaces (Sec. 5, "Example geometries"); the shapes below follow
that recipe on the cube [-1, 1]^3.
"""
from __future__ import annotations

import numpy as np

DOMAIN_LO = -1.0
DOMAIN_WIDTH = 2.0


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_cube(n: int, seed: int):
    """n points U([-1, 1]^3) and charges U(-1, 1)."""
    g = rng(seed)
    pts = g.uniform(-1.0, 1.0, (n, 3))
    q = g.uniform(-1.0, 1.0, n)
    return pts, q


def ellipsoid_surface(n: int, axes=(1.0, 0.5, 0.25), seed: int = 3):
    """n points area-uniform on the ellipsoid surface with the given semi-axes
    (rejection sampling of the sphere map), charges N(0, 1)."""
    g = rng(seed)
    a = np.asarray(axes, dtype=np.float64)
    out = np.empty((0, 3))
    # acceptance weight: area element of the ellipsoid relative to the sphere, up to a constant
    wmax = np.max([a[1] * a[2], a[0] * a[2], a[0] * a[1]])
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 1024
        u = g.standard_normal((m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        wgt = np.sqrt((a[1] * a[2] * u[:, 0]) ** 2 + (a[0] * a[2] * u[:, 1]) ** 2
                      + (a[0] * a[1] * u[:, 2]) ** 2)
        keep = g.uniform(0.0, wmax, m) < wgt
        out = np.concatenate([out, u[keep] * a[None, :]])
    pts = out[:n] * 0.999  # stay strictly inside the unit cube
    q = g.standard_normal(n)
    return pts, q


def sphere_surface(n: int, seed: int, radius: float = 0.999):
    """n points uniform on a sphere of the given radius, charges N(0, 1)."""
    g = rng(seed)
    u = g.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return radius * u, g.standard_normal(n)


def gaussian_vectors(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """rows x cols i.i.d. N(0, 1) values (multipole vectors, loss weights)."""
    return rng(seed).standard_normal((rows, cols)).astype(dtype)


def full_grid(level: int) -> np.ndarray:
    """[8^level, 3] int32 integer coordinates of a full level, x fastest."""
    n = 1 << level
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.ascontiguousarray(np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int32))


def occupied_cells(pts: np.ndarray, level: int) -> np.ndarray:
    """[n, 3] int32 coordinates of the non-empty cells at `level`, x fastest."""
    n = 1 << level
    w = DOMAIN_WIDTH / n
    ijk = np.clip(np.floor((np.asarray(pts) - DOMAIN_LO) / w).astype(np.int64), 0, n - 1)
    lin = np.unique(ijk[:, 0] + n * ijk[:, 1] + n * n * ijk[:, 2])
    return np.ascontiguousarray(np.stack([lin % n, (lin // n) % n, lin // (n * n)], axis=1).astype(np.int32))


def batched_tree_specs(ntrees: int = 64, seed: int = 4):
    """Per-tree parameters of the batched workload: N log-uniform in [1e4, 1e6],
    geometry alternating uniform cube / sphere surface, leaf level
    clamp(round(log_8(N / 64)), 3, 6), order ell uniform in {4, 5, 6}."""
    g = rng(seed)
    specs = []
    for i in range(ntrees):
        n = int(round(10.0 ** g.uniform(4.0, 6.0)))
        leaf = int(np.clip(np.round(np.log(n / 64.0) / np.log(8.0)), 3, 6))
        ell = int(g.integers(4, 7))
        specs.append({"n": n, "geometry": "cube" if i % 2 == 0 else "sphere", "leaf_level": leaf,
                      "ell": ell, "seed": 1000 + i})
    return specs


def tree_points(spec):
    if spec["geometry"] == "cube":
        return uniform_cube(spec["n"], spec["seed"])
    return sphere_surface(spec["n"], spec["seed"])

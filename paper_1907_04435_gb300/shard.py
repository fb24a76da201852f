"""Receivers split across ranks: host-side plumbing of the multi-GPU path.

Receivers are independent of one another: each one's shadowed steps depend only on the
scene and the sun (Sec. 4, Step 2 tests each receiver against the map on its own; Sec. 5
traces each receiver's own rays).  So one workload shards by receivers with the scene and
its BVH built on every rank, no exchange while computing, and one gather of the results:
  - facade points: contiguous index ranges of balanced sizes, in input order;
  - a ground grid: bands of whole rows.  A band is a grid of its own whose origin is the
    parent's origin moved by the band's first row, and its cell centres must round to the
    parent's in FP32 (they do for integer steps and origins, as in the district, 1 m
    cells at integer coordinates); `grid_band` refuses a band whose centres would not.
The results gather on rank 0 in rank order, which is input order.  Nothing here computes
shadows: every rank calls the library on its own receivers.
"""
from __future__ import annotations

import numpy as np


def split(n: int, rank: int, world: int) -> tuple[int, int]:
    """[a, b): rank's share of n items, contiguous, sizes differing by at most one (the
    larger shares first)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad split")
    base, rem = divmod(n, world)
    a = rank * base + min(rank, rem)
    return a, a + base + (1 if rank < rem else 0)


def _centres(o: float, dx: float, first: int, count: int) -> np.ndarray:
    """FP32 cell centres o + (i + 0.5) dx for i in [first, first + count), rounded as the
    library rounds them (each operation once, in FP32)."""
    i = np.arange(first, first + count, dtype=np.float32)
    return np.float32(o) + (i + np.float32(0.5)) * np.float32(dx)


def grid_band(grid, rank: int, world: int):
    """Rank's band of rows of grid (x0, y0, dx, nx, ny): (x0, y0', dx, nx, rows, row0), the
    band as a grid of its own and its first row in the parent.  Raises ValueError if the
    band's FP32 cell centres differ from the parent's."""
    x0, y0, dx, nx, ny = grid
    r0, r1 = split(int(ny), rank, world)
    y0b = float(np.float32(np.float32(y0) + np.float32(r0) * np.float32(dx)))
    if r1 > r0 and not np.array_equal(_centres(y0b, dx, 0, r1 - r0), _centres(y0, dx, r0, r1 - r0)):
        raise ValueError("grid_band: the band's cell centres do not round to the grid's; "
                         "use an origin and cell size on which they do (e.g. integers)")
    return float(x0), y0b, float(dx), int(nx), r1 - r0, r0


def gather_to_root(parts, dist=None):
    """Concatenates each rank's list of 1-D host arrays on rank 0, in rank order (None on
    the other ranks); the list itself when not distributed."""
    parts = [np.ascontiguousarray(p) for p in parts]
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return parts
    world, rank = dist.get_world_size(), dist.get_rank()
    got = [None] * world if rank == 0 else None
    dist.gather_object(parts, got, dst=0)
    if rank != 0:
        return None
    return [np.concatenate([g[k] for g in got]) for k in range(len(parts))]

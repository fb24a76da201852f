"""The synthetic workloads, by name (seeded, deterministic).

  boxes16     4 x 4 boxes, 64 x 64 ground receivers at 2 m, 21 Jun 09-17 h @ 2 min (241 steps)
  district    2,000 convex buildings (~60k triangles), 2048^2 ground at 1 m + 1M facade
              samples, 21 Jun 09-17 h @ 1 min (481 steps)
  season      50,000 buildings (~1.5M triangles), central 4096^2 ground at 1 m,
              92 days (21 Jun - 20 Sep) x 481 steps
  park        500 x 300 m park at 0.5 m (600k receivers) ringed by 200 buildings
              (median 60 m), equinox 09-17 h @ 1 min
  district_small / facade_small   parity-sized cases with ragged tails

All at latitude 40.7 N.  The paper's Manhattan mesh is not available; these stand in
for it (same building count and triangle scale for `season`).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import city as C
from .sun import SunTable, sun_table

LAT = 40.7


@dataclass
class Workload:
    name: str
    city: C.City
    mesh: C.Mesh
    ground: C.GroundGrid | None
    facade_pos: np.ndarray | None      # float32 [Rf, 3]
    facade_nrm: np.ndarray | None      # float32 [Rf, 3]
    sun: SunTable

    @property
    def R(self) -> int:
        g = self.ground.R if self.ground is not None else 0
        f = 0 if self.facade_pos is None else int(self.facade_pos.shape[0])
        return g + f


def boxes16(seed_off: int = 1) -> Workload:
    city = C.city_boxes(C.SEED_BASE + seed_off)
    extent = 4 * 55.0 - 15.0
    g = C.GroundGrid(x0=extent / 2 - 64.0, y0=extent / 2 - 64.0, dx=2.0, nx=64, ny=64)
    sun = sun_table(LAT, [172], 9.0, 17.0, 2.0)
    return Workload("boxes16", city, C.extrude(city), g, None, None, sun)


def district(n_facade: int = 1_000_000, with_ground: bool = True, seed_off: int = 2) -> Workload:
    city = C.city_district(C.SEED_BASE + seed_off)
    g = C.GroundGrid(x0=0.0, y0=0.0, dx=1.0, nx=2048, ny=2048) if with_ground else None
    fp, fn = (C.facade_samples(city, n_facade, C.SEED_BASE + 100 + seed_off)
              if n_facade else (None, None))
    sun = sun_table(LAT, [172], 9.0, 17.0, 1.0)
    return Workload("district", city, C.extrude(city), g, fp, fn, sun)


def season(n_days: int = 92, ground_n: int = 4096) -> Workload:
    city = C.city_district(C.SEED_BASE + 3, extent=10240.0, n_buildings=50_000)
    off = (10240.0 - ground_n) / 2
    g = C.GroundGrid(x0=off, y0=off, dx=1.0, nx=ground_n, ny=ground_n)
    sun = sun_table(LAT, list(range(172, 172 + n_days)), 9.0, 17.0, 1.0)
    return Workload("season", city, C.extrude(city), g, None, None, sun)


def park(width: float = 500.0, depth: float = 300.0, dx: float = 0.5, n_buildings: int = 200,
         band: float = 300.0, step: float = 1.0, seed_off: int = 5) -> Workload:
    """A width x depth park sampled at dx, ringed by c2-style buildings (median 60 m)."""
    city = C.city_ring_around_park(C.SEED_BASE + seed_off, park=(0.0, 0.0, width, depth),
                                   band=band, n_buildings=n_buildings)
    g = C.GroundGrid(x0=0.0, y0=0.0, dx=dx, nx=int(round(width / dx)), ny=int(round(depth / dx)))
    sun = sun_table(LAT, [79], 9.0, 17.0, step)
    return Workload("park", city, C.extrude(city), g, None, None, sun)


def district_small(seed_off: int = 6, n_buildings: int = 120, extent: float = 520.0,
                   nx: int = 200, ny: int = 150, dx: float = 2.5, n_facade: int = 3001,
                   doys=(172,), t0: float = 9.0, t1: float = 17.0, step: float = 4.0) -> Workload:
    """A few hundred metres of district: several 32 x 32 tiles with ragged edges."""
    city = C.city_district(C.SEED_BASE + seed_off, extent=extent, n_buildings=n_buildings)
    g = C.GroundGrid(x0=8.25, y0=6.75, dx=dx, nx=nx, ny=ny)
    fp, fn = (C.facade_samples(city, n_facade, C.SEED_BASE + 200 + seed_off)
              if n_facade else (None, None))
    sun = sun_table(LAT, list(doys), t0, t1, step)
    return Workload("district_small", city, C.extrude(city), g, fp, fn, sun)


BY_NAME = {"boxes16": boxes16, "district": district, "season": season, "park": park,
           "district_small": district_small}


# ------------------------------------------------------------------ batched scenarios
@dataclass
class Scenarios:
    """Development variants of a base city: each adds towers and removes the base
    buildings whose footprints they overlap; each has a square receiver region (cells of
    the base ground grid) around its towers; the same sun intervals apply to all."""
    base: Workload
    tower_tris: list          # per variant: float32 [n, 9] tower triangles (12 per tower)
    removed: list             # per variant: int32 base building ids removed
    regions: np.ndarray       # int32 [V, 4]: ix0, iy0, nx, ny (clipped to the grid)
    intervals: list           # SunTable per interval

    @property
    def V(self) -> int:
        return len(self.tower_tris)

    def variant_mesh(self, v: int):
        """Triangle soup [T, 9] and building ids of variant v (towers get ids B, B+1, ...)."""
        m = self.base.mesh
        keep = ~np.isin(m.tri_building, self.removed[v])
        t9 = m.tri9()[keep]
        tb = m.tri_building[keep]
        tw = self.tower_tris[v]
        tbw = self.base.city.B + np.arange(tw.shape[0], dtype=np.int32) // 12
        return (np.concatenate([t9, tw]).astype(np.float32),
                np.concatenate([tb, tbw]).astype(np.int32))


def scenarios(n_variants: int = 64, days: int = 31, step: float = 1.0, base=None,
              region_sides=(256, 512, 1024, 2048), centres=(79, 172, 266, 355),
              t0: float = 9.0, t1: float = 17.0, seed_off: int = 4) -> Scenarios:
    """The batched-scenario workload: base district + n_variants x U{1..5} towers (square
    30-60 m, heights U(150, 450)) x 4 seasonal intervals (`days` days around the solstices
    and equinoxes) x receiver regions with side log-uniform in `region_sides`."""
    rng = np.random.default_rng(C.SEED_BASE + seed_off)
    w = base if base is not None else district(n_facade=0)
    g = w.ground
    ext = g.nx * g.dx
    fps = w.city.footprints
    boxes = np.array([[f[:, 0].min(), f[:, 1].min(), f[:, 0].max(), f[:, 1].max()] for f in fps])
    towers, removed, regions = [], [], []
    for v in range(n_variants):
        nt = int(rng.integers(1, 6))
        fp_list, hs, rem = [], [], set()
        cx0, cy0 = rng.uniform(0.2 * ext, 0.8 * ext, 2)
        for _ in range(nt):
            side = rng.uniform(30.0, 60.0)
            cx, cy = cx0 + rng.uniform(-150, 150), cy0 + rng.uniform(-150, 150)
            x0, y0 = g.x0 + cx - side / 2, g.y0 + cy - side / 2
            x1, y1 = x0 + side, y0 + side
            # no overlap with earlier towers of this variant
            if any(not (x1 < f[0, 0] - 2 or x0 > f[1, 0] + 2 or y1 < f[0, 1] - 2 or y0 > f[2, 1] + 2)
                   for f in fp_list):
                continue
            fp_list.append(C.box_footprint(x0, y0, x1, y1))
            hs.append(rng.uniform(150.0, 450.0))
            hit = ~((boxes[:, 2] < x0 - 1) | (boxes[:, 0] > x1 + 1) | (boxes[:, 3] < y0 - 1) |
                    (boxes[:, 1] > y1 + 1))
            rem |= set(np.nonzero(hit)[0].tolist())
        tw = C.extrude(C.City(fp_list, np.asarray(hs, np.float32))).tri9()
        towers.append(tw)
        removed.append(np.asarray(sorted(rem), np.int32))
        side = int(region_sides[int(rng.integers(0, len(region_sides)))])
        mx = np.mean([f[:, 0].mean() for f in fp_list]) - g.x0
        my = np.mean([f[:, 1].mean() for f in fp_list]) - g.y0
        ix0 = int(np.clip(round(mx / g.dx) - side // 2, 0, max(g.nx - side, 0)))
        iy0 = int(np.clip(round(my / g.dx) - side // 2, 0, max(g.ny - side, 0)))
        regions.append((ix0, iy0, min(side, g.nx), min(side, g.ny)))
    intervals = [sun_table(LAT, [((c - 1 + k) % 365) + 1 for k in range(-(days // 2), days - days // 2)],
                           t0, t1, step) for c in centres]
    return Scenarios(w, towers, removed, np.asarray(regions, np.int32), intervals)


def step_counts(n_intervals: int, R: int, S: int, zero_frac: float = 0.5, seed: int = 7) -> np.ndarray:
    """Seeded per-cell step counts int32 [n_intervals, R] in 0..S, a share `zero_frac` of
    them 0 (cells never shadowed): inputs of the analysis measures, which take counts."""
    rng = np.random.default_rng(C.SEED_BASE + seed)
    c = rng.integers(1, S + 1, size=(n_intervals, R), dtype=np.int64)
    c[rng.random((n_intervals, R)) < zero_frac] = 0
    return c.astype(np.int32)

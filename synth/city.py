"""Seeded synthetic cities and receiver sets (harness inputs; none of the method's arithmetic).

The paper evaluates on the OpenStreetMap mesh of Manhattan (43k buildings, 1.5M
triangles, Sec. 8.2).  That dataset is not available here, so these generators build
Manhattan-like stand-ins: convex extruded footprints on a rectangular block grid, with
lognormal heights.  Everything is deterministic in the seed.

Mesh convention: vertices float32 [V,3] (ENU metres, ground z = 0), triangles int32
[T,3] wound counter-clockwise seen from outside (outward normals), one building id per
triangle.  A building is a closed prism: walls (optionally split into horizontal bands),
a roof fan and a bottom fan at z = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 19070443  # configs use SEED_BASE + config number


@dataclass
class City:
    footprints: list            # list of float64 [v,2] CCW convex polygons
    heights: np.ndarray         # float32 [B]
    band_height: float = 0.0    # walls split into ceil(h / band_height) bands (0 = one band)

    @property
    def B(self) -> int:
        return len(self.footprints)


@dataclass
class Mesh:
    verts: np.ndarray           # float32 [V,3]
    tris: np.ndarray            # int32 [T,3]
    tri_building: np.ndarray    # int32 [T]
    # per vertex: building id and whether z equals that building's height (roof ring)
    vert_building: np.ndarray = field(default=None)
    vert_is_roof: np.ndarray = field(default=None)

    @property
    def T(self) -> int:
        return int(self.tris.shape[0])

    def tri9(self) -> np.ndarray:
        """Triangle soup float32 [T, 9] (v0, v1, v2)."""
        return np.ascontiguousarray(self.verts[self.tris].reshape(-1, 9), dtype=np.float32)


def band_counts(city: City, heights=None) -> np.ndarray:
    """Wall bands per building: ceil(h / band_height), at least 1 (1 if no banding)."""
    hs = np.asarray(city.heights if heights is None else heights, dtype=np.float32)
    if city.band_height <= 0:
        return np.ones(len(hs), np.int32)
    return np.asarray([max(1, int(math.ceil(float(h) / city.band_height))) for h in hs], np.int32)


def extrude(city: City, heights: np.ndarray | None = None, bands=None) -> Mesh:
    """Closed prisms from convex CCW footprints; roof/bottom fans; walls in bands.
    `bands` fixes the band count per building (default: from the heights)."""
    hs = np.asarray(city.heights if heights is None else heights, dtype=np.float32)
    nbs = band_counts(city, hs) if bands is None else np.asarray(bands, np.int32)
    verts, tris, tb, vb, vroof = [], [], [], [], []
    base = 0
    for b, fp in enumerate(city.footprints):
        fp = np.asarray(fp, dtype=np.float32)
        v = fp.shape[0]
        h = hs[b]
        nb = int(nbs[b])
        zs = h * (np.arange(nb + 1, dtype=np.float32) / np.float32(nb))
        zs[-1] = h
        # rings k = 0..nb, each v vertices
        for k in range(nb + 1):
            for i in range(v):
                verts.append((fp[i, 0], fp[i, 1], zs[k]))
                vb.append(b)
                vroof.append(k == nb)
        ring = lambda k, i: base + k * v + (i % v)
        for k in range(nb):
            for i in range(v):
                a0, b0, b1, a1 = ring(k, i), ring(k, i + 1), ring(k + 1, i + 1), ring(k + 1, i)
                tris.append((a0, b0, b1)); tris.append((a0, b1, a1))
                tb.extend((b, b))
        for i in range(1, v - 1):
            tris.append((ring(nb, 0), ring(nb, i), ring(nb, i + 1))); tb.append(b)
        for i in range(1, v - 1):
            tris.append((ring(0, 0), ring(0, i + 1), ring(0, i))); tb.append(b)
        base += (nb + 1) * v
    return Mesh(verts=np.asarray(verts, dtype=np.float32).reshape(-1, 3),
                tris=np.asarray(tris, dtype=np.int32).reshape(-1, 3),
                tri_building=np.asarray(tb, dtype=np.int32),
                vert_building=np.asarray(vb, dtype=np.int32),
                vert_is_roof=np.asarray(vroof, dtype=bool))


def box_footprint(x0, y0, x1, y1) -> np.ndarray:
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.float64)


def convex_footprint(rng, cx, cy, ax, ay, nv) -> np.ndarray:
    """nv points on an axis-aligned ellipse at sorted random angles: always convex, CCW."""
    while True:
        ang = np.sort(rng.uniform(0.0, 2 * math.pi, nv))
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * math.pi]))
        if gaps.min() > 0.25 and gaps.max() < math.pi - 0.1:
            break
    return np.stack([cx + ax * np.cos(ang), cy + ay * np.sin(ang)], axis=1)


# ------------------------------------------------------------------------- configs

def city_boxes(seed: int, nx: int = 4, ny: int = 4, street: float = 15.0,
               side=(20.0, 40.0), height=(10.0, 100.0)) -> City:
    """nx x ny axis-aligned boxes: sides U(side) independently in x and y, heights U(height).

    Lots are side[1] wide with `street` between them; the box sits at the lot centre.
    The city spans [0, nx*pitch - street] x [0, ny*pitch - street].
    """
    rng = np.random.default_rng(seed)
    pitch = side[1] + street
    fps, hs = [], []
    for j in range(ny):
        for i in range(nx):
            sx, sy = rng.uniform(side[0], side[1], 2)
            cx, cy = i * pitch + side[1] / 2, j * pitch + side[1] / 2
            fps.append(box_footprint(cx - sx / 2, cy - sy / 2, cx + sx / 2, cy + sy / 2))
            hs.append(rng.uniform(height[0], height[1]))
    return City(footprints=fps, heights=np.asarray(hs, dtype=np.float32))


def _lots(extent_x, extent_y, block_x=80.0, block_y=250.0, street=18.0, cols=2, rows=8,
          origin=(0.0, 0.0)):
    """Lot rectangles (x0, y0, x1, y1) of a block grid centred in [0,extent_x] x [0,extent_y]."""
    px, py = block_x + street, block_y + street
    nbx = int((extent_x + street) // px)
    nby = int((extent_y + street) // py)
    offx = origin[0] + (extent_x - (nbx * px - street)) / 2
    offy = origin[1] + (extent_y - (nby * py - street)) / 2
    lw, lh = block_x / cols, block_y / rows
    lots = []
    for bj in range(nby):
        for bi in range(nbx):
            for r in range(rows):
                for c in range(cols):
                    x0 = offx + bi * px + c * lw
                    y0 = offy + bj * py + r * lh
                    lots.append((x0, y0, x0 + lw, y0 + lh))
    return np.asarray(lots, dtype=np.float64)


def _district_from_lots(rng, lots, n_buildings, h_median, h_sigma, h_cap, band_height,
                        margin=1.0) -> City:
    pick = np.sort(rng.choice(lots.shape[0], size=n_buildings, replace=False))
    fps = []
    for li in pick:
        x0, y0, x1, y1 = lots[li]
        cx, cy = (x0 + x1) / 2, (y0 + y1) / 2
        f = rng.uniform(0.6, 1.0)
        ax, ay = f * ((x1 - x0) / 2 - margin), f * ((y1 - y0) / 2 - margin)
        nv = int(rng.integers(4, 9))
        fps.append(convex_footprint(rng, cx, cy, ax, ay, nv))
    hs = np.minimum(rng.lognormal(math.log(h_median), h_sigma, n_buildings), h_cap)
    return City(footprints=fps, heights=hs.astype(np.float32), band_height=band_height)


def city_district(seed: int, extent: float = 2048.0, n_buildings: int = 2000,
                  h_median: float = 30.0, h_sigma: float = 0.8, h_cap: float = 400.0,
                  band_height: float = 30.0) -> City:
    """Manhattan-like district: 80 x 250 m blocks, 18 m streets, 2 x 8 lots per block.

    `n_buildings` lots are chosen at random (the rest stay empty); footprints are convex
    4-8 gons inscribed in the lot; heights lognormal (median `h_median`, sigma), capped.
    Walls split into 30 m bands bring ~2000 buildings to ~60k triangles.
    """
    rng = np.random.default_rng(seed)
    lots = _lots(extent, extent)
    return _district_from_lots(rng, lots, n_buildings, h_median, h_sigma, h_cap, band_height)


def city_ring_around_park(seed: int, park=(0.0, 0.0, 500.0, 300.0), band: float = 300.0,
                          n_buildings: int = 200, h_median: float = 60.0,
                          h_sigma: float = 0.8, h_cap: float = 400.0,
                          band_height: float = 30.0) -> City:
    """District lots within `band` metres of a rectangular park (and not inside it + street)."""
    rng = np.random.default_rng(seed)
    px0, py0, px1, py1 = park
    street = 18.0
    ex, ey = (px1 - px0) + 2 * band, (py1 - py0) + 2 * band
    lots = _lots(ex, ey, origin=(px0 - band, py0 - band))
    keep = []
    for k, (x0, y0, x1, y1) in enumerate(lots):
        inside_park = (x1 > px0 - street and x0 < px1 + street and
                       y1 > py0 - street and y0 < py1 + street)
        dx = max(px0 - x1, 0.0, x0 - px1)
        dy = max(py0 - y1, 0.0, y0 - py1)
        if not inside_park and max(dx, dy) <= band:
            keep.append(k)
    lots = lots[np.asarray(keep, dtype=np.int64)]
    return _district_from_lots(rng, lots, n_buildings, h_median, h_sigma, h_cap, band_height)


# ------------------------------------------------------------------------- receivers

@dataclass
class GroundGrid:
    x0: float
    y0: float
    dx: float
    nx: int
    ny: int

    @property
    def R(self) -> int:
        return self.nx * self.ny

    def positions(self) -> np.ndarray:
        """Cell centres, float32 [R, 3], row-major (index = iy * nx + ix), z = 0."""
        xs = (np.float32(self.x0) + (np.arange(self.nx, dtype=np.float32) + np.float32(0.5))
              * np.float32(self.dx))
        ys = (np.float32(self.y0) + (np.arange(self.ny, dtype=np.float32) + np.float32(0.5))
              * np.float32(self.dx))
        X, Y = np.meshgrid(xs, ys)
        return np.stack([X.ravel(), Y.ravel(), np.zeros(self.R, np.float32)], 1).astype(np.float32)


def facade_samples(city: City, n: int, seed: int):
    """n points uniform by wall area: float32 positions [n,3] and outward unit normals [n,3]."""
    rng = np.random.default_rng(seed)
    walls = []   # (ax, ay, bx, by, h)
    for fp, h in zip(city.footprints, city.heights):
        v = fp.shape[0]
        for i in range(v):
            a, b = fp[i], fp[(i + 1) % v]
            walls.append((a[0], a[1], b[0], b[1], float(h)))
    W = np.asarray(walls, dtype=np.float64)
    length = np.hypot(W[:, 2] - W[:, 0], W[:, 3] - W[:, 1])
    area = length * W[:, 4]
    k = rng.choice(W.shape[0], size=n, p=area / area.sum())
    s = rng.uniform(0.0, 1.0, n)
    z = rng.uniform(0.0, 1.0, n) * W[k, 4]
    px = W[k, 0] + s * (W[k, 2] - W[k, 0])
    py = W[k, 1] + s * (W[k, 3] - W[k, 1])
    ex, ey = (W[k, 2] - W[k, 0]) / length[k], (W[k, 3] - W[k, 1]) / length[k]
    pos = np.stack([px, py, z], 1).astype(np.float32)
    nrm = np.stack([ey, -ex, np.zeros(n)], 1).astype(np.float32)   # CCW footprint: outward
    return pos, nrm

"""The analysis measures of Sec. 7.2 on the device against the FP64 oracle: the shadow area
over a polygonal region from the accrual raster's own counts, the shadow score built from
it, and each building's contribution to the region's shadow."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle
from parity import workload

pytestmark = pytest.mark.gpu

POLYGONS = {
    "convex": [[60.0, 40.0], [420.0, 90.0], [480.0, 250.0], [300.0, 330.0], [90.0, 300.0]],
    "non_convex": [[40.0, 30.0], [300.0, 30.0], [300.0, 120.0], [140.0, 120.0], [140.0, 360.0],
                   [40.0, 360.0]],
    "partly_outside": [[-100.0, -50.0], [250.0, -80.0], [320.0, 200.0], [-60.0, 260.0]],
    "whole_grid": [[8.25, 6.75], [508.25, 6.75], [508.25, 381.75], [8.25, 381.75]],
}


@pytest.mark.parametrize("name", sorted(POLYGONS))
def test_shadow_area_matches_the_oracle(cuda_lib, name):
    B = cuda_lib
    w = workload("district_small")
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    gross, _, cont = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
    poly = np.array(POLYGONS[name], np.float32)
    G = (g.x0, g.y0, g.dx, g.nx, g.ny)
    for counts in (gross, cont):
        got = B.sa_shadow_area(grid, counts, w.sun.S, poly)
        want = oracle.shadow_area(G, counts.cpu().numpy(), w.sun.S, poly)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-9), (name, got, want)
    assert B.sa_shadow_area(grid, gross, w.sun.S, poly) > 0


def _table3_weights():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table3_month_weights.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array([float(r[1]) for r in rows])


@pytest.mark.parametrize("name", ["convex", "non_convex", "whole_grid"])
def test_shadow_score_matches_the_oracle(cuda_lib, name):
    """The score over the twelve months of Table 3 (seeded per-cell counts of each month,
    each out of its own step total) equals the oracle's weighted sum of areas to 1e-12; one
    interval of weight 1 is the shadow area."""
    from synth import configs
    B = cuda_lib
    w = workload("district_small")
    g = w.ground
    G = (g.x0, g.y0, g.dx, g.nx, g.ny)
    grid = B.Receivers.ground_grid(*G)
    totals = np.array([300 + 17 * m for m in range(12)], np.int32)
    counts = configs.step_counts(12, g.R, int(totals.min()), seed=30)
    wts = _table3_weights()
    poly = np.array(POLYGONS[name], np.float32)
    dev = torch.from_numpy(counts).cuda()
    got = B.sa_shadow_score(grid, dev, totals, wts, poly)
    areas = [oracle.shadow_area(G, counts[m], int(totals[m]), poly) for m in range(12)]
    want = oracle.shadow_score(areas, wts)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-9 * max(areas)), (got, want)
    one = B.sa_shadow_score(grid, dev[3:4], totals[3:4], [1.0], poly)
    assert one == pytest.approx(areas[3], rel=1e-12)
    assert one == pytest.approx(B.sa_shadow_area(grid, dev[3], int(totals[3]), poly), rel=1e-12)


def test_shadow_score_of_a_summer_and_a_winter_day(cuda_lib):
    """Two seasons of the same city weighted +1 (summer) and -1 (winter), each counted by
    the oracle on the parity grid: the device score of those counts equals the oracle's,
    and is negative (winter shadows are longer)."""
    from synth import configs
    B = cuda_lib
    poly = np.array(POLYGONS["convex"], np.float32)
    counts, totals, areas = [], [], []
    for doy in (172, 355):
        w = configs.district_small(doys=(doy,), n_facade=0, dx=5.0, nx=100, ny=75)
        g = w.ground
        G = (g.x0, g.y0, g.dx, g.nx, g.ny)
        og, _, _, _ = oracle.accumulate(w.mesh.tri9(), w.mesh.tri_building, g.positions(), None,
                                        w.sun.dirs, w.sun.day_start, w.sun.step_minutes)
        counts.append(og)
        totals.append(w.sun.S)
        areas.append(oracle.shadow_area(G, og, w.sun.S, poly))
    grid = B.Receivers.ground_grid(*G)
    got = B.sa_shadow_score(grid, torch.from_numpy(np.stack(counts)).cuda(), totals, [1.0, -1.0], poly)
    want = oracle.shadow_score(areas, [1.0, -1.0])
    assert got == pytest.approx(want, rel=1e-12)
    assert areas[1] > areas[0] and got < 0


def test_shadow_score_rejects_bad_arguments(cuda_lib):
    B = cuda_lib
    grid = B.Receivers.ground_grid(0.0, 0.0, 1.0, 8, 8)
    steps = torch.zeros((2, 64), dtype=torch.int32, device="cuda")
    tri = [[0, 0], [4, 0], [4, 4]]
    with pytest.raises(B.SAError):
        B.sa_shadow_score(grid, steps, [10, 10], [1.0, -1.5], tri)      # weight outside [-1, 1]
    with pytest.raises(B.SAError):
        B.sa_shadow_score(grid, steps, [10, 0], [1.0, -1.0], tri)       # total 0
    with pytest.raises(B.SAError):
        B.sa_shadow_score(grid, steps, [10], [1.0], tri)                # one total for two
    with pytest.raises(B.SAError):
        B.sa_shadow_score(grid, steps, [10, 10], [1.0, -1.0], [[0, 0], [1, 1]])
    assert B.sa_shadow_score(grid, steps, [10, 10], [1.0, -1.0], tri) == 0.0


def test_shadow_area_rejects_bad_arguments(cuda_lib):
    B = cuda_lib
    grid = B.Receivers.ground_grid(0.0, 0.0, 1.0, 8, 8)
    steps = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(B.SAError):
        B.sa_shadow_area(grid, steps, 10, [[0, 0], [1, 1]])
    with pytest.raises(B.SAError):
        B.sa_shadow_area(grid, steps, 0, [[0, 0], [4, 0], [4, 4]])
    pts = B.Receivers.points(np.zeros((4, 3), np.float32))
    with pytest.raises(B.SAError):
        B.sa_shadow_area(pts, steps, 10, [[0, 0], [4, 0], [4, 4]])
    assert B.sa_shadow_area(grid, steps, 10, [[0, 0], [4, 0], [4, 4]]) == 0.0


# ------------------------------------------------------------- building contribution
def _region_centres(g, poly):
    """Cell centres of the grid inside the polygon, rounded as the receivers' (FP32)."""
    ix, iy = np.meshgrid(np.arange(g.nx, dtype=np.float32), np.arange(g.ny, dtype=np.float32))
    cx = (np.float32(g.x0) + (ix + np.float32(0.5)) * np.float32(g.dx)).ravel()
    cy = (np.float32(g.y0) + (iy + np.float32(0.5)) * np.float32(g.dx)).ravel()
    keep = oracle.point_in_polygon(cx.astype(np.float64), cy.astype(np.float64), poly.astype(np.float64))
    return np.stack([cx[keep], cy[keep], np.zeros(int(keep.sum()), np.float32)], 1)


@pytest.mark.parametrize("name", ["convex", "non_convex"])
def test_building_contribution_matches_the_oracle(cuda_lib, name):
    """Per-building counts on the device against the FP64 oracle's: each building's casting
    count within its own near-boundary pairs, the nearest-caster counts within the pairs
    near the shadow boundary of any building, and the nearest counts plus the unattributed
    cell-steps equal to the region's gross shadow area from the raster's own counts."""
    B = cuda_lib
    w = workload("district_small")
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    poly = np.array(POLYGONS[name], np.float32)
    casting, nearest, (over, unattributed) = B.sa_building_contribution(scene, grid, sun, poly)
    unit = g.dx * g.dx / w.sun.S
    cnt_c = casting / unit
    cnt_n = nearest / unit
    assert np.allclose(cnt_c, np.round(cnt_c), atol=1e-6) and np.allclose(cnt_n, np.round(cnt_n), atol=1e-6)
    cnt_c, cnt_n = np.round(cnt_c).astype(np.int64), np.round(cnt_n).astype(np.int64)
    assert over == 0
    # internal consistency: the nearest casters partition the raster's shadowed cell-steps
    gross, _, _ = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
    area = B.sa_shadow_area(grid, gross, w.sun.S, poly)
    assert (cnt_n.sum() + unattributed) * unit == pytest.approx(area, rel=1e-12)
    # against the oracle on the region's cell centres
    pos = _region_centres(g, poly)
    c_o, n_o, u_o, u_any = oracle.building_steps(w.mesh.tri9(), w.mesh.tri_building, pos, None,
                                                 w.sun.dirs, w.sun.day_start, w.city.B)
    assert c_o.sum() > 10000
    dc = np.abs(cnt_c - c_o)
    assert np.all(dc <= u_o), (np.nonzero(dc > u_o)[0], dc[dc > u_o], u_o[dc > u_o])
    dn = np.abs(cnt_n - n_o)
    assert dn.sum() <= 2 * u_any, (dn.sum(), u_any)
    assert unattributed <= u_any
    assert np.all(cnt_n <= cnt_c)


def test_building_contribution_of_two_boxes_in_line(cuda_lib):
    """Two boxes one behind the other toward a low morning sun: every cell shadowed by the
    farther box alone is credited to it, and where both boxes shadow a cell the nearer box
    is the nearest caster; the device agrees with the oracle pair by pair."""
    B = cuda_lib
    from synth import city as C
    city = C.City([C.box_footprint(40, 45, 50, 55), C.box_footprint(70, 45, 80, 55)],
                  np.array([30.0, 60.0], np.float32))
    mesh = C.extrude(city)
    el = np.radians(np.linspace(15.0, 25.0, 8))
    az = np.radians(np.linspace(-8.0, 8.0, 8))
    dirs = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1).astype(np.float32)
    day_start = np.array([0, 8], np.int32)
    scene = B.Scene(mesh.verts, mesh.tris, mesh.tri_building, 2, closed=True)
    sun = B.Sun(dirs, day_start)
    x0, y0, dx, nx, ny = 0.0, 0.0, 1.0, 100, 100
    grid = B.Receivers.ground_grid(x0, y0, dx, nx, ny)
    poly = np.array([[0.0, 20.0], [40.0, 20.0], [40.0, 80.0], [0.0, 80.0]], np.float32)
    casting, nearest, (over, unattributed) = B.sa_building_contribution(scene, grid, sun, poly)
    pos = _region_centres(SimpleNamespace(x0=x0, y0=y0, dx=dx, nx=nx, ny=ny), poly)
    c_o, n_o, u_o, u_any = oracle.building_steps(mesh.tri9(), mesh.tri_building, pos, None, dirs,
                                                 day_start, 2)
    unit = dx * dx / 8
    cnt_c, cnt_n = np.round(casting / unit).astype(np.int64), np.round(nearest / unit).astype(np.int64)
    assert np.all(np.abs(cnt_c - c_o) <= u_o)
    assert np.abs(cnt_n - n_o).sum() <= 2 * u_any
    assert c_o[1] > n_o[1] > 0 and n_o[0] == c_o[0] > 0     # the tall far box reaches past the near one
    assert over == 0


def test_building_contribution_rejects_bad_arguments(cuda_lib):
    B = cuda_lib
    w = workload("district_small")
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    with pytest.raises(B.SAError):
        B.sa_building_contribution(scene, grid, sun, [[0, 0], [1, 1]])
    with pytest.raises(B.SAError):
        B.sa_building_contribution(scene, grid, sun, [[0, 0], [np.nan, 0], [4, 4]])
    pts = B.Receivers.points(np.zeros((4, 3), np.float32))
    with pytest.raises(B.SAError):
        B.sa_building_contribution(scene, pts, sun, [[0, 0], [4, 0], [4, 4]])
    # a region holding no cell centre credits nothing
    c, n, st = B.sa_building_contribution(scene, grid, sun, [[0, 0], [1, 0], [1, 1]])
    assert not c.any() and not n.any() and st == (0, 0)


def test_building_contribution_without_buildings_and_with_ragged_grids(cuda_lib):
    """An empty scene credits nothing; a grid whose sides are not multiples of the raster's
    32-cell tiles gives the same per-building counts as the oracle on its centres."""
    B = cuda_lib
    from synth import city as C
    empty = B.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), None, 0)
    w = workload("district_small")
    g = w.ground
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    c, n, st = B.sa_building_contribution(empty, grid, sun, POLYGONS["convex"])
    assert c.size == 0 and n.size == 0 and st == (0, 0)
    city = C.City([C.box_footprint(20, 20, 32, 29), C.box_footprint(45, 12, 51, 40)],
                  np.array([25.0, 40.0], np.float32))
    mesh = C.extrude(city)
    scene = B.Scene(mesh.verts, mesh.tris, mesh.tri_building, 2, closed=True)
    x0, y0, dx, nx, ny = -3.0, -2.0, 0.7, 101, 77
    grid = B.Receivers.ground_grid(x0, y0, dx, nx, ny)
    poly = np.array([[-3.0, -2.0], [60.0, -2.0], [60.0, 45.0], [-3.0, 45.0]], np.float32)
    casting, nearest, (over, un) = B.sa_building_contribution(scene, grid, sun, poly)
    pos = _region_centres(SimpleNamespace(x0=x0, y0=y0, dx=dx, nx=nx, ny=ny), poly)
    c_o, n_o, u_o, u_any = oracle.building_steps(mesh.tri9(), mesh.tri_building, pos, None,
                                                 w.sun.dirs, w.sun.day_start, 2)
    unit = dx * dx / w.sun.S
    cnt_c = np.round(casting / unit).astype(np.int64)
    cnt_n = np.round(nearest / unit).astype(np.int64)
    assert np.all(np.abs(cnt_c - c_o) <= u_o) and np.abs(cnt_n - n_o).sum() <= 2 * u_any
    assert c_o.min() > 0 and over == 0


@pytest.mark.parametrize("n_buildings", [20, 70000])
def test_building_contribution_of_a_row_of_twenty_boxes(cuda_lib, n_buildings):
    """Twenty thin boxes in a row toward a low sun: a ray from behind the row meets up to
    twenty buildings, more than the per-run list holds, so the lanes recount ray by ray.
    Counts agree with the oracle pair by pair, both with 16-bit building ids (20
    buildings) and with 32-bit ones (70,000 declared, the rest crediting nothing)."""
    B = cuda_lib
    from synth import city as C
    feet = [C.box_footprint(30.0 + 4.0 * k, 40.0, 31.5 + 4.0 * k, 60.0) for k in range(20)]
    city = C.City(feet, np.full(20, 12.0, np.float32))
    mesh = C.extrude(city)
    el = np.radians(np.linspace(6.0, 9.0, 12))
    az = np.radians(np.linspace(-4.0, 4.0, 12))
    dirs = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1).astype(np.float32)
    day_start = np.array([0, 12], np.int32)
    scene = B.Scene(mesh.verts, mesh.tris, mesh.tri_building, n_buildings, closed=True)
    sun = B.Sun(dirs, day_start)
    x0, y0, dx, nx, ny = 0.0, 30.0, 0.5, 60, 60
    grid = B.Receivers.ground_grid(x0, y0, dx, nx, ny)
    poly = np.array([[0.0, 30.0], [29.0, 30.0], [29.0, 60.0], [0.0, 60.0]], np.float32)
    casting, nearest, (over, un) = B.sa_building_contribution(scene, grid, sun, poly)
    assert casting.shape == (n_buildings,)
    pos = _region_centres(SimpleNamespace(x0=x0, y0=y0, dx=dx, nx=nx, ny=ny), poly)
    c_o, n_o, u_o, u_any = oracle.building_steps(mesh.tri9(), mesh.tri_building, pos, None, dirs,
                                                 day_start, 20)
    unit = dx * dx / 12
    cnt_c = np.round(casting / unit).astype(np.int64)
    cnt_n = np.round(nearest / unit).astype(np.int64)
    assert not cnt_c[20:].any() and not cnt_n[20:].any()
    cnt_c, cnt_n = cnt_c[:20], cnt_n[:20]
    assert over == 0
    assert (c_o > 0).sum() >= 12, c_o          # most of the row reaches the region
    assert np.all(np.abs(cnt_c - c_o) <= u_o), (cnt_c, c_o, u_o)
    assert np.abs(cnt_n - n_o).sum() <= 2 * u_any

"""The shadow area over a polygonal region (Sec. 7.2) on the device against the FP64 oracle,
from the accrual raster's own counts, and the shadow score built from it."""
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


def test_shadow_score_over_intervals(cuda_lib):
    """Two seasons of the same city weighted +1 (summer) and -1 (winter): the score is the
    difference of the device areas, equal to the oracle's on the same counts."""
    B = cuda_lib
    from synth import configs
    poly = np.array(POLYGONS["convex"], np.float32)
    areas, want = [], []
    for doy in (172, 355):
        w = configs.district_small(doys=(doy,), n_facade=0)
        g = w.ground
        scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
        sun = B.Sun(w.sun.dirs, w.sun.day_start)
        grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
        gross, _, _ = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
        areas.append(B.sa_shadow_area(grid, gross, w.sun.S, poly))
        want.append(oracle.shadow_area((g.x0, g.y0, g.dx, g.nx, g.ny), gross.cpu().numpy(), w.sun.S, poly))
    s = B.shadow_score(areas, [1.0, -1.0])
    assert s == pytest.approx(oracle.shadow_score(want, [1.0, -1.0]), rel=1e-9, abs=1e-9)
    assert areas[1] > areas[0]          # winter shadows are longer: the score is negative
    assert s < 0


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

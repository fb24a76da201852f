"""sa_accumulate_grid_noalloc: the ground accrual raster without any device allocation.

It is meant for callers that cannot allocate device memory while they run (a host
application that reserved the device's memory up front, or a loop that must not pay the
allocator's synchronisation).  Its scratch is a fixed array inside the library, shared by
every call, so these tests check that two calls in a row -- the second seeing whatever
the first left behind -- both match the allocating entry point exactly.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from synth import configs

pytestmark = pytest.mark.gpu


def _setup(B, w, block_len=0):
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    sun = B.Sun(w.sun.dirs, w.sun.day_start, block_len)
    return scene, grid, sun


def _outputs(R):
    return (torch.full((R,), -7, dtype=torch.int32, device="cuda"),
            torch.full((R,), -7.0, dtype=torch.float32, device="cuda"),
            torch.full((R,), -7, dtype=torch.int32, device="cuda"))


def test_noalloc_matches_sa_accumulate_on_two_calls_in_a_row(cuda_lib):
    B = cuda_lib
    cases = [configs.district_small(), configs.boxes16()]
    for w in cases:
        scene, grid, sun = _setup(B, w)
        ref_g, ref_m, ref_c = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
        for call in range(2):
            g, m, c = _outputs(grid.R)
            B.sa_accumulate_grid_noalloc(scene, grid, sun, w.sun.step_minutes, g, m, c)
            torch.cuda.synchronize()
            assert torch.equal(g, ref_g), f"{w.name}: gross differs on call {call}"
            assert torch.equal(m, ref_m), f"{w.name}: minutes differ on call {call}"
            assert torch.equal(c, ref_c), f"{w.name}: continuous differs on call {call}"


def test_noalloc_without_continuous_buffer_and_accumulating(cuda_lib):
    B = cuda_lib
    w = configs.district_small(doys=(172, 250), step=8.0, n_facade=0)
    scene, grid, sun = _setup(B, w, 13)
    ref_g, _, ref_c = B.sa_accumulate(scene, grid, sun, 8.0, "accrual_sam")
    g = torch.zeros(grid.R, dtype=torch.int32, device="cuda")
    B.sa_accumulate_grid_noalloc(scene, grid, sun, 8.0, g)          # no minutes, no continuous
    assert torch.equal(g, ref_g)
    # day by day into the same buffers equals the one-shot result
    ds = w.sun.day_start
    g2 = torch.zeros(grid.R, dtype=torch.int32, device="cuda")
    c2 = torch.zeros(grid.R, dtype=torch.int32, device="cuda")
    for k in range(len(ds) - 1):
        d = w.sun.dirs[ds[k]:ds[k + 1]]
        sun_k = B.Sun(d, np.array([0, d.shape[0]], np.int32), 13)
        B.sa_accumulate_grid_noalloc(scene, grid, sun_k, 8.0, g2, None, c2, accumulate_into=True)
    torch.cuda.synchronize()
    assert torch.equal(g2, ref_g) and torch.equal(c2, ref_c)


def test_noalloc_rejects_grids_above_its_limit(cuda_lib):
    B = cuda_lib
    w = configs.boxes16()
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    big = B.Receivers.ground_grid(0.0, 0.0, 1.0, 2049, 2048)       # one column too many
    g = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(B.SAError) as e:
        B.sa_accumulate_grid_noalloc(scene, big, sun, 1.0, g)
    assert e.value.status == -1 and "SA_NOALLOC_MAX_CELLS" in str(e.value)
    pts = B.Receivers.points(w.ground.positions()[:8])
    with pytest.raises(B.SAError) as e:
        B.sa_accumulate_grid_noalloc(scene, pts, sun, 1.0, g)
    assert e.value.status == -8

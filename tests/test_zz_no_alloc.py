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


def _slabs(n):
    """n horizontal triangles, 0.25 m apart from 10 m up, each containing the whole
    2048 x 2048 m grid: every one of them bins into every tile of every block (4096 tiles),
    so a block's bins are exactly n x 4096."""
    v, t = [], []
    for k in range(n):
        z = 10.0 + 0.25 * k
        v += [[-5000.0, -5000.0, z], [10000.0, -5000.0, z], [-5000.0, 10000.0, z]]
        t.append([3 * k, 3 * k + 1, 3 * k + 2])
    return np.array(v, np.float32), np.array(t, np.int32)


def test_noalloc_with_an_empty_sun(cuda_lib):
    """No steps: zero counts, as sa_accumulate gives, and unchanged ones when accumulating."""
    B = cuda_lib
    w = configs.boxes16()
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    sun = B.Sun(np.zeros((0, 3), np.float32), np.array([0, 0], np.int32))
    ref = B.sa_accumulate(scene, grid, sun, 2.0, "accrual_sam")
    out = _outputs(grid.R)
    B.sa_accumulate_grid_noalloc(scene, grid, sun, 2.0, *out)
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b) and not a.any()
    out = _outputs(grid.R)
    B.sa_accumulate_grid_noalloc(scene, grid, sun, 2.0, *out, accumulate_into=True)
    torch.cuda.synchronize()
    assert all(bool((a == -7).all()) for a in out)


def test_noalloc_at_its_limit_on_the_district(cuda_lib):
    """The full district: 2048 x 2048 cells (SA_NOALLOC_MAX_CELLS) and 481 steps, bit for
    bit the allocating call's result, on two calls in a row."""
    B = cuda_lib
    w = configs.district(n_facade=0)
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    assert grid.R == 4194304
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    ref = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
    for call in range(2):
        out = _outputs(grid.R)
        B.sa_accumulate_grid_noalloc(scene, grid, sun, w.sun.step_minutes, *out)
        torch.cuda.synchronize()
        for a, b, name in zip(out, ref, ("gross", "minutes", "continuous")):
            assert torch.equal(a, b), f"district {name} differs on call {call}"


def test_noalloc_halves_chunks_whose_bins_do_not_fit(cuda_lib):
    """256 slabs over a 2048^2 grid bin 1,048,576 triangle-tile pairs per block; the nine
    blocks of a day (9.4M) exceed the ~8.2M bins the scratch holds beside the run and
    longest-run state of 4M cells, so the call cuts the day into chunks of five and four
    blocks -- with the allocating call's result."""
    B = cuda_lib
    v, t = _slabs(256)
    scene = B.Scene(v, t)
    grid = B.Receivers.ground_grid(0.0, 0.0, 1.0, 2048, 2048)
    st = configs.district(n_facade=0, with_ground=False).sun
    sun = B.Sun(st.dirs, st.day_start)
    assert sun.n_blocks == 9
    ref_g, ref_m, _ = B.sa_accumulate(scene, grid, sun, 1.0, "accrual_sam")
    assert int(ref_g.min()) == st.S          # every cell under the slabs at every step
    for call in range(2):
        g, m, _ = _outputs(grid.R)
        B.sa_accumulate_grid_noalloc(scene, grid, sun, 1.0, g, m, None)
        torch.cuda.synchronize()
        assert torch.equal(g, ref_g) and torch.equal(m, ref_m), call


def test_noalloc_rejects_a_block_whose_bins_do_not_fit(cuda_lib):
    """2,100 slabs bin 8.6M pairs in a single block, more than the scratch holds: the call
    is refused with SA_ERR_INVALID_ARG before any output is written, accumulating or not."""
    B = cuda_lib
    v, t = _slabs(2100)
    scene = B.Scene(v, t)
    grid = B.Receivers.ground_grid(0.0, 0.0, 1.0, 2048, 2048)
    st = configs.district(n_facade=0, with_ground=False).sun
    sun = B.Sun(st.dirs, st.day_start)
    for acc in (False, True):
        g, m, _ = _outputs(grid.R)
        with pytest.raises(B.SAError) as e:
            B.sa_accumulate_grid_noalloc(scene, grid, sun, 1.0, g, m, None, accumulate_into=acc)
        assert e.value.status == -1 and "do not fit" in str(e.value)
        torch.cuda.synchronize()
        assert bool((g == -7).all()) and bool((m == -7.0).all())


def test_noalloc_allocates_nothing(cuda_lib):
    """The call takes no scratch from the library's pool and maps no device memory: the
    library's allocation count and the device's free memory are the same before and after
    two calls (after one warm-up call, which loads the kernels)."""
    B = cuda_lib
    w = configs.district_small()
    scene, grid, sun = _setup(B, w)
    out = _outputs(grid.R)
    torch.cuda.synchronize()
    s0 = B.sa_scratch_stats()
    B.sa_accumulate_grid_noalloc(scene, grid, sun, w.sun.step_minutes, *out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        B.sa_accumulate_grid_noalloc(scene, grid, sun, w.sun.step_minutes, *out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    s1 = B.sa_scratch_stats()
    assert s1["allocations"] == s0["allocations"] and s1["bytes"] == s0["bytes"], (s0, s1)
    assert free1 == free0, (free0, free1)
    # the count does move when the allocating call runs
    B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
    torch.cuda.synchronize()
    assert B.sa_scratch_stats()["allocations"] > s1["allocations"]

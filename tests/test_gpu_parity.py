"""GPU parity of every exact method against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
from synth import city as C
from synth import configs
from synth.sun import sun_table

from parity import (assert_bits_parity, assert_counts_parity, block_sizes, cached_oracle,
                    unpack_masks, workload)

pytestmark = pytest.mark.gpu

EXACT = ["sweep_trace", "accrual_trace", "accrual_sam", "sweep_raster"]
POINT_METHODS = ["sweep_trace", "accrual_trace", "accrual_sam"]


def _scene(B, w):
    return B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)


def _ground(B, w):
    g = w.ground
    return B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)


def _run(B, scene, recv, sun, method, minutes=1.0):
    g, m, c = B.sa_accumulate(scene, recv, sun, minutes, method)
    torch.cuda.synchronize()
    return g.cpu().numpy(), m.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("method", EXACT)
def test_boxes16_ground_counts(cuda_lib, method):
    B = cuda_lib
    w = workload("boxes16")
    bits, near = cached_oracle("boxes16/ground", w, "ground")
    sc, rc, sun = _scene(B, w), _ground(B, w), B.Sun(w.sun.dirs, w.sun.day_start)
    g, m, c = _run(B, sc, rc, sun, method, w.sun.step_minutes)
    assert_counts_parity(g, c, bits, near, w.sun.day_start, method)
    assert np.allclose(m, g * np.float32(w.sun.step_minutes))


@pytest.mark.parametrize("method", EXACT)
def test_boxes16_ground_bits(cuda_lib, method):
    B = cuda_lib
    w = workload("boxes16")
    bits, near = cached_oracle("boxes16/ground", w, "ground")
    sc, rc, sun = _scene(B, w), _ground(B, w), B.Sun(w.sun.dirs, w.sun.day_start)
    masks = B.sa_shadow_masks(sc, rc, sun, method)
    torch.cuda.synchronize()
    gb = unpack_masks(masks, block_sizes(w.sun.day_start))
    assert_bits_parity(gb, bits, near, method)


@pytest.mark.parametrize("method", EXACT)
@pytest.mark.parametrize("block_len", [0, 7, 64])
def test_district_small_ground(cuda_lib, method, block_len):
    """200 x 150 cells (ragged 32-cell tiles and 8 x 4 warp patches), 120 buildings."""
    B = cuda_lib
    w = workload("district_small")
    bits, near = cached_oracle("district_small/ground", w, "ground")
    sc, rc = _scene(B, w), _ground(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start, block_len)
    g, _, c = _run(B, sc, rc, sun, method)
    assert_counts_parity(g, c, bits, near, w.sun.day_start, f"{method}/K{block_len}")
    masks = B.sa_shadow_masks(sc, rc, sun, method)
    gb = unpack_masks(masks, block_sizes(w.sun.day_start, block_len))
    assert_bits_parity(gb, bits, near, f"{method}/K{block_len}")


@pytest.mark.parametrize("method", POINT_METHODS)
def test_district_small_facades(cuda_lib, method):
    B = cuda_lib
    w = workload("district_small")
    bits, near = cached_oracle("district_small/facade", w, "facade")
    sc = _scene(B, w)
    rc = B.Receivers.points(w.facade_pos, w.facade_nrm)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    g, _, c = _run(B, sc, rc, sun, method)
    assert_counts_parity(g, c, bits, near, w.sun.day_start, method)
    masks = B.sa_shadow_masks(sc, rc, sun, method)
    gb = unpack_masks(masks, block_sizes(w.sun.day_start))
    assert_bits_parity(gb, bits, near, method)


def test_point_receivers_on_the_ground_match_the_grid(cuda_lib):
    """Ground cells passed as points (no normal) give the grid's result."""
    B = cuda_lib
    w = workload("district_small")
    sc = _scene(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    gg, _, gc = _run(B, sc, _ground(B, w), sun, "accrual_trace")
    pg, _, pc = _run(B, sc, B.Receivers.points(w.ground.positions()), sun, "accrual_trace")
    assert np.array_equal(gg, pg) and np.array_equal(gc, pc)


def test_theorem1_accrual_raster_equals_per_step_raster(cuda_lib):
    """Theorem 1 (Sec. 4): one accrual pass per block gives the same slices as one map per
    step -- here bit for bit, over every receiver, boundary or not."""
    B = cuda_lib
    w = workload("district_small")
    sc, rc = _scene(B, w), _ground(B, w)
    for K in (0, 13, 64):
        sun = B.Sun(w.sun.dirs, w.sun.day_start, K)
        a = B.sa_shadow_masks(sc, rc, sun, "accrual_sam")
        b = B.sa_shadow_masks(sc, rc, sun, "sweep_raster")
        assert torch.equal(a, b)


def test_multi_day_stitching_and_progressive_accumulation(cuda_lib):
    """Three days: runs restart each day (continuous = max over days), blocks of 7 steps
    are stitched with prefix / max / suffix, and day-by-day accumulation equals one call."""
    B = cuda_lib
    w = configs.district_small(doys=(172, 200, 250), step=8.0, n_facade=0)
    bits, near = cached_oracle("district_small_3d/ground", w, "ground")
    sc, rc = _scene(B, w), _ground(B, w)
    ds = w.sun.day_start
    for method in EXACT:
        sun = B.Sun(w.sun.dirs, ds, 7)
        g, _, c = _run(B, sc, rc, sun, method, 8.0)
        assert_counts_parity(g, c, bits, near, ds, method)
        gacc = torch.zeros(rc.R, dtype=torch.int32, device="cuda")
        cacc = torch.zeros(rc.R, dtype=torch.int32, device="cuda")
        for k in range(len(ds) - 1):
            d = w.sun.dirs[ds[k]:ds[k + 1]]
            sun_k = B.Sun(d, np.array([0, d.shape[0]], np.int32), 7)
            B.sa_accumulate(sc, rc, sun_k, 8.0, method, accumulate_into=True, gross=gacc,
                            continuous=cacc, want_minutes=False)
        assert np.array_equal(gacc.cpu().numpy(), g) and np.array_equal(cacc.cpu().numpy(), c)


def test_empty_scene_and_empty_receivers(cuda_lib):
    B = cuda_lib
    w = workload("boxes16")
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    empty = B.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    rc = _ground(B, w)
    for method in EXACT:
        g, _, c = _run(B, empty, rc, sun, method)
        assert g.sum() == 0 and c.sum() == 0
    none = B.Receivers.points(np.zeros((0, 3), np.float32))
    g, m, c = B.sa_accumulate(_scene(B, w), none, sun, 2.0, "accrual_trace")
    assert g.numel() == 0


def test_single_triangle_scene(cuda_lib):
    B = cuda_lib
    v = np.array([[0, 0, 10], [10, 0, 10], [0, 10, 10]], np.float32)
    t = np.array([[0, 1, 2]], np.int32)
    sc = B.Scene(v, t)
    st = sun_table(40.7, [172], 11.0, 13.0, 5.0)
    sun = B.Sun(st.dirs, st.day_start)
    grid = C.GroundGrid(-20.0, -20.0, 0.5, 80, 80)
    rc = B.Receivers.ground_grid(grid.x0, grid.y0, grid.dx, grid.nx, grid.ny)
    bits = oracle.shadow_bits(v.reshape(1, 9), None, grid.positions(), None, st.dirs)
    near = oracle.near_boundary(v.reshape(1, 9), None, grid.positions(), None, st.dirs,
                                st.day_start, bits)
    for method in EXACT:
        g, _, c = _run(B, sc, rc, sun, method)
        assert_counts_parity(g, c, bits, near, st.day_start, method)
        assert g.sum() > 0


def test_receivers_inside_footprints_are_always_shadowed(cuda_lib):
    B = cuda_lib
    w = workload("boxes16")
    cen = np.array([[fp[:, 0].mean(), fp[:, 1].mean(), 0.0] for fp in w.city.footprints], np.float32)
    sc, sun = _scene(B, w), B.Sun(w.sun.dirs, w.sun.day_start)
    for method in POINT_METHODS:
        g, _, c = _run(B, sc, B.Receivers.points(cen), sun, method)
        assert (g == w.sun.S).all() and (c == w.sun.S).all()


def test_raster_methods_reject_point_receivers(cuda_lib):
    B = cuda_lib
    w = workload("boxes16")
    sc, sun = _scene(B, w), B.Sun(w.sun.dirs, w.sun.day_start)
    rc = B.Receivers.points(w.ground.positions()[:10])
    with pytest.raises(B.SAError) as e:
        B.sa_accumulate(sc, rc, sun, 1.0, "sweep_raster")
    assert e.value.status == -8


@pytest.mark.parametrize("mode", ["packet", "lane"])
@pytest.mark.parametrize("method", ["sweep_trace", "accrual_trace"])
def test_traversal_modes_give_the_same_parity(cuda_lib, mode, method):
    """Both BVH traversal modes, on ground grids and facade points."""
    B = cuda_lib
    w = workload("district_small")
    key = B.SA_OPT_SWEEP_TRAVERSAL if method == "sweep_trace" else B.SA_OPT_ACCRUAL_TRAVERSAL
    B.sa_set_option(key, B.TRAVERSAL[mode])
    try:
        sc = _scene(B, w)
        sun = B.Sun(w.sun.dirs, w.sun.day_start)
        for part, rc in (("ground", _ground(B, w)),
                         ("facade", B.Receivers.points(w.facade_pos, w.facade_nrm))):
            bits, near = cached_oracle(f"district_small/{part}", w, part)
            masks = B.sa_shadow_masks(sc, rc, sun, method)
            gb = unpack_masks(masks, block_sizes(w.sun.day_start))
            assert_bits_parity(gb, bits, near, f"{method}/{mode}/{part}")
    finally:
        B.sa_set_option(key, 0)


@pytest.mark.parametrize("block_len", [0, 9])
def test_closed_scene_rasters_only_sun_facing_faces(cuda_lib, block_len):
    """A scene declared closed skips faces turned away from the sun; parity and Theorem 1
    still hold."""
    B = cuda_lib
    w = workload("district_small")
    bits, near = cached_oracle("district_small/ground", w, "ground")
    sc = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    rc = _ground(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start, block_len)
    a = B.sa_shadow_masks(sc, rc, sun, "accrual_sam")
    b = B.sa_shadow_masks(sc, rc, sun, "sweep_raster")
    assert torch.equal(a, b)
    gb = unpack_masks(a, block_sizes(w.sun.day_start, block_len))
    assert_bits_parity(gb, bits, near, f"closed/K{block_len}")
    g, _, c = _run(B, sc, rc, sun, "accrual_sam")
    assert_counts_parity(g, c, bits, near, w.sun.day_start, "closed")


def test_facade_sam_multi_day_and_progressive(cuda_lib):
    """The light-space accrual map of facade points over three days, blocks of 7 steps:
    oracle parity, and day-by-day accumulation equal to one call."""
    B = cuda_lib
    w = configs.district_small(doys=(172, 200, 250), step=8.0, n_facade=1500)
    bits, near = cached_oracle("district_small_3d/facade", w, "facade")
    sc = _scene(B, w)
    rc = B.Receivers.points(w.facade_pos, w.facade_nrm)
    ds = w.sun.day_start
    sun = B.Sun(w.sun.dirs, ds, 7)
    g, _, c = _run(B, sc, rc, sun, "accrual_sam", 8.0)
    assert_counts_parity(g, c, bits, near, ds, "facade sam")
    masks = B.sa_shadow_masks(sc, rc, sun, "accrual_sam")
    assert_bits_parity(unpack_masks(masks, block_sizes(ds, 7)), bits, near, "facade sam bits")
    gacc = torch.zeros(rc.R, dtype=torch.int32, device="cuda")
    cacc = torch.zeros(rc.R, dtype=torch.int32, device="cuda")
    for k in range(len(ds) - 1):
        d = w.sun.dirs[ds[k]:ds[k + 1]]
        sun_k = B.Sun(d, np.array([0, d.shape[0]], np.int32), 7)
        B.sa_accumulate(sc, rc, sun_k, 8.0, "accrual_sam", accumulate_into=True, gross=gacc,
                        continuous=cacc, want_minutes=False)
    assert np.array_equal(gacc.cpu().numpy(), g) and np.array_equal(cacc.cpu().numpy(), c)
    # A closed scene tests only the faces turned toward the sun.  A ray that meets a
    # closed solid crosses one of them, so the bits agree with the open scene's everywhere
    # except where a ray grazes a silhouette edge, which FP32 may decide either way on the
    # two face sets: only steps the oracle classes as near a boundary may differ.
    scc = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    mc = unpack_masks(B.sa_shadow_masks(scc, rc, sun, "accrual_sam"), block_sizes(ds, 7))
    mo = unpack_masks(masks, block_sizes(ds, 7))
    assert_bits_parity(mc, mo, near, "facade sam closed vs open")
    assert_bits_parity(mc, bits, near, "facade sam closed")


@pytest.mark.parametrize("closed", [True, False])
def test_accrual_maps_do_not_depend_on_the_run_length(cuda_lib, closed):
    """Steps per set-up (ground 1..32, points 1..32) only regroup the same per-step tests
    (Theorem 1), so both accrual maps give identical counts for every run length."""
    B = cuda_lib
    w = workload("district_small")
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=closed)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = _ground(B, w)
    fac = B.Receivers.points(w.facade_pos, w.facade_nrm)
    for r, key, runs in ((grid, B.SA_OPT_RASTER_RUN, (1, 3, 13, 24, 32)),
                         (fac, B.SA_OPT_POINT_RUN, (1, 3, 13, 20, 32))):
        old = B.sa_get_option(key)
        try:
            B.sa_set_option(key, 8)
            want = _run(B, scene, r, sun, "accrual_sam")
            for run in runs:
                B.sa_set_option(key, run)
                got = _run(B, scene, r, sun, "accrual_sam")
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[2], want[2]), run
        finally:
            B.sa_set_option(key, old)


def test_non_finite_points_are_rejected_and_the_context_stays_usable(cuda_lib):
    B = cuda_lib
    pos = np.random.default_rng(0).uniform(0, 50, (1000, 3)).astype(np.float32)
    nrm = np.tile(np.array([[1.0, 0.0, 0.0]], np.float32), (1000, 1))
    bad = pos.copy()
    bad[617, 1] = np.nan
    with pytest.raises(B.SAError) as ex:
        B.Receivers.points(bad, nrm)
    assert ex.value.status == -5 and "position 617" in str(ex.value)
    badn = nrm.copy()
    badn[42, 2] = np.inf
    with pytest.raises(B.SAError) as ex:
        B.Receivers.points(torch.from_numpy(pos).cuda(), torch.from_numpy(badn).cuda())
    assert ex.value.status == -5 and "normal 42" in str(ex.value)
    ok = B.Receivers.points(pos, nrm)
    assert ok.R == 1000


def test_scene_from_device_buffers_equals_scene_from_host_buffers(cuda_lib):
    """sa_scene_from_mesh with device_ptrs = 1 reads the caller's device buffers in place and
    builds the same scene (same counts for every method) as from host buffers; bad device
    input is rejected with the same errors."""
    import ctypes as ct
    B = cuda_lib
    L = B.lib()
    w = workload("district_small")
    host = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    dv = torch.from_numpy(np.ascontiguousarray(w.mesh.verts, np.float32)).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(w.mesh.tris, np.int32)).cuda()
    db = torch.from_numpy(np.ascontiguousarray(w.mesh.tri_building, np.int32)).cuda()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = ct.c_void_p()
    assert L.sa_scene_from_mesh(ct.c_void_p(dv.data_ptr()), dv.shape[0], ct.c_void_p(dt.data_ptr()),
                                dt.shape[0], ct.c_void_p(db.data_ptr()), w.city.B, 1, stream,
                                ct.byref(h)) == 0
    dev = B.Scene.__new__(B.Scene)
    dev.handle, dev.n_buildings = h, w.city.B
    B.lib().sa_scene_declare_closed(h, 1)
    assert dev.info() == host.info()
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = _ground(B, w)
    fac = B.Receivers.points(w.facade_pos, w.facade_nrm)
    for r, methods in ((grid, EXACT), (fac, POINT_METHODS)):
        for m in methods:
            a = _run(B, host, r, sun, m)
            b = _run(B, dev, r, sun, m)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2]), m
    bad = dt.clone()
    bad[5, 1] = dv.shape[0]
    h2 = ct.c_void_p()
    assert L.sa_scene_from_mesh(ct.c_void_p(dv.data_ptr()), dv.shape[0], ct.c_void_p(bad.data_ptr()),
                                bad.shape[0], None, 1, 1, stream, ct.byref(h2)) == -1
    assert b"triangle 5" in L.sa_last_error()


@pytest.mark.parametrize("on_device", [False, True])
def test_mesh_contents_are_checked_on_the_device(cuda_lib, on_device):
    """A non-finite vertex (SA_ERR_DEGENERATE), a vertex index or a building id out of
    range (SA_ERR_INVALID_ARG) fail the scene with the first offending vertex or triangle
    named, from host or device buffers; a vertex no triangle uses still counts for the
    finiteness check but not for the bounds, and the context stays usable."""
    import ctypes as ct
    B = cuda_lib
    L = B.lib()
    from synth import city as C
    mesh = C.extrude(C.city_boxes(3, nx=3, ny=2))
    v0 = np.concatenate([mesh.verts, np.array([[5.0, 5.0, -40.0]], np.float32)])   # unused vertex
    t0, b0 = mesh.tris.copy(), mesh.tri_building.copy()
    nb = int(b0.max()) + 1
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    keep = []

    def ptr(a):
        a = np.ascontiguousarray(a)
        if on_device:
            a = torch.from_numpy(a).cuda()
            keep.append(a)
            return ct.c_void_p(a.data_ptr())
        keep.append(a)
        return a.ctypes.data_as(ct.c_void_p)

    def make(v, t, b):
        h = ct.c_void_p()
        st = L.sa_scene_from_mesh(ptr(v), v.shape[0], ptr(t), t.shape[0], ptr(b), nb,
                                  1 if on_device else 0, stream, ct.byref(h))
        return st, L.sa_last_error().decode(), h

    v = v0.copy()
    v[17, 2] = np.nan
    v[40, 0] = np.inf
    st, msg, _ = make(v, t0, b0)
    assert st == -5 and "non-finite vertex 17" in msg, msg
    v = v0.copy()
    v[-1, 1] = np.nan                       # unused, still checked
    st, msg, _ = make(v, t0, b0)
    assert st == -5 and f"non-finite vertex {v0.shape[0] - 1}" in msg, msg
    t = t0.copy()
    t[23, 1] = v0.shape[0]
    t[30, 0] = -1
    st, msg, _ = make(v0, t, b0)
    assert st == -1 and f"triangle 23 indexes vertex {v0.shape[0]}" in msg, msg
    b = b0.copy()
    b[11] = nb
    t = t0.copy()
    t[12, 2] = -7
    st, msg, _ = make(v0, t, b)
    assert st == -1 and f"building id {nb} of triangle 11" in msg, msg
    st, msg, h = make(v0, t0, b0)
    assert st == 0, msg
    sc = B.Scene.__new__(B.Scene)
    sc.handle, sc.n_buildings = h, nb
    info = sc.info()
    assert info["n_tris"] == t0.shape[0] and info["n_buildings"] == nb
    assert info["min_z"] == float(mesh.verts[t0.ravel(), 2].min())  # the unused vertex is not a bound
    # the scene works: same counts as the binding's own scene of the plain mesh
    ref = B.Scene(mesh.verts, mesh.tris, mesh.tri_building, nb)
    st_ = configs.boxes16().sun
    sun = B.Sun(st_.dirs, st_.day_start)
    pts = B.Receivers.points(np.array([[x, y, 0.0] for x in range(0, 120, 7) for y in range(0, 80, 9)], np.float32))
    a = B.sa_accumulate(ref, pts, sun, 2.0, "accrual_trace")[0]
    c = B.sa_accumulate(sc, pts, sun, 2.0, "accrual_trace")[0]
    assert torch.equal(a, c) and int(a.sum()) > 0


@pytest.mark.parametrize("up", [True, False])
@pytest.mark.parametrize("closed", [False, True])
def test_cells_on_a_shared_edge_are_covered(cuda_lib, up, closed):
    """A square roof of two triangles at z = 1 and a sun at azimuth 45 deg (d_x = d_y
    exactly): the projected diagonal, the triangles' shared edge, passes exactly through
    the cell centres (c, c), where the edge value is an exact zero in both triangles.
    Every exact method still shadows those cells at every step, whichever way the
    triangles face (open scene: the back-facing case too; a closed scene is declared
    only with the faces up)."""
    B = cuda_lib
    if closed and not up:
        pytest.skip("a closed scene's sun-facing faces point up")
    v = np.array([[0, 0, 1], [4, 0, 1], [4, 4, 1], [0, 4, 1]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]] if up else [[0, 2, 1], [0, 3, 2]], np.int32)
    scene = B.Scene(v, t, None, 1, closed=closed)
    el = np.radians(np.array([50.0, 55.0, 60.0, 65.0]))
    h = (np.cos(el) / np.sqrt(2.0)).astype(np.float32)
    dirs = np.stack([h, h, np.sin(el).astype(np.float32)], 1).astype(np.float32)
    assert np.array_equal(dirs[:, 0], dirs[:, 1])
    sun = B.Sun(dirs, np.array([0, 4], np.int32))
    grid = B.Receivers.ground_grid(-2.0, -2.0, 1.0, 8, 8)
    diag = [(c + 2) * 8 + (c + 2) for c in (0, 1, 2)]       # centres (0.5, 0.5) ... (2.5, 2.5)
    for m in ("accrual_sam", "sweep_raster", "accrual_trace", "sweep_trace"):
        g, _, _ = _run(B, scene, grid, sun, m)
        assert (g[diag] == 4).all(), (m, g[diag])
    pts = B.Receivers.points(np.array([[c, c, 0.0] for c in (0.5, 1.5, 2.5)], np.float32))
    for m in POINT_METHODS:
        g, _, _ = _run(B, scene, pts, sun, m)
        assert (g == 4).all(), (m, g)

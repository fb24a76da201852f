"""Full-size workloads in the benchmark's launch configuration (closed scene, blocks of 60
steps, the accrual maps for ground and facades), checked against the FP64 oracle on
sampled receivers it can compute one by one."""
import numpy as np
import pytest
import torch

import oracle
from synth import city as C
from synth import configs

from parity import assert_bits_parity, assert_counts_parity, block_sizes, unpack_masks
from test_gpu_adjoint import flips_per_day

pytestmark = pytest.mark.gpu


def _closed_scene(B, w):
    return B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)


def _grid(B, g):
    return B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)


def test_district_full_size_sampled(cuda_lib):
    """2,000 buildings, 2048^2 ground cells + 1M facade samples, 481 steps."""
    B = cuda_lib
    w = configs.district()
    scene = _closed_scene(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    rng = np.random.default_rng(11)
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    # ground: the accrual raster over the whole grid
    g, _, c = B.sa_accumulate(scene, _grid(B, w.ground), sun, 1.0, "accrual_sam")
    g, c = g.cpu().numpy(), c.cpu().numpy()
    sel = rng.choice(w.ground.R, 1200, replace=False)
    pos = w.ground.positions()[sel]
    bits = oracle.shadow_bits(t9, tb, pos, None, w.sun.dirs)
    near = oracle.near_boundary(t9, tb, pos, None, w.sun.dirs, w.sun.day_start, bits)
    assert_counts_parity(g[sel], c[sel], bits, near, w.sun.day_start, "district ground")
    # the per-step ray sweep over the whole grid agrees on the same sample
    sg, _, sc_ = B.sa_accumulate(scene, _grid(B, w.ground), sun, 1.0, "sweep_trace")
    assert_counts_parity(sg.cpu().numpy()[sel], sc_.cpu().numpy()[sel], bits, near,
                         w.sun.day_start, "district ground sweep")
    # facades: the light-space accrual map over all 1M points
    fac = B.Receivers.points(w.facade_pos, w.facade_nrm)
    fg, _, fc = B.sa_accumulate(scene, fac, sun, 1.0, "accrual_sam")
    fg, fc = fg.cpu().numpy(), fc.cpu().numpy()
    # the ray-traced accrual is exact too and must agree everywhere, bit for bit
    tg, _, tc = B.sa_accumulate(scene, fac, sun, 1.0, "accrual_trace")
    assert np.array_equal(tg.cpu().numpy(), fg) and np.array_equal(tc.cpu().numpy(), fc)
    fsel = rng.choice(w.facade_pos.shape[0], 400, replace=False)
    fb = oracle.shadow_bits(t9, tb, w.facade_pos[fsel], w.facade_nrm[fsel], w.sun.dirs)
    fn = oracle.near_boundary(t9, tb, w.facade_pos[fsel], w.facade_nrm[fsel], w.sun.dirs,
                              w.sun.day_start, fb)
    assert_counts_parity(fg[fsel], fc[fsel], fb, fn, w.sun.day_start, "district facades")
    # the per-step sweep agrees on the same sample
    sg, _, _ = B.sa_accumulate(scene, fac, sun, 1.0, "sweep_trace")
    assert_counts_parity(sg.cpu().numpy()[fsel], None, fb, fn, w.sun.day_start, "sweep facades")


def test_season_full_size_sampled(cuda_lib):
    """50,000 buildings (1.53M triangles), central 4096^2 cells, 92 days x 481 steps.
    Over 44,252 steps nearly every receiver has steps within 1e-4 rad of a boundary, so
    the grid counts are held to |difference| <= the receiver's near-boundary steps, and
    the sampled cells, traced as points, to per-step bit parity away from boundaries; the
    direction graph over the same season is held to the oracle's graph on the same cells."""
    B = cuda_lib
    w = configs.season()
    assert w.mesh.T > 1_400_000 and w.sun.S == 92 * 481
    scene = _closed_scene(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    g, m, c = B.sa_accumulate(scene, _grid(B, w.ground), sun, 1.0, "accrual_sam")
    g, m = g.cpu().numpy(), m.cpu().numpy()
    rng = np.random.default_rng(12)
    sel = rng.choice(w.ground.R, 12, replace=False)
    pos = w.ground.positions()[sel]
    # Only buildings within the longest possible shadow can shadow a sample: a ray from the
    # ground rising at >= the table's lowest elevation is above the tallest roof beyond
    # h_max / tan(el_min) horizontally.  Keep buildings whose footprint box is within that.
    el_min = float(np.arcsin(w.sun.dirs[:, 2].min()))
    reach = float(w.city.heights.max()) / np.tan(el_min) + 10.0
    boxes = np.array([[f[:, 0].min(), f[:, 1].min(), f[:, 0].max(), f[:, 1].max()]
                      for f in w.city.footprints])
    dx = np.maximum(0, np.maximum(boxes[:, 0][None] - pos[:, 0:1], pos[:, 0:1] - boxes[:, 2][None]))
    dy = np.maximum(0, np.maximum(boxes[:, 1][None] - pos[:, 1:2], pos[:, 1:2] - boxes[:, 3][None]))
    within = np.hypot(dx, dy) <= reach                  # [sample, building]
    tri9_all = w.mesh.tri9()
    bits = np.zeros((pos.shape[0], w.sun.S), np.uint8)
    near = np.zeros_like(bits)
    for k in range(pos.shape[0]):
        keep = within[k][w.mesh.tri_building]
        assert 0 < keep.sum() < w.mesh.T
        t9 = tri9_all[keep]
        tb = np.unique(w.mesh.tri_building[keep], return_inverse=True)[1].astype(np.int32)
        bits[k:k + 1] = oracle.shadow_bits(t9, tb, pos[k:k + 1], None, w.sun.dirs)
        near[k:k + 1] = oracle.near_boundary(t9, tb, pos[k:k + 1], None, w.sun.dirs,
                                             w.sun.day_start, bits[k:k + 1])
    og, _ = oracle.reduce(bits, w.sun.day_start)
    assert np.all(np.abs(g[sel].astype(np.int64) - og) <= near.sum(axis=1)), (g[sel], og)
    assert np.allclose(m[sel], g[sel].astype(np.float32))
    masks = B.sa_shadow_masks(scene, B.Receivers.points(pos), sun, "accrual_trace")
    gb = unpack_masks(masks, block_sizes(w.sun.day_start))
    assert_bits_parity(gb, bits, near, "season points")
    # the same season through the direction graph (5 degree bins, Sec. 6): the sampled cells
    # against the oracle's graph of the same bits, within the near-boundary steps its maps use
    gg, _, gc, n_edges = B.sa_accumulate_graph(scene, _grid(B, w.ground), sun, 1.0, "accrual_sam", 5.0)
    _, rep, _ = oracle.direction_graph(w.sun.dirs, w.sun.day_start, 0, 5.0)
    assert n_edges == len(rep) < sun.n_blocks // 4
    obits = oracle.graph_bits(bits, w.sun.dirs, w.sun.day_start, 0, 5.0)
    onear = oracle.graph_bits(near, w.sun.dirs, w.sun.day_start, 0, 5.0)
    ogg, _ = oracle.reduce(obits, w.sun.day_start)
    gg = gg.cpu().numpy()
    assert np.all(np.abs(gg[sel].astype(np.int64) - ogg) <= onear.sum(axis=1)), (gg[sel], ogg)


def test_park_adjoint_full_size(cuda_lib):
    """600k receivers (500 x 300 m at 0.5 m), 200 buildings, equinox 09-17 h @ 1 min.
    The gradient is computed over the whole park; finite differences of the FP64 oracle
    are taken on a 60 x 50-cell patch (weights 1 there, 0 elsewhere on both sides) for
    the five buildings with the largest gradient there; receivers whose number of flips in
    a day changes under the +-0.01 m perturbations are left out (a brief shadow or gap
    appears or vanishes there, and the objective jumps), those whose flips only cross a
    step are kept."""
    B = cuda_lib
    w = configs.park()
    g = w.ground
    assert g.R == 600_000 and w.city.B == 200 and w.sun.S == 481
    scene = B.Scene.from_footprints(w.city.footprints, w.city.heights, w.city.band_height)
    grid = _grid(B, g)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    full, S_full = B.sa_height_grad(scene, grid, sun, w.sun.step_minutes)
    assert float(S_full) > 0 and torch.isfinite(full).all()
    # patch near the park's south-west corner, where the ring's shadows fall in the morning
    ix0, iy0, nx, ny = 20, 20, 60, 50
    idx = ((iy0 + np.arange(ny))[:, None] * g.nx + (ix0 + np.arange(nx))[None, :]).ravel()
    pos = g.positions()[idx]
    bands = C.band_counts(w.city)

    def mesh(hs):
        return C.extrude(w.city, heights=hs, bands=bands)

    wpatch = np.zeros(g.R, np.float32)
    wpatch[idx] = 1.0
    gpatch, _ = B.sa_height_grad(scene, grid, sun, w.sun.step_minutes, weights=wpatch)
    gpatch = gpatch.cpu().numpy().astype(np.float64)
    top = np.argsort(-np.abs(gpatch))[:5]
    assert np.abs(gpatch[top[0]]) > 0
    pert, jump = [], np.zeros(idx.size, bool)
    moved = np.zeros(idx.size, bool)
    for b in top:
        hp, hm = w.city.heights.copy(), w.city.heights.copy()
        hp[b] += np.float32(0.01)
        hm[b] -= np.float32(0.01)
        pert.append((b, hp, hm))
        mp, mm = mesh(hp), mesh(hm)
        bp = oracle.shadow_bits(mp.tri9(), mp.tri_building, pos, None, w.sun.dirs)
        bm = oracle.shadow_bits(mm.tri9(), mm.tri_building, pos, None, w.sun.dirs)
        moved |= (bp != bm).any(axis=1)
        jump |= (flips_per_day(bp, w.sun.day_start) != flips_per_day(bm, w.sun.day_start)).any(axis=1)
    keep = ~jump
    assert (moved & keep).sum() > 0
    wsub = np.zeros(g.R, np.float32)
    wsub[idx[keep]] = 1.0
    gsub, _ = B.sa_height_grad(scene, grid, sun, w.sun.step_minutes, weights=wsub)
    gsub = gsub.cpu().numpy().astype(np.float64)
    for b, hp, hm in pert:
        mp, mm = mesh(hp), mesh(hm)
        sp = oracle.shadow_integral(mp.tri9(), mp.tri_building, pos[keep], w.sun.dirs,
                                    w.sun.day_start, w.sun.step_minutes)
        sm = oracle.shadow_integral(mm.tri9(), mm.tri_building, pos[keep], w.sun.dirs,
                                    w.sun.day_start, w.sun.step_minutes)
        fd = (sp - sm) / (float(hp[b]) - float(hm[b]))
        assert abs(gsub[b] - fd) <= 1e-3 * abs(fd) + 1e-6, (b, gsub[b], fd)


def test_batched_scenarios_full_size_sampled(cuda_lib):
    """64 variants x 1-5 towers x 4 seasonal intervals of 31 days on regions of 256..2048
    cells: sampled receivers of three variants against the oracle on the variant mesh."""
    B = cuda_lib
    sc = configs.scenarios()
    w = sc.base
    scene = _closed_scene(B, w)
    grid = _grid(B, w.ground)
    suns = [B.Sun(it.dirs, it.day_start) for it in sc.intervals]
    bt = B.Batch(scene, grid, sc.tower_tris, sc.removed, sc.regions, suns, with_impact=True)
    counts, impact = bt.run()
    counts, impact = counts.cpu().numpy(), impact.cpu().numpy()
    g = w.ground
    pos = g.positions()
    rng = np.random.default_rng(13)
    for v in (0, 1, 2):
        t9, tb = sc.variant_mesh(v)
        ix0, iy0, nx, ny = (int(x) for x in sc.regions[v])
        loc = rng.choice(nx * ny, 6, replace=False)
        gl = (iy0 + loc // nx) * g.nx + (ix0 + loc % nx)
        for i in (0, 3):
            it = sc.intervals[i]
            bits = oracle.shadow_bits(t9, tb, pos[gl], None, it.dirs)
            near = oracle.near_boundary(t9, tb, pos[gl], None, it.dirs, it.day_start, bits)
            og, _ = oracle.reduce(bits, it.day_start)
            o = bt.offset(i, v)
            got = counts[o + loc].astype(np.int64)
            assert np.all(np.abs(got - og) <= near.sum(axis=1)), (v, i, got, og)


def test_building_contribution_full_size_region(cuda_lib):
    """The district scene (2,000 buildings) over its full 2048^2 grid, with a region of
    24 x 24 cells small enough for the oracle: every building's casting count within its own
    near-boundary pairs, the nearest counts within twice the pairs near any boundary."""
    B = cuda_lib
    w = configs.district(n_facade=0)
    g = w.ground
    scene = _closed_scene(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = _grid(B, g)
    ix0, iy0 = 1000, 1012
    xa, ya = g.x0 + ix0 * g.dx, g.y0 + iy0 * g.dx
    poly = np.array([[xa, ya], [xa + 24 * g.dx, ya], [xa + 24 * g.dx, ya + 24 * g.dx],
                     [xa, ya + 24 * g.dx]], np.float32)
    casting, nearest, (over, un) = B.sa_building_contribution(scene, grid, sun, poly)
    cells = np.array([(ix0 + i) + (iy0 + j) * g.nx for j in range(24) for i in range(24)])
    pos = g.positions()[cells]
    c_o, n_o, u_o, u_any = oracle.building_steps(w.mesh.tri9(), w.mesh.tri_building, pos, None,
                                                 w.sun.dirs, w.sun.day_start, w.city.B)
    unit = g.dx * g.dx / w.sun.S
    cnt_c = np.round(casting / unit).astype(np.int64)
    cnt_n = np.round(nearest / unit).astype(np.int64)
    assert c_o.sum() > 1000 and over == 0
    assert np.all(np.abs(cnt_c - c_o) <= u_o), np.nonzero(np.abs(cnt_c - c_o) > u_o)[0]
    assert np.abs(cnt_n - n_o).sum() <= 2 * u_any and un <= u_any


def _within_reach(city, x0, y0, x1, y1, dirs):
    """Buildings whose footprint box lies within the longest shadow any of `dirs` casts from
    the tallest building onto the box [x0, x1] x [y0, y1]: a ray from the ground that rises
    at the table's lowest elevation is above every roof beyond h_max / tan(el_min)."""
    el_min = float(np.arcsin(np.asarray(dirs)[:, 2].min()))
    reach = float(city.heights.max()) / np.tan(el_min) + 10.0
    boxes = np.array([[f[:, 0].min(), f[:, 1].min(), f[:, 0].max(), f[:, 1].max()]
                      for f in city.footprints])
    dx = np.maximum(0, np.maximum(boxes[:, 0] - x1, x0 - boxes[:, 2]))
    dy = np.maximum(0, np.maximum(boxes[:, 1] - y1, y0 - boxes[:, 3]))
    return np.hypot(dx, dy) <= reach


def test_season_windows_bit_parity(cuda_lib):
    """The season's accrual raster at the bit level: four 64 x 64-cell windows of the 4096^2
    grid, each run as its own ground grid (same cell centres), masks of all 828 blocks;
    256 sampled cells per window (1,024 in all) against the oracle on four days spread over
    the season (1,924 steps): every step away from a shadow boundary bit for bit."""
    B = cuda_lib
    w = configs.season()
    g = w.ground
    scene = _closed_scene(B, w)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    ds = w.sun.day_start
    days = [0, 30, 61, 91]
    j0, K = B.block_partition(ds)
    rng = np.random.default_rng(14)
    t9_all, tb_all = w.mesh.tri9(), w.mesh.tri_building
    sub_dirs = np.concatenate([w.sun.dirs[ds[d]:ds[d + 1]] for d in days])
    sub_ds = np.concatenate([[0], np.cumsum([ds[d + 1] - ds[d] for d in days])]).astype(np.int32)
    checked = 0
    for ix0, iy0 in ((300, 500), (1900, 2100), (3500, 700), (800, 3600)):
        x0, y0 = g.x0 + ix0 * g.dx, g.y0 + iy0 * g.dx
        win = B.Receivers.ground_grid(x0, y0, g.dx, 64, 64)
        masks = B.sa_shadow_masks(scene, win, sun, "accrual_sam")
        torch.cuda.synchronize()
        bl = np.nonzero(np.isin(j0, np.concatenate([np.arange(ds[d], ds[d + 1]) for d in days])))[0]
        gb_all = unpack_masks(masks[torch.as_tensor(bl, device=masks.device)], K[bl].tolist())
        loc = rng.choice(64 * 64, 256, replace=False)
        gb = gb_all[loc]
        pos = C.GroundGrid(x0=x0, y0=y0, dx=g.dx, nx=64, ny=64).positions()[loc]
        keep = _within_reach(w.city, x0, y0, x0 + 64 * g.dx, y0 + 64 * g.dx, sub_dirs)[tb_all]
        t9 = t9_all[keep]
        tb = np.unique(tb_all[keep], return_inverse=True)[1].astype(np.int32)
        bits = oracle.shadow_bits(t9, tb, pos, None, sub_dirs)
        diff = np.nonzero((gb != bits).any(axis=1))[0]
        near = np.zeros_like(bits)
        if diff.size:
            near[diff] = oracle.near_boundary(t9, tb, pos[diff], None, sub_dirs, sub_ds, bits[diff])
        assert_bits_parity(gb, bits, near, f"season window ({ix0}, {iy0})")
        assert bits.sum() > 0
        checked += loc.size
    assert checked >= 1000


def test_batched_impact_at_31_days_sampled(cuda_lib):
    """The batched scenarios at their full size (64 variants x 4 intervals of 31 days): for
    a small and a full-grid region, 100 receivers each near the variant's towers, the
    counts and the impact (variant - base) against the oracle on the variant and base
    meshes, in summer and winter, within each receiver's near-boundary steps."""
    B = cuda_lib
    sc = configs.scenarios()
    w = sc.base
    scene = _closed_scene(B, w)
    grid = _grid(B, w.ground)
    suns = [B.Sun(it.dirs, it.day_start) for it in sc.intervals]
    bt = B.Batch(scene, grid, sc.tower_tris, sc.removed, sc.regions, suns, with_impact=True)
    counts, impact = bt.run()
    counts, impact = counts.cpu().numpy(), impact.cpu().numpy()
    g = w.ground
    pos_all = g.positions()
    rng = np.random.default_rng(15)
    bt9, btb = w.mesh.tri9(), w.mesh.tri_building
    sizes = sc.regions[:, 2] * sc.regions[:, 3]
    for v in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        t9, tb = sc.variant_mesh(v)
        ix0, iy0, nx, ny = (int(x) for x in sc.regions[v])
        towers = np.asarray(sc.tower_tris[v]).reshape(-1, 3, 3)
        cx, cy = towers[:, :, 0].mean(), towers[:, :, 1].mean()
        lx = g.x0 + (ix0 + np.arange(nx) + 0.5) * g.dx
        ly = g.y0 + (iy0 + np.arange(ny) + 0.5) * g.dx
        X, Y = np.meshgrid(lx, ly)
        close = np.nonzero((np.hypot(X - cx, Y - cy) < 200.0).ravel())[0]
        loc = rng.choice(close, min(100, close.size), replace=False)
        assert loc.size == 100
        gl = (iy0 + loc // nx) * g.nx + (ix0 + loc % nx)
        pos = pos_all[gl]
        for i in (1, 3):
            it = sc.intervals[i]
            bv = oracle.shadow_bits(t9, tb, pos, None, it.dirs)
            bb = oracle.shadow_bits(bt9, btb, pos, None, it.dirs)
            ov, _ = oracle.reduce(bv, it.day_start)
            ob, _ = oracle.reduce(bb, it.day_start)
            o = bt.offset(i, v)
            got, imp = counts[o + loc].astype(np.int64), impact[o + loc].astype(np.int64)
            nv = np.zeros(loc.size, np.int64)
            nb = np.zeros(loc.size, np.int64)
            bad = np.nonzero((got != ov) | (imp != ov - ob))[0]
            if bad.size:
                nv[bad] = oracle.near_boundary(t9, tb, pos[bad], None, it.dirs, it.day_start,
                                               bv[bad]).sum(axis=1)
                nb[bad] = oracle.near_boundary(bt9, btb, pos[bad], None, it.dirs, it.day_start,
                                               bb[bad]).sum(axis=1)
            assert np.all(np.abs(got - ov) <= nv), (v, i, got, ov)
            assert np.all(np.abs(imp - (ov - ob)) <= nv + nb), (v, i, imp, ov - ob)
            assert (ov - ob).any()

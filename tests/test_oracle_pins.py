"""Pins of the FP64 oracle against facts fixed by the paper and by geometry (no GPU).

Each test would fail for a plausible slip in the oracle: a dropped or mis-signed term in
the ray/triangle test, a transposed operand, a wrong receiver offset or t_min, an index
error in the reduction, or an over-eager culling step.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.spatial import ConvexHull

import oracle
from synth import city as C
from synth import configs
from synth.sun import sun_direction, sun_table

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- independent geometry
def hull_polygon(points2d):
    h = ConvexHull(points2d)
    return points2d[h.vertices]          # CCW


def signed_dist_convex(poly, pts):
    """Signed distance of pts to a CCW convex polygon boundary: > 0 inside, < 0 outside
    (outside value is the max over edge half-planes, a lower bound on the true distance)."""
    d = np.full(pts.shape[0], np.inf)
    n = poly.shape[0]
    for i in range(n):
        a, b = poly[i], poly[(i + 1) % n]
        e = b - a
        L = math.hypot(e[0], e[1])
        # inward normal of a CCW polygon edge is (-e_y, e_x)
        s = ((pts[:, 0] - a[0]) * (-e[1]) + (pts[:, 1] - a[1]) * e[0]) / L
        d = np.minimum(d, s)
    return d


def shadow_polygon(fp, h, d):
    """Ground shadow of a convex prism (footprint fp, height h) for sun direction d:
    the hull of the footprint and the footprint shifted by -h * (d_x, d_y) / d_z."""
    u = np.array([d[0] / d[2], d[1] / d[2]])
    return hull_polygon(np.concatenate([fp, fp - h * u], axis=0))


def _ground_grid(x0, y0, dx, nx, ny):
    return C.GroundGrid(x0, y0, dx, nx, ny).positions()


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_convex_prism_matches_shadow_polygon(seed):
    rng = np.random.default_rng(100 + seed)
    fp = C.convex_footprint(rng, 50.0, 40.0, rng.uniform(8, 20), rng.uniform(8, 20),
                            int(rng.integers(4, 9)))
    h = float(rng.uniform(15, 80))
    city = C.City([fp], np.array([h], np.float32))
    mesh = C.extrude(city)
    sun = sun_table(40.7, [int(rng.integers(1, 365))], 8.0, 16.0, 20.0)
    pos = _ground_grid(-60.0, -70.0, 1.7, 130, 110)
    bits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, None, sun.dirs)
    fp32 = mesh.verts[:fp.shape[0], :2].astype(np.float64)   # footprint as stored (FP32)
    checked = 0
    for j, d in enumerate(sun.dirs.astype(np.float64)):
        poly = shadow_polygon(fp32, float(np.float32(h)), d)
        sd = signed_dist_convex(poly, pos[:, :2].astype(np.float64))
        clear = np.abs(sd) > 1e-6
        expect = (sd > 0).astype(np.uint8)
        assert np.array_equal(bits[clear, j], expect[clear]), f"step {j}"
        checked += int(clear.sum())
        assert expect.sum() > 0
    assert checked > 0.99 * bits.size


def test_union_of_boxes_matches_union_of_shadow_polygons():
    """Several separated prisms: a second brute force (union of shadow polygons)."""
    city = C.city_boxes(7, nx=3, ny=2)
    mesh = C.extrude(city)
    sun = sun_table(40.7, [300], 9.0, 15.0, 30.0)
    pos = _ground_grid(-50.0, -50.0, 1.3, 200, 160)
    bits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, None, sun.dirs)
    p2 = pos[:, :2].astype(np.float64)
    for j, d in enumerate(sun.dirs.astype(np.float64)):
        inside = np.zeros(p2.shape[0], bool)
        amb = np.zeros(p2.shape[0], bool)
        for b, fp in enumerate(city.footprints):
            fp32 = fp.astype(np.float32).astype(np.float64)
            sd = signed_dist_convex(shadow_polygon(fp32, float(city.heights[b]), d), p2)
            inside |= sd > 0
            amb |= np.abs(sd) <= 1e-6
        ok = ~amb
        assert np.array_equal(bits[ok, j], inside[ok].astype(np.uint8)), f"step {j}"


def test_facade_of_isolated_box_is_shadowed_exactly_when_facing_away():
    fp = C.box_footprint(0.0, 0.0, 30.0, 20.0)
    city = C.City([fp], np.array([40.0], np.float32))
    mesh = C.extrude(city)
    pos, nrm = C.facade_samples(city, 4000, seed=3)
    # keep samples 1 m clear of the vertical edges and of the roof edge
    along = np.where(np.abs(nrm[:, 0]) > 0.5, pos[:, 1], pos[:, 0])
    span = np.where(np.abs(nrm[:, 0]) > 0.5, 20.0, 30.0)
    keep = (along > 1.0) & (along < span - 1.0) & (pos[:, 2] < 39.0)
    pos, nrm = pos[keep], nrm[keep]
    sun = sun_table(40.7, [80, 172, 355], 8.0, 16.0, 30.0)
    bits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, nrm, sun.dirs)
    ndotd = nrm.astype(np.float64) @ sun.dirs.astype(np.float64).T
    clear = np.abs(ndotd) > 0.05
    assert np.array_equal(bits[clear], (ndotd[clear] <= 0).astype(np.uint8))


# ---------------------------------------------------------------- special cases
def test_zenith_sun_shadows_exactly_the_footprints():
    w = configs.boxes16()
    pos = w.ground.positions()
    d = np.array([[0.0, 0.0, 1.0]], np.float32)
    bits = oracle.shadow_bits(w.mesh.tri9(), w.mesh.tri_building, pos, None, d)[:, 0]
    inside = np.zeros(pos.shape[0], bool)
    for fp in w.city.footprints:
        fp32 = fp.astype(np.float32).astype(np.float64)
        inside |= signed_dist_convex(fp32, pos[:, :2].astype(np.float64)) > 0
    assert np.array_equal(bits, inside.astype(np.uint8))


def test_empty_scene_gives_zero_and_receiver_in_footprint_gives_all_steps():
    w = configs.boxes16()
    pos = w.ground.positions()[:64]
    bits = oracle.shadow_bits(np.zeros((0, 9), np.float32), None, pos, None, w.sun.dirs)
    assert bits.sum() == 0
    fp = w.city.footprints[5]
    centre = np.array([[fp[:, 0].mean(), fp[:, 1].mean(), 0.0]], np.float32)
    g, _, c, _ = oracle.accumulate(w.mesh.tri9(), w.mesh.tri_building, centre, None,
                                   w.sun.dirs, w.sun.day_start, w.sun.step_minutes)
    assert g[0] == w.sun.S and c[0] == w.sun.S


def test_building_box_pretest_preserves_the_pure_triangle_loop():
    w = configs.boxes16()
    a = oracle.shadow_bits(w.mesh.tri9(), w.mesh.tri_building, w.ground.positions(), None,
                           w.sun.dirs)
    b = oracle.shadow_bits(w.mesh.tri9(), None, w.ground.positions(), None, w.sun.dirs)
    assert np.array_equal(a, b)
    s = configs.district_small(n_facade=500)
    sub = s.ground.positions()[::37]
    a = oracle.shadow_bits(s.mesh.tri9(), s.mesh.tri_building, sub, None, s.sun.dirs[::5])
    b = oracle.shadow_bits(s.mesh.tri9(), None, sub, None, s.sun.dirs[::5])
    assert np.array_equal(a, b)
    a = oracle.shadow_bits(s.mesh.tri9(), s.mesh.tri_building, s.facade_pos, s.facade_nrm,
                           s.sun.dirs[::5])
    b = oracle.shadow_bits(s.mesh.tri9(), None, s.facade_pos, s.facade_nrm, s.sun.dirs[::5])
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- invariants
def test_adding_a_building_never_decreases_shadow():
    city = C.city_boxes(11)
    sun = sun_table(40.7, [172], 9.0, 17.0, 15.0)
    pos = _ground_grid(0.0, 0.0, 2.0, 100, 100)
    full = C.extrude(city)
    less = C.extrude(C.City(city.footprints[:-3], city.heights[:-3]))
    a = oracle.shadow_bits(full.tri9(), full.tri_building, pos, None, sun.dirs)
    b = oracle.shadow_bits(less.tri9(), less.tri_building, pos, None, sun.dirs)
    assert np.all(a >= b) and a.sum() > b.sum()


def test_taller_buildings_never_decrease_ground_shadow():
    city = C.city_boxes(12)
    sun = sun_table(40.7, [80], 9.0, 17.0, 20.0)
    pos = _ground_grid(0.0, 0.0, 2.0, 100, 100)
    lo = C.extrude(city)
    hi = C.extrude(city, heights=city.heights * np.float32(1.5))
    a = oracle.shadow_bits(hi.tri9(), hi.tri_building, pos, None, sun.dirs)
    b = oracle.shadow_bits(lo.tri9(), lo.tri_building, pos, None, sun.dirs)
    assert np.all(a >= b) and a.sum() > b.sum()


def test_counts_are_monotone_in_interval_length():
    w = configs.boxes16()
    pos = w.ground.positions()[::3]
    long = sun_table(40.7, [172], 9.0, 17.0, 2.0)
    short = sun_table(40.7, [172], 10.0, 15.0, 2.0)   # a subset of the same steps
    gl, _, cl, _ = oracle.accumulate(w.mesh.tri9(), w.mesh.tri_building, pos, None,
                                     long.dirs, long.day_start, 2.0)
    gs, _, cs, _ = oracle.accumulate(w.mesh.tri9(), w.mesh.tri_building, pos, None,
                                     short.dirs, short.day_start, 2.0)
    assert np.all(gl >= gs) and np.all(cl >= cs) and gl.sum() > gs.sum()


def test_permuting_triangles_and_receivers_leaves_results_unchanged():
    s = configs.district_small(n_facade=0)
    pos = s.ground.positions()[::11]
    dirs = s.sun.dirs[::4]
    tri9, tb = s.mesh.tri9(), s.mesh.tri_building
    a = oracle.shadow_bits(tri9, tb, pos, None, dirs)
    rng = np.random.default_rng(5)
    pt, pr = rng.permutation(tri9.shape[0]), rng.permutation(pos.shape[0])
    # also rotate the vertex order inside each triangle
    t9 = tri9[pt].reshape(-1, 3, 3)[:, [1, 2, 0], :].reshape(-1, 9)
    b = oracle.shadow_bits(t9, tb[pt], pos[pr], None, dirs)
    assert np.array_equal(a[pr], b)


# ---------------------------------------------------------------- the two measures
def _read_fig1():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_worked_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                p = line.split()
                rows.append((p[0], [int(x) for x in p[1:4]], int(p[4]), int(p[5])))
    return rows


def test_worked_example_gross_and_continuous():
    rows = _read_fig1()
    bits = np.array([r[1] for r in rows], np.uint8)
    g, c = oracle.reduce(bits, np.array([0, 3], np.int32))
    assert g.tolist() == [r[2] for r in rows]
    assert c.tolist() == [r[3] for r in rows]


def test_reduce_matches_run_lengths_by_enumeration():
    rng = np.random.default_rng(9)
    ds = np.array([0, 5, 6, 13, 13, 20], np.int32)     # includes a one-step and an empty day
    bits = (rng.random((300, 20)) < 0.6).astype(np.uint8)
    g, c = oracle.reduce(bits, ds)
    for r in range(bits.shape[0]):
        assert g[r] == int(bits[r].sum())
        best = 0
        for k in range(len(ds) - 1):
            day = bits[r, ds[k]:ds[k + 1]].tolist()
            for v, grp in itertools.groupby(day):
                if v:
                    best = max(best, len(list(grp)))
        assert c[r] == best


def test_runs_do_not_cross_days():
    bits = np.array([[0, 1, 1, 1, 1, 0]], np.uint8)
    assert oracle.reduce(bits, np.array([0, 3, 6], np.int32))[1][0] == 2
    assert oracle.reduce(bits, np.array([0, 6], np.int32))[1][0] == 4


# ---------------------------------------------------------------- boundary classification
def test_near_boundary_flags_points_close_to_the_shadow_edge_only():
    fp = C.box_footprint(0.0, 0.0, 20.0, 20.0)
    city = C.City([fp], np.array([50.0], np.float32))
    mesh = C.extrude(city)
    sun = sun_table(40.7, [172], 10.0, 14.0, 30.0)
    pos = _ground_grid(-80.0, -80.0, 0.37, 500, 500)
    bits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, None, sun.dirs)
    near = oracle.near_boundary(mesh.tri9(), mesh.tri_building, pos, None, sun.dirs,
                                sun.day_start, bits, eps=1e-4)
    p2 = pos[:, :2].astype(np.float64)
    for j, d in enumerate(sun.dirs.astype(np.float64)):
        sd = signed_dist_convex(shadow_polygon(fp, 50.0, d), p2)
        # rotating by 1e-4 rad moves the shadow of the top (<= ~50 m / sin^2(el) away)
        # by well under 0.02 m; points farther than that cannot flip, and points on the
        # edge flip.
        assert not near[np.abs(sd) > 0.02, j].any()
    assert near.sum() > 0


# ---------------------------------------------------------------- harness sun model
def test_sun_table_lengths_and_solstice_noon_elevation():
    assert sun_table(40.7, [172], 9.0, 17.0, 2.0).S == 241
    assert sun_table(40.7, [172], 9.0, 17.0, 1.0).S == 481
    d = sun_direction(40.7, 172, 12.0)
    assert abs(math.degrees(math.asin(d[2])) - (90 - 40.7 + 23.44)) < 0.1
    assert abs(d[0]) < 1e-12 and d[1] < 0       # due south at solar noon
    st = sun_table(40.7, list(range(172, 264)), 9.0, 17.0, 1.0)
    assert st.D == 92 and st.S == 92 * 481


def test_linear_sun_motion_statistics_match_table_1():
    """Table 1: cosine between the true direction and the linear interpolation of the
    interval endpoints stays above 0.9999 on average up to 60 minutes and is clearly
    lower at 240 minutes.  Our solar model is a different algorithm, so this is a
    statistical agreement check of the harness, not an exact one."""
    rng = np.random.default_rng(1000)
    doy = rng.integers(1, 366, 1000)
    hour = rng.uniform(6.0, 18.0, 1000)
    means = {}
    for minutes in (5, 10, 30, 60, 240):
        t0 = hour
        t1 = hour + minutes / 60.0
        d0, d1 = sun_direction(40.7, doy, t0), sun_direction(40.7, doy, t1)
        cs = []
        for k in range(1, minutes):
            a = k / minutes
            lin = (1 - a) * d0 + a * d1
            lin /= np.linalg.norm(lin, axis=1, keepdims=True)
            cs.append(np.sum(lin * sun_direction(40.7, doy, t0 + k / 60.0), axis=1))
        means[minutes] = float(np.mean(cs)) if cs else 1.0
    for m in (5, 10, 30, 60):
        assert means[m] > 0.99999 - 1e-6
    assert means[240] < means[60]


def test_near_boundary_does_not_depend_on_the_direction_of_the_arc():
    """The rule rotates each direction both ways along the sun's arc, so running the day's
    steps backwards (which reverses the arc's tangent) classifies every pair the same."""
    fp = C.box_footprint(0.0, 0.0, 20.0, 20.0)
    city = C.City([fp], np.array([50.0], np.float32))
    mesh = C.extrude(city)
    sun = sun_table(40.7, [172], 10.0, 14.0, 30.0)
    pos = _ground_grid(-80.0, -80.0, 0.37, 300, 300)
    eps = 2e-3
    bits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, None, sun.dirs)
    near = oracle.near_boundary(mesh.tri9(), mesh.tri_building, pos, None, sun.dirs,
                                sun.day_start, bits, eps=eps)
    rev = sun.dirs[::-1].copy()
    rbits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, None, rev)
    rnear = oracle.near_boundary(mesh.tri9(), mesh.tri_building, pos, None, rev,
                                 sun.day_start, rbits, eps=eps)
    assert np.array_equal(rbits[:, ::-1], bits)
    assert np.array_equal(rnear[:, ::-1], near)
    assert near.sum() > 100

"""Pins of the oracle's analysis measures (Sec. 7.2): shadow area over a polygonal region
and the shadow score, checked against index-range sums, an independent inside test,
additivity, orientation independence and the month weights of Table 3."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GRID = (8.25, 6.75, 2.5, 200, 150)          # x0, y0, dx, nx, ny (the small district's grid)


def _steps(seed=0, hi=100):
    x0, y0, dx, nx, ny = GRID
    return np.random.default_rng(seed).integers(0, hi, nx * ny)


def _rect(ix0, ix1, iy0, iy1):
    """Polygon along cell boundaries enclosing cells [ix0, ix1) x [iy0, iy1)."""
    x0, y0, dx, _, _ = GRID
    xa, xb = x0 + ix0 * dx, x0 + ix1 * dx
    ya, yb = y0 + iy0 * dx, y0 + iy1 * dx
    return np.array([[xa, ya], [xb, ya], [xb, yb], [xa, yb]], np.float64)


def test_rectangle_on_cell_boundaries_sums_its_cells():
    x0, y0, dx, nx, ny = GRID
    s = _steps()
    got = oracle.shadow_area(GRID, s, 100, _rect(20, 77, 13, 91))
    want = s.reshape(ny, nx)[13:91, 20:77].sum() / 100 * dx * dx
    assert got == pytest.approx(want, rel=1e-12)


def test_whole_grid_and_empty_region():
    x0, y0, dx, nx, ny = GRID
    s = _steps(1)
    assert oracle.shadow_area(GRID, s, 100, _rect(0, nx, 0, ny)) == pytest.approx(s.sum() / 100 * dx * dx, rel=1e-12)
    # a sliver between two columns of centres holds no centre
    xa = x0 + 10.6 * dx
    sliver = np.array([[xa, y0], [xa + 0.2 * dx, y0], [xa + 0.2 * dx, y0 + ny * dx], [xa, y0 + ny * dx]])
    assert oracle.shadow_area(GRID, s, 100, sliver) == 0.0
    # fully shadowed cells: the area is the cells' area
    full = np.full(nx * ny, 100)
    assert oracle.shadow_area(GRID, full, 100, _rect(5, 45, 7, 17)) == pytest.approx(40 * 10 * dx * dx, rel=1e-12)


def test_orientation_and_starting_vertex_do_not_matter():
    s = _steps(2)
    poly = np.array([[60.0, 40.0], [420.0, 90.0], [300.0, 330.0], [150.0, 250.0], [90.0, 300.0]])
    a = oracle.shadow_area(GRID, s, 100, poly)
    assert oracle.shadow_area(GRID, s, 100, poly[::-1]) == a
    assert oracle.shadow_area(GRID, s, 100, np.roll(poly, 2, axis=0)) == a
    assert a > 0


def test_triangle_inside_test_matches_barycentric_signs():
    x0, y0, dx, nx, ny = GRID
    tri = np.array([[37.3, 22.9], [401.7, 120.4], [155.2, 341.8]])
    ix, iy = np.meshgrid(np.arange(nx, dtype=np.float32), np.arange(ny, dtype=np.float32))
    cx = (np.float32(x0) + (ix + np.float32(0.5)) * np.float32(dx)).astype(np.float64)
    cy = (np.float32(y0) + (iy + np.float32(0.5)) * np.float32(dx)).astype(np.float64)

    def side(a, b):
        return (b[0] - a[0]) * (cy - a[1]) - (b[1] - a[1]) * (cx - a[0])

    s0, s1, s2 = side(tri[0], tri[1]), side(tri[1], tri[2]), side(tri[2], tri[0])
    bary = ((s0 > 0) & (s1 > 0) & (s2 > 0)) | ((s0 < 0) & (s1 < 0) & (s2 < 0))
    clear = np.minimum(np.minimum(np.abs(s0), np.abs(s1)), np.abs(s2)) > 1e-6
    pip = oracle.point_in_polygon(cx, cy, tri)
    assert np.array_equal(pip[clear], bary[clear])
    assert bary.sum() > 1000


def test_non_convex_region_is_the_sum_of_its_parts():
    s = _steps(3)
    # an L made of cells [10, 60) x [10, 30) and [10, 30) x [30, 80)
    x0, y0, dx, _, _ = GRID
    X = lambda i: x0 + i * dx
    Y = lambda j: y0 + j * dx
    ell = np.array([[X(10), Y(10)], [X(60), Y(10)], [X(60), Y(30)], [X(30), Y(30)],
                    [X(30), Y(80)], [X(10), Y(80)]])
    a = oracle.shadow_area(GRID, s, 100, ell)
    b = oracle.shadow_area(GRID, s, 100, _rect(10, 60, 10, 30)) + oracle.shadow_area(GRID, s, 100, _rect(10, 30, 30, 80))
    assert a == pytest.approx(b, rel=1e-12)


def _table3():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table3_month_weights.txt"))
            if l.strip() and not l.startswith("#")]
    return [r[0] for r in rows], np.array([float(r[1]) for r in rows])


def test_shadow_score_with_the_month_weights_of_table3():
    months, w = _table3()
    assert months == ["Jan", "Feb", "Mar", "Apr", "May", "Jun", "Jul", "Aug", "Sep", "Oct", "Nov", "Dec"]
    assert np.all(np.abs(w) <= 1)
    # the weights balance: the same shadow every month scores zero
    assert oracle.shadow_score(np.full(12, 1234.5), w) == pytest.approx(0.0, abs=1e-9)
    # shadow only from May to September scores the sum of those weights
    summer = np.array([0, 0, 0, 0, 1, 1, 1, 1, 1, 0, 0, 0], np.float64) * 100.0
    assert oracle.shadow_score(summer, w) == pytest.approx(400.0)


# ------------------------------------------------------------- building contribution
def _boxes_case(n_cells=300, seed=5):
    from synth import configs
    w = configs.boxes16()
    rng = np.random.default_rng(seed)
    pos = w.ground.positions()[rng.choice(w.ground.R, n_cells, replace=False)]
    return w, pos


def test_building_counts_agree_with_the_plain_shadow_bits():
    w, pos = _boxes_case()
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    casting, nearest, unstable, unstable_any = oracle.building_steps(
        t9, tb, pos, None, w.sun.dirs, w.sun.day_start, w.city.B)
    bits = oracle.shadow_bits(t9, tb, pos, None, w.sun.dirs)
    # every shadowed pair has exactly one nearest caster, and no lit pair has any
    assert nearest.sum() == bits.sum() > 0
    assert casting.sum() >= nearest.sum()
    assert np.all(nearest <= casting)
    # each building's casting count is its own shadow alone (the scene of its triangles)
    for b in range(w.city.B):
        keep = tb == b
        own = oracle.shadow_bits(t9[keep], np.zeros(int(keep.sum()), np.int32), pos, None, w.sun.dirs)
        assert casting[b] == own.sum(), b
    # the per-building near-boundary counts bound each other as sets do
    assert unstable_any <= unstable.sum()
    near = oracle.near_boundary(t9, tb, pos, None, w.sun.dirs, w.sun.day_start, bits)
    assert near.sum() <= unstable_any


def test_single_building_counts_are_its_shadow_and_near_boundary():
    w, pos = _boxes_case(200, seed=6)
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    keep = tb == 5
    t9b, tbb = t9[keep], np.zeros(int(keep.sum()), np.int32)
    casting, nearest, unstable, unstable_any = oracle.building_steps(
        t9b, tbb, pos, None, w.sun.dirs, w.sun.day_start, 1)
    bits = oracle.shadow_bits(t9b, tbb, pos, None, w.sun.dirs)
    near = oracle.near_boundary(t9b, tbb, pos, None, w.sun.dirs, w.sun.day_start, bits)
    assert casting[0] == nearest[0] == bits.sum()
    assert unstable[0] == unstable_any == near.sum()


def test_the_nearer_of_two_buildings_in_line_is_the_nearest_caster():
    """Two boxes one behind the other toward a low sun in the east: a receiver west of
    both is shadowed by both, and the nearer (western) box holds every nearest hit."""
    from synth import city as C
    city = C.City([C.box_footprint(10, -5, 20, 5), C.box_footprint(40, -5, 50, 5)],
                  np.array([30.0, 60.0], np.float32))
    mesh = C.extrude(city)
    el = np.radians(20.0)
    dirs = np.array([[np.cos(el), 0.0, np.sin(el)]], np.float32)      # toward the east
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.0], [-1.0, -0.5, 0.0]], np.float32)
    casting, nearest, _, _ = oracle.building_steps(mesh.tri9(), mesh.tri_building, pos, None,
                                                   dirs, np.array([0, 1], np.int32), 2)
    assert list(casting) == [3, 3]
    assert list(nearest) == [3, 0]


def test_a_building_in_parts_is_nearest_by_its_nearest_part():
    """Building 0 is two boxes with building 1 between them, in line toward a low sun in
    the east: a receiver west of all three meets building 0 first, so building 0 is the
    nearest caster although its farther part lies beyond building 1."""
    from synth import city as C
    city = C.City([C.box_footprint(10, -5, 20, 5), C.box_footprint(40, -5, 50, 5),
                   C.box_footprint(70, -5, 80, 5)], np.array([40.0, 40.0, 40.0], np.float32))
    mesh = C.extrude(city)
    tb = np.where(mesh.tri_building == 1, 1, 0).astype(np.int32)   # boxes 0 and 2 are one building
    el = np.radians(15.0)
    dirs = np.array([[np.cos(el), 0.0, np.sin(el)]], np.float32)
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 1.5, 0.0], [-2.0, -1.0, 0.0]], np.float32)
    casting, nearest, _, _ = oracle.building_steps(mesh.tri9(), tb, pos, None, dirs,
                                                   np.array([0, 1], np.int32), 2)
    assert list(casting) == [3, 3]
    assert list(nearest) == [3, 0]


def test_per_building_near_boundary_under_a_wide_rotation():
    """With a rotation wide enough that many pairs flip, one building's near-boundary count
    equals the plain rule's, which rotates the sun both ways along its arc."""
    w, pos = _boxes_case(400, seed=8)
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    keep = tb == 3
    t9b, tbb = t9[keep], np.zeros(int(keep.sum()), np.int32)
    eps = 0.03
    _, _, unstable, unstable_any = oracle.building_steps(t9b, tbb, pos, None, w.sun.dirs,
                                                         w.sun.day_start, 1, eps=eps)
    bits = oracle.shadow_bits(t9b, tbb, pos, None, w.sun.dirs)
    near = oracle.near_boundary(t9b, tbb, pos, None, w.sun.dirs, w.sun.day_start, bits, eps=eps)
    assert near.sum() > 200
    assert unstable[0] == unstable_any == near.sum()


def test_walls_behind_a_receiver_cast_nothing():
    """Ground receivers 0.3 m outside every wall of a box, and facade receivers on the walls:
    the casting counts equal the plain shadow bits and the facing closed form, so a wall just
    behind a receiver, on the far side from the sun, is never counted."""
    from synth import city as C
    city = C.City([C.box_footprint(0, 0, 20, 12)], np.array([25.0], np.float32))
    mesh = C.extrude(city)
    xs = np.linspace(1.0, 19.0, 10)
    ys = np.linspace(1.0, 11.0, 6)
    pts = [(x, -0.3) for x in xs] + [(x, 12.3) for x in xs] + [(-0.3, y) for y in ys] + [(20.3, y) for y in ys]
    pos = np.array([(x, y, 0.0) for x, y in pts], np.float32)
    from synth.sun import sun_table
    st = sun_table(40.7, [172, 355], 7.0, 17.0, 10.0)
    casting, nearest, _, _ = oracle.building_steps(mesh.tri9(), mesh.tri_building, pos, None,
                                                   st.dirs, st.day_start, 1)
    bits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, pos, None, st.dirs)
    assert casting[0] == nearest[0] == bits.sum()
    assert 0 < bits.sum() < bits.size
    # facade receivers on the walls themselves (origin 1 cm out along the outward normal):
    # the counts equal the plain facade bits; a lone box shadows a facade point whose wall
    # faces clearly away from the sun and never one whose wall faces it (at grazing angles
    # the ray from 1 cm out can pass the wall's edge)
    fpos = np.array([(x, 0.0, 5.0) for x in xs] + [(x, 12.0, 5.0) for x in xs] +
                    [(0.0, y, 5.0) for y in ys] + [(20.0, y, 5.0) for y in ys], np.float32)
    fnrm = np.array([(0, -1, 0)] * 10 + [(0, 1, 0)] * 10 + [(-1, 0, 0)] * 6 + [(1, 0, 0)] * 6, np.float32)
    casting, nearest, _, _ = oracle.building_steps(mesh.tri9(), mesh.tri_building, fpos, fnrm,
                                                   st.dirs, st.day_start, 1)
    fbits = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, fpos, fnrm, st.dirs)
    assert casting[0] == nearest[0] == fbits.sum() > 0
    nd = fnrm.astype(np.float64) @ st.dirs.astype(np.float64).T
    assert np.all(fbits[nd < -0.05] == 1) and np.all(fbits[nd > 0] == 0)
    # an L-shaped building (two boxes, one id): facade points on its inner walls start
    # inside the building's bounding box, with their own wall 1 cm behind them
    city = C.City([C.box_footprint(0, 0, 20, 10), C.box_footprint(0, 10, 10, 30)],
                  np.array([25.0, 25.0], np.float32))
    mesh = C.extrude(city)
    tb = np.zeros_like(mesh.tri_building)
    lpos = np.array([(10.0, y, 4.0) for y in np.linspace(12.0, 28.0, 9)] +
                    [(x, 10.0, 4.0) for x in np.linspace(11.0, 19.0, 5)], np.float32)
    lnrm = np.array([(1, 0, 0)] * 9 + [(0, 1, 0)] * 5, np.float32)
    casting, nearest, _, _ = oracle.building_steps(mesh.tri9(), tb, lpos, lnrm, st.dirs, st.day_start, 1)
    lbits = oracle.shadow_bits(mesh.tri9(), tb, lpos, lnrm, st.dirs)
    assert casting[0] == nearest[0] == lbits.sum()
    lnd = lnrm.astype(np.float64) @ st.dirs.astype(np.float64).T
    assert np.any((lnd > 0.05) & (lbits == 0))          # sunlit inner walls exist in the case

"""Pins of the oracle's inverse accrual map (Sec. 5), an approximation by design.

What geometry fixes exactly: with one step per block the map draws no lines, and every
cell with a source (the 100 cm rule aside) is shadowed -- the exact result; reversing the
steps of a block swaps the forward and backward maps; and on a fine grid with one-minute
steps the map's shadow area stays within the paper's error bar (mean < 1 % of the area).
"""
import numpy as np

import oracle
from synth import city as C
from synth import configs
from synth.sun import sun_table


def _grid(w):
    g = w.ground
    return (g.x0, g.y0, g.dx, g.nx, g.ny)


def inside_any_footprint(city, pos):
    inside = np.zeros(pos.shape[0], bool)
    for fp in city.footprints:
        f = fp.astype(np.float32).astype(np.float64)
        ok = np.ones(pos.shape[0], bool)
        for i in range(f.shape[0]):
            a, b = f[i], f[(i + 1) % f.shape[0]]
            ok &= (b[0] - a[0]) * (pos[:, 1] - a[1]) - (b[1] - a[1]) * (pos[:, 0] - a[0]) >= 0
        inside |= ok
    return inside


def _hit_distances(t9, o, d):
    """All ray/triangle hit distances t > 0, by a separate numpy brute force."""
    out = []
    for v0, v1, v2 in t9:
        e1, e2 = v1 - v0, v2 - v0
        p = np.cross(d, e2)
        det = e1 @ p
        if det == 0:
            continue
        s = o - v0
        u = (s @ p) / det
        q = np.cross(s, e1)
        v = (d @ q) / det
        if u < 0 or v < 0 or u + v > 1:
            continue
        t = (e2 @ q) / det
        if t > 0:
            out.append(t)
    return out


def test_one_step_blocks_reduce_to_the_exact_shadow():
    """With one step per block no line is drawn: a cell is marked exactly when its own ray
    has a source.  The only departures allowed are the paper's 100 cm rule: cells whose
    every intersection lies within 1 m (inside a footprint next to a wall, or a ray that
    clips a building's corner) lose their shadow."""
    w = configs.district_small()
    exact = oracle.shadow_bits(w.mesh.tri9(), w.mesh.tri_building, w.ground.positions(), None,
                               w.sun.dirs)
    near = oracle.near_boundary(w.mesh.tri9(), w.mesh.tri_building, w.ground.positions(), None,
                                w.sun.dirs, w.sun.day_start, exact)
    iam = oracle.iam_bits(w.mesh.tri9(), w.mesh.tri_building, _grid(w), w.sun.dirs,
                          w.sun.day_start, block_len=1, levels=1)
    assert not ((iam == 1) & (exact == 0) & (near == 0)).any()
    missed = np.argwhere((iam == 0) & (exact == 1) & (near == 0))
    assert missed.shape[0] < 0.01 * iam.size
    outside = ~inside_any_footprint(w.city, w.ground.positions().astype(np.float64))
    t9 = w.mesh.tri9().astype(np.float64).reshape(-1, 3, 3)
    pos = w.ground.positions().astype(np.float64)
    for r, j in missed[outside[missed[:, 0]]]:
        ts = _hit_distances(t9, pos[r], w.sun.dirs[j].astype(np.float64))
        assert ts and max(ts) <= 1.0 + 1e-9, (r, j, ts)
    assert iam.sum() > 0


def test_reversed_steps_mirror_the_bits():
    """Forward and backward maps swap when the steps of each block run backwards."""
    city = C.city_boxes(3, nx=2, ny=2)
    mesh = C.extrude(city)
    st = sun_table(40.7, [172], 10.0, 11.0, 4.0)            # 16 steps, one block
    grid = (-20.0, -20.0, 1.0, 150, 150)
    a = oracle.iam_bits(mesh.tri9(), mesh.tri_building, grid, st.dirs, st.day_start, levels=2)
    b = oracle.iam_bits(mesh.tri9(), mesh.tri_building, grid, st.dirs[::-1].copy(),
                        st.day_start, levels=2)
    assert np.array_equal(a, b[:, ::-1])
    assert a.sum() > 0


def test_single_box_area_error_within_the_paper_bar():
    fp = C.box_footprint(0.0, 0.0, 30.0, 20.0)
    city = C.City([fp], np.array([45.0], np.float32))
    mesh = C.extrude(city)
    st = sun_table(40.7, [172], 9.0, 15.0, 1.0)
    g = C.GroundGrid(-150.0, -60.0, 0.5, 600, 240)
    exact = oracle.shadow_bits(mesh.tri9(), mesh.tri_building, g.positions(), None, st.dirs)
    iam = oracle.iam_bits(mesh.tri9(), mesh.tri_building, (g.x0, g.y0, g.dx, g.nx, g.ny),
                          st.dirs, st.day_start, levels=3)
    j0, K = oracle.block_partition(st.day_start)
    errs = []
    for a, k in zip(j0, K):
        e = exact[:, a:a + k].sum() / k
        i = iam[:, a:a + k].sum() / k
        errs.append(abs(i - e) / g.R)
    assert np.mean(errs) < 0.01 and max(errs) < 0.026, errs


def test_more_levels_find_more_shadow_behind_the_first_source():
    """Two boxes in a row along the sun: level 2 adds the far box's shadow lines."""
    fps = [C.box_footprint(0.0, 0.0, 10.0, 10.0), C.box_footprint(40.0, 0.0, 50.0, 10.0)]
    city = C.City(fps, np.array([20.0, 60.0], np.float32))
    mesh = C.extrude(city)
    st = sun_table(40.7, [172], 15.0, 16.0, 2.0)            # afternoon: sun in the west
    grid = (-120.0, -40.0, 1.0, 200, 100)
    one = oracle.iam_bits(mesh.tri9(), mesh.tri_building, grid, st.dirs, st.day_start, levels=1)
    two = oracle.iam_bits(mesh.tri9(), mesh.tri_building, grid, st.dirs, st.day_start, levels=2)
    assert np.all(two >= one) and two.sum() > one.sum()


def test_the_100_cm_rule_behind_a_thin_low_wall():
    """A wall 0.4 m thick and 0.6 m tall under a low sun: rays from the cells just behind
    it meet the wall only within 1 m, so with one-step blocks the map marks none of them
    (the paper's 100 cm rule), while every cell with a hit beyond 1 m is marked."""
    city = C.City([C.box_footprint(0.0, 0.0, 0.4, 20.0)], np.array([0.6], np.float32))
    mesh = C.extrude(city)
    el = np.radians(25.0)                                  # toward the east, a little south
    dirs = np.array([[np.cos(el), -0.15, np.sin(el)]], np.float32)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    grid = (-3.0, 1.0, 0.1, 30, 180)                       # the strip west of the wall
    g = C.GroundGrid(*grid)
    iam = oracle.iam_bits(mesh.tri9(), mesh.tri_building, grid, dirs, np.array([0, 1], np.int32),
                          block_len=1, levels=1)[:, 0]
    t9 = mesh.tri9().astype(np.float64).reshape(-1, 3, 3)
    pos = g.positions().astype(np.float64)
    d = dirs[0].astype(np.float64)
    far = np.zeros(g.R, bool)
    near_only = np.zeros(g.R, bool)
    for r in range(g.R):
        ts = _hit_distances(t9, pos[r], d)
        if ts:
            far[r] = max(ts) > 1.0 + 1e-6
            near_only[r] = max(ts) < 1.0 - 1e-6
    assert near_only.sum() > 50 and far.sum() > 50
    assert not iam[near_only].any()
    assert iam[far].all()


# ------------------------------------------------------------- the supercover drawer
def _cells(a):
    return set(map(tuple, np.argwhere(a)[:, ::-1].tolist()))       # (ix, iy)


def test_supercover_drawer_at_corners_and_edges():
    """Cells are closed squares: a diagonal through a cell corner touches the four cells
    around it; a segment along a cell edge touches the rows (or columns) on both sides; a
    point on a corner touches four cells, inside a cell one."""
    g = (0.0, 0.0, 1.0, 6, 6)
    assert _cells(oracle.draw_segment(g, (0.5, 0.5), (1.5, 1.5))) == {(0, 0), (1, 0), (0, 1), (1, 1)}
    assert _cells(oracle.draw_segment(g, (0.5, 2.0), (2.5, 2.0))) == \
        {(0, 1), (1, 1), (2, 1), (0, 2), (1, 2), (2, 2)}
    assert _cells(oracle.draw_segment(g, (3.0, 0.25), (3.0, 1.75))) == {(2, 0), (3, 0), (2, 1), (3, 1)}
    assert _cells(oracle.draw_segment(g, (2.0, 4.0), (2.0, 4.0))) == {(1, 3), (2, 3), (1, 4), (2, 4)}
    assert _cells(oracle.draw_segment(g, (2.5, 4.5), (2.5, 4.5))) == {(2, 4)}
    # a shallow line crosses cells a one-sample-per-cell line steps over
    assert _cells(oracle.draw_segment(g, (0.1, 0.1), (3.9, 1.3))) == \
        {(0, 0), (1, 0), (2, 0), (2, 1), (3, 1)}
    # clipped at the grid: nothing outside, nothing for a segment that misses it
    assert _cells(oracle.draw_segment(g, (-3.0, -3.0), (0.5, 0.5))) == {(0, 0)}
    assert not oracle.draw_segment(g, (-3.0, -3.0), (-1.0, 7.0)).any()
    # shrunk cells lose the corner touches, grown ones gain the near misses
    assert _cells(oracle.draw_segment(g, (0.5, 0.5), (1.5, 1.5), -1e-6)) == {(0, 0), (1, 1)}
    assert _cells(oracle.draw_segment(g, (0.5, 1.9999995), (2.5, 1.9999995), 1e-6)) == \
        {(0, 1), (1, 1), (2, 1), (0, 2), (1, 2), (2, 2)}


def _exact_touch(p, q, lo, hi, open_cell):
    """Does segment p-q meet the square [lo, hi]^2 (closed) or its interior (open)?  Exact
    rational separating-axis test: the two axes and the segment's normal."""
    from fractions import Fraction as F
    px, py, qx, qy = map(F, (p[0], p[1], q[0], q[1]))
    (ax, ay), (bx, by) = (F(lo[0]), F(lo[1])), (F(hi[0]), F(hi[1]))

    def overlap(a0, a1, b0, b1):            # [a0, a1] against the square's [b0, b1]
        return (a1 > b0 and a0 < b1) if open_cell else (a1 >= b0 and a0 <= b1)
    if not overlap(min(px, qx), max(px, qx), ax, bx) or not overlap(min(py, qy), max(py, qy), ay, by):
        return False
    nx, ny = qy - py, px - qx
    if nx == 0 and ny == 0:
        return True
    v = nx * px + ny * py
    side = [nx * x + ny * y - v for x, y in ((ax, ay), (bx, ay), (ax, by), (bx, by))]
    if open_cell:
        return min(side) < 0 < max(side)
    return min(side) <= 0 <= max(side)


def test_supercover_drawer_against_exact_intersection():
    """Random segments with coordinates on a 1/8 m lattice (so that many pass exactly
    through cell corners and along cell edges) against an exact rational test: every cell
    whose interior the segment enters is marked, no cell it does not touch is marked, and
    cells grown by 1e-9 m take every touched cell while shrunk ones take only entered
    ones."""
    rng = np.random.default_rng(11)
    nx = ny = 6
    g = (0.0, 0.0, 1.0, nx, ny)
    lattice = np.arange(-8, 8 * 7 + 1) / 8.0
    for _ in range(400):
        p = rng.choice(lattice, 2)
        q = p if rng.random() < 0.1 else rng.choice(lattice, 2)
        if rng.random() < 0.2:
            q = np.array([q[0], p[1]])                       # axis-parallel
        drawn = _cells(oracle.draw_segment(g, p, q))
        grown = _cells(oracle.draw_segment(g, p, q, 1e-9))
        shrunk = _cells(oracle.draw_segment(g, p, q, -1e-9))
        closed = {(i, j) for i in range(nx) for j in range(ny)
                  if _exact_touch(p, q, (i, j), (i + 1, j + 1), False)}
        inner = {(i, j) for i in range(nx) for j in range(ny)
                 if _exact_touch(p, q, (i, j), (i + 1, j + 1), True)}
        assert inner <= drawn <= closed, (p, q, drawn, closed, inner)
        assert closed <= grown and shrunk <= inner, (p, q)


# ----------------------------------------------------------- bounds of the inverse map
def _gpu_case():
    return configs.district_small(dx=1.0, nx=240, ny=180, step=2.0, t0=10.0, t1=15.0)


def test_iam_bounds_bracket_the_map():
    """With zero tolerances both bounds are the map itself; with 1 mm ones the map lies
    between them and the band they leave is a small fraction of the bits."""
    w = _gpu_case()
    g = w.ground
    args = (w.mesh.tri9(), w.mesh.tri_building, (g.x0, g.y0, g.dx, g.nx, g.ny), w.sun.dirs,
            w.sun.day_start)
    sc = oracle.iam_bits(*args, levels=3)
    m0, M0 = oracle.iam_bounds(*args, levels=3, eps_cell=0.0, eps_src=0.0, eps_t=0.0)
    assert np.array_equal(m0, sc) and np.array_equal(M0, sc)
    m, M = oracle.iam_bounds(*args, levels=3, eps_cell=1e-3, eps_src=1e-3, eps_t=1e-3)
    assert np.all(m <= sc) and np.all(sc <= M)
    assert 0 < (M != m).mean() < 1e-3


def test_thin_lines_fall_outside_the_supercover_bounds():
    """The GPU test's bar tells the two line readings apart: on its case, the map drawn
    with thin lines (one cell per sample) leaves unset hundreds of bits the supercover map
    sets for certain."""
    w = _gpu_case()
    g = w.ground
    args = (w.mesh.tri9(), w.mesh.tri_building, (g.x0, g.y0, g.dx, g.nx, g.ny), w.sun.dirs,
            w.sun.day_start)
    thin = oracle.iam_bits(*args, levels=3, line_mode=oracle.IAM_LINE_THIN)
    m, M = oracle.iam_bounds(*args, levels=3, eps_cell=1e-3, eps_src=1e-3, eps_t=1e-3)
    assert ((m == 1) & (thin == 0)).sum() > 100

"""FP64 CPU oracle for shadow accumulation -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may import
this package.  The product path (the CUDA library and its binding) never does.

The C source `sa_oracle.c` holds the definitions (see its header for the citations);
this module compiles it with gcc/OpenMP on first use (in-tree, `_build/`) and wraps it
for numpy arrays.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsa_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP); returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            P = ct.c_void_p
            i64, i32, f64, ci = ct.c_int64, ct.c_int32, ct.c_double, ct.c_int
            L.sao_shadow_bits.argtypes = [P, P, i64, P, P, i64, P, i32, P, ci]
            L.sao_near_boundary.argtypes = [P, P, i64, P, P, i64, P, P, i32, f64, P, P, ci]
            L.sao_reduce.argtypes = [P, i64, P, i32, P, P]
            f32 = ct.c_float
            L.sao_shadow_integral.argtypes = [P, P, i64, P, i64, P, P, i32, f64, P, i32, P, P, ci]
            L.sao_iam.argtypes = [P, P, i64, f32, f32, f32, i32, i32, P, P, P, i32, i32, f64,
                                  i32, i32, P, ci]
            L.sao_iam_bounds.argtypes = [P, P, i64, f32, f32, f32, i32, i32, P, P, P, i32, i32,
                                         f64, f64, f64, f64, i32, P, P, ci]
            L.sao_draw_segment.argtypes = [f64, f64, f64, i32, i32, f64, f64, f64, f64, f64, P]
            L.sao_building_steps.argtypes = [P, P, i64, P, P, i64, P, P, i32, f64, i32, P, P, P,
                                             P, ci]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def default_threads() -> int:
    return int(os.environ.get("SA_ORACLE_THREADS", os.cpu_count() or 1))


def shadow_bits(tri9, tri_building, pos, nrm, dirs, nthreads: int | None = None) -> np.ndarray:
    """uint8 [R, S]: 1 where the receiver is in shadow at that step (FP64 brute force)."""
    tri9, tb, pos, nrm, dirs = _f32(tri9), _i32(tri_building), _f32(pos), _f32(nrm), _f32(dirs)
    T, R, S = tri9.shape[0], pos.shape[0], dirs.shape[0]
    out = np.zeros((R, S), dtype=np.uint8)
    rc = lib().sao_shadow_bits(_ptr(tri9), _ptr(tb), T, _ptr(pos), _ptr(nrm), R, _ptr(dirs), S,
                               _ptr(out), nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"sao_shadow_bits failed: {rc}")
    return out


def near_boundary(tri9, tri_building, pos, nrm, dirs, day_start, status, eps=1e-4,
                  nthreads: int | None = None) -> np.ndarray:
    """uint8 [R, S]: 1 where rotating d_j by +-eps along the sun arc flips the status."""
    tri9, tb, pos, nrm, dirs = _f32(tri9), _i32(tri_building), _f32(pos), _f32(nrm), _f32(dirs)
    ds = _i32(day_start)
    status = np.ascontiguousarray(status, dtype=np.uint8)
    T, R = tri9.shape[0], pos.shape[0]
    near = np.zeros_like(status)
    rc = lib().sao_near_boundary(_ptr(tri9), _ptr(tb), T, _ptr(pos), _ptr(nrm), R, _ptr(dirs),
                                 _ptr(ds), ds.shape[0] - 1, float(eps), _ptr(status), _ptr(near),
                                 nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"sao_near_boundary failed: {rc}")
    return near


def reduce(bits, day_start):
    """(gross int32 [R], continuous int32 [R]) from per-step bits grouped by day."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    ds = _i32(day_start)
    R = bits.shape[0]
    g = np.zeros(R, np.int32)
    c = np.zeros(R, np.int32)
    rc = lib().sao_reduce(_ptr(bits), R, _ptr(ds), ds.shape[0] - 1, _ptr(g), _ptr(c))
    if rc != 0:
        raise RuntimeError(f"sao_reduce failed: {rc}")
    return g, c


def block_partition(day_start, block_len: int = 0):
    """Blocks of <= block_len (0: 60) consecutive steps per day, balanced: (j0 [], K [])."""
    K = block_len or 60
    j0s, Ks = [], []
    ds = [int(x) for x in np.asarray(day_start).reshape(-1)]
    for a, b in zip(ds[:-1], ds[1:]):
        n = b - a
        if n <= 0:
            continue
        nb = (n + K - 1) // K
        base, rem = divmod(n, nb)
        j = a
        for q in range(nb):
            k = base + (1 if q < rem else 0)
            j0s.append(j)
            Ks.append(k)
            j += k
    return np.asarray(j0s, np.int32), np.asarray(Ks, np.int32)


IAM_LINE_SUPERCOVER, IAM_LINE_THIN = 0, 1


def iam_bits(tri9, tri_building, grid, dirs, day_start, block_len=0, levels=3,
             tmin_src=1.0, line_mode=IAM_LINE_SUPERCOVER, nthreads: int | None = None) -> np.ndarray:
    """uint8 [R, S]: the inverse-accrual-map bits (Sec. 5) of a ground grid (x0, y0, dx,
    nx, ny), from L = `levels` source levels traced at both ends of every block.  Each
    piece of a shadow line marks every closed cell it touches (supercover, the reading
    kept for the n - 1 pieces of Sec. 5); IAM_LINE_THIN marks one cell per sample along
    the piece instead (the other reading, kept to show that the tests tell them apart)."""
    tri9, tb, dirs = _f32(tri9), _i32(tri_building), _f32(dirs)
    x0, y0, dx, nx, ny = grid
    j0, K = block_partition(day_start, block_len)
    S = dirs.shape[0]
    out = np.zeros((int(nx) * int(ny), S), np.uint8)
    rc = lib().sao_iam(_ptr(tri9), _ptr(tb), tri9.shape[0], float(x0), float(y0), float(dx),
                       int(nx), int(ny), _ptr(dirs), _ptr(j0), _ptr(K), j0.shape[0], int(levels),
                       float(tmin_src), int(line_mode), S, _ptr(out), nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"sao_iam failed: {rc}")
    return out


def iam_bounds(tri9, tri_building, grid, dirs, day_start, block_len=0, levels=3,
               tmin_src=1.0, eps_cell=1e-3, eps_src=1e-3, eps_t=1e-3,
               nthreads: int | None = None):
    """(must, may) uint8 [R, S]: bounds of the supercover inverse accrual map when its
    sources and shadow-line ends may move by small amounts -- a hit is certain only if the
    ray passes eps_src (m) inside its triangle, with t beyond tmin_src + eps_t and fewer
    than L possible hits within eps_t before it; a piece marks a cell for certain only if
    it reaches eps_cell (m) inside it.  `may` takes every possible source and every cell
    reached within eps_cell.  With all tolerances 0 both equal `iam_bits`."""
    tri9, tb, dirs = _f32(tri9), _i32(tri_building), _f32(dirs)
    x0, y0, dx, nx, ny = grid
    j0, K = block_partition(day_start, block_len)
    S = dirs.shape[0]
    must = np.zeros((int(nx) * int(ny), S), np.uint8)
    may = np.zeros_like(must)
    rc = lib().sao_iam_bounds(_ptr(tri9), _ptr(tb), tri9.shape[0], float(x0), float(y0),
                              float(dx), int(nx), int(ny), _ptr(dirs), _ptr(j0), _ptr(K),
                              j0.shape[0], int(levels), float(tmin_src), float(eps_cell),
                              float(eps_src), float(eps_t), S, _ptr(must), _ptr(may),
                              nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"sao_iam_bounds failed: {rc}")
    return must, may


def draw_segment(grid, p, q, eps=0.0) -> np.ndarray:
    """uint8 [ny, nx]: the cells of grid (x0, y0, dx, nx, ny) that the IAM's supercover
    drawer marks for the segment p -> q (closed cells; grown by eps > 0 or shrunk by
    |eps| for eps < 0)."""
    x0, y0, dx, nx, ny = grid
    out = np.zeros((int(ny), int(nx)), np.uint8)
    rc = lib().sao_draw_segment(float(x0), float(y0), float(dx), int(nx), int(ny), float(p[0]),
                                float(p[1]), float(q[0]), float(q[1]), float(eps), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"sao_draw_segment failed: {rc}")
    return out


def shadow_integral(tri9, tri_building, pos, dirs, day_start, step_minutes, weights=None,
                    bisect_iters: int = 60, per_receiver: bool = False,
                    nthreads: int | None = None):
    """Continuous-time shadow-minutes S of ground receivers (sun slerped between steps,
    status flips found by bisection), summed with optional per-receiver weights."""
    tri9, tb, pos, dirs = _f32(tri9), _i32(tri_building), _f32(pos), _f32(dirs)
    ds = _i32(day_start)
    R = pos.shape[0]
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    S = ct.c_double()
    per = np.zeros(R, np.float64) if per_receiver else None
    rc = lib().sao_shadow_integral(_ptr(tri9), _ptr(tb), tri9.shape[0], _ptr(pos), R, _ptr(dirs),
                                   _ptr(ds), ds.shape[0] - 1, float(step_minutes), _ptr(w),
                                   int(bisect_iters), ct.byref(S), _ptr(per),
                                   nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"sao_shadow_integral failed: {rc}")
    return (S.value, per) if per_receiver else S.value


def accumulate(tri9, tri_building, pos, nrm, dirs, day_start, step_minutes,
               nthreads: int | None = None):
    """Oracle gross steps, gross minutes (gross x step length) and continuous steps."""
    bits = shadow_bits(tri9, tri_building, pos, nrm, dirs, nthreads)
    g, c = reduce(bits, day_start)
    return g, (g.astype(np.float64) * step_minutes).astype(np.float32), c, bits


# ------------------------------------------------------------------ analysis measures
def point_in_polygon(x, y, poly):
    """Even-odd rule for points (x, y) (FP64 arrays) against a polygon [n, 2]: a point is
    inside when a ray from it toward +x crosses an odd number of edges."""
    poly = np.asarray(poly, dtype=np.float64).reshape(-1, 2)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    inside = np.zeros(np.broadcast(x, y).shape, dtype=bool)
    n = poly.shape[0]
    for i in range(n):
        ax, ay = poly[i]
        bx, by = poly[(i + 1) % n]
        crosses = (ay > y) != (by > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (y - ay) / (by - ay)
            xc = ax + t * (bx - ax)
        inside ^= crosses & (x < xc)
    return inside


def shadow_area(grid, steps, total_steps, poly):
    """Shadow area over a polygonal region (Sec. 7.2): the sum over the grid cells whose
    centre lies in the polygon of (steps / total_steps) x dx^2.  grid = (x0, y0, dx, nx, ny);
    the centres are the receivers' FP32 centres."""
    x0, y0, dx, nx, ny = grid
    ix = np.arange(nx, dtype=np.float32)
    iy = np.arange(ny, dtype=np.float32)
    cx = np.float32(x0) + (ix + np.float32(0.5)) * np.float32(dx)
    cy = np.float32(y0) + (iy + np.float32(0.5)) * np.float32(dx)
    X, Y = np.meshgrid(cx.astype(np.float64), cy.astype(np.float64))
    inside = point_in_polygon(X, Y, poly).ravel()
    frac = np.asarray(steps, dtype=np.float64).ravel() / float(total_steps)
    return float(frac[inside].sum()) * float(np.float32(dx)) ** 2


def shadow_score(areas, weights):
    """Shadow score (Sec. 7.2): the sum over intervals of weight x shadow area."""
    return float(np.dot(np.asarray(weights, np.float64), np.asarray(areas, np.float64)))


def building_steps(tri9, tri_building, pos, nrm, dirs, day_start, n_buildings, eps=1e-4,
                   nthreads: int | None = None):
    """Building contribution counts (Sec. 7.2) over the given receivers and all steps:
    (casting [B], nearest [B], unstable [B], unstable_any) as int64 -- pairs whose ray meets
    each building, pairs whose nearest hit is on it, pairs where meeting it flips under a
    +-eps rotation along the sun arc, and pairs where any building flips."""
    t9 = _f32(tri9).reshape(-1, 9)
    tb = _i32(tri_building).reshape(-1)
    p = _f32(pos).reshape(-1, 3)
    n = None if nrm is None else _f32(nrm).reshape(-1, 3)
    d = _f32(dirs).reshape(-1, 3)
    ds = _i32(day_start).reshape(-1)
    out = [np.zeros(int(n_buildings), np.int64) for _ in range(3)]
    anyc = np.zeros(1, np.int64)
    rc = lib().sao_building_steps(_ptr(t9), _ptr(tb), t9.shape[0], _ptr(p), _ptr(n), p.shape[0],
                                  _ptr(d), _ptr(ds), ds.shape[0] - 1, float(eps), int(n_buildings),
                                  _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(anyc),
                                  nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"sao_building_steps failed ({rc})")
    return out[0], out[1], out[2], int(anyc[0])


# ------------------------------------------------------------- endpoint-interpolated sun
def sun_interpolate(dirs, day_start, block_len: int = 0):
    """The paper's short-interval sun (Sec. 3.2, Sec. 4): inside each block of
    `block_partition`, only the first and last directions d_1, d_n are kept and the steps
    between are rebuilt from them, the sun moving at a constant angular rate along the great
    circle through d_1 and d_n: step i (i' = i - 1 = 0 .. n-1) is d_1 rotated toward d_n by
    i' theta / (n - 1), theta the angle between them.  (This is what the tangent law of
    Sec. 4 draws on a shadow plane orthogonal to d_1; the denominator n - 1 makes the last
    step land on d_n.)  Blocks of one or two steps, and the first and last step of every
    block, are unchanged.  Returns float32 [S, 3] (FP64 arithmetic, rounded once)."""
    d = np.asarray(dirs, np.float32).reshape(-1, 3).astype(np.float64)
    out = d.copy()
    j0, K = block_partition(day_start, block_len)
    for a, n in zip(j0.tolist(), K.tolist()):
        if n <= 2:
            continue
        d1 = d[a] / np.linalg.norm(d[a])
        dn = d[a + n - 1] / np.linalg.norm(d[a + n - 1])
        theta = float(np.arctan2(np.linalg.norm(np.cross(d1, dn)), np.dot(d1, dn)))
        tau = np.arange(1, n - 1, dtype=np.float64) / (n - 1)
        if theta < 1e-12:
            mid = np.repeat(d1[None, :], n - 2, axis=0)
        else:
            s = np.sin(theta)
            mid = (np.sin((1.0 - tau) * theta) / s)[:, None] * d1[None, :] + \
                  (np.sin(tau * theta) / s)[:, None] * dn[None, :]
        out[a + 1:a + n - 1] = mid
    return out.astype(np.float32)


# ------------------------------------------------------------- direction bins and graph
def direction_bins(dirs, bin_deg: float = 5.0):
    """Sec. 6 direction bins: the hemisphere cut into quads bounded by bin_deg in both
    angles -- elevation bands [k b, (k+1) b) above the horizon and azimuth sectors
    [m b, (m+1) b), azimuth measured from +y toward +x.  (elev_bin, az_bin) int64 [S]."""
    d = np.asarray(dirs, np.float32).reshape(-1, 3).astype(np.float64)
    n = np.linalg.norm(d, axis=1)
    el = np.degrees(np.arcsin(np.clip(d[:, 2] / n, -1.0, 1.0)))
    az = np.degrees(np.arctan2(d[:, 0], d[:, 1]))
    return np.floor(el / bin_deg).astype(np.int64), np.floor(az / bin_deg).astype(np.int64)


def direction_graph(dirs, day_start, block_len: int = 0, bin_deg: float = 5.0):
    """Sec. 6 direction graph over the blocks of `block_partition`: a block (an interval of
    the day) is the pair (bin of its first direction, bin of its last direction); blocks
    with the same pair and the same number of steps are one edge, numbered in order of
    first appearance.  The edge's map is computed once, from one of its blocks: the middle
    one in time order (element (m - 1) // 2 of its m blocks), so that the sun of the map
    lies inside the spread of the intervals it stands for.  Returns (edge [n_blocks],
    rep [E] = the block each edge's map is computed from, weight [E] = how many blocks the
    edge stands for)."""
    j0, K = block_partition(day_start, block_len)
    eb, ab = direction_bins(dirs, bin_deg)
    ids, rep, weight = {}, [], []
    edge = np.zeros(len(j0), np.int64)
    for b, (a, k) in enumerate(zip(j0.tolist(), K.tolist())):
        key = (eb[a], ab[a], eb[a + k - 1], ab[a + k - 1], k)
        if key not in ids:
            ids[key] = len(rep)
            rep.append(b)
            weight.append(0)
        edge[b] = ids[key]
        weight[ids[key]] += 1
    for e in range(len(rep)):
        members = np.nonzero(edge == e)[0]
        rep[e] = int(members[(len(members) - 1) // 2])
    return edge, np.asarray(rep, np.int64), np.asarray(weight, np.int64)


def graph_bits(bits, dirs, day_start, block_len: int = 0, bin_deg: float = 5.0):
    """Per-step bits as the direction graph sees them: every block takes the bits its
    edge's map holds, i.e. those of the edge's chosen block (Sec. 6: one map per edge,
    reused for every interval on that edge).  Gross and continuous counts of the graph
    are `reduce` of this array: Eq. 1 sums the edge maps with their weights, and the
    continuous count stitches each day's path of edges in time order."""
    bits = np.asarray(bits)
    j0, K = block_partition(day_start, block_len)
    edge, rep, _ = direction_graph(dirs, day_start, block_len, bin_deg)
    out = np.empty_like(bits)
    for b, (a, k) in enumerate(zip(j0.tolist(), K.tolist())):
        r0 = int(j0[rep[edge[b]]])
        out[:, a:a + k] = bits[:, r0:r0 + k]
    return out

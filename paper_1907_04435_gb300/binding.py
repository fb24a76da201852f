"""Thin Python binding of libshadowaccrual (ctypes).

Functions carry the C names (see include/shadowaccrual.h) and only marshal arguments:
torch tensors become device pointers, the current torch stream becomes the cudaStream_t,
and a non-zero sa_status becomes an SAError.  Every step of the computation runs in the
library's CUDA kernels; there is no Python or CPU fallback.  If the library is missing it
is built with nvcc; if that fails, importing raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np
import torch

from . import build as _build

SA_SWEEP_TRACE, SA_SWEEP_RASTER, SA_ACCRUAL_TRACE, SA_ACCRUAL_SAM, SA_IAM = range(5)
SA_ACCUMULATE_INTO = 1
METHODS = {"sweep_trace": SA_SWEEP_TRACE, "sweep_raster": SA_SWEEP_RASTER,
           "accrual_trace": SA_ACCRUAL_TRACE, "accrual_sam": SA_ACCRUAL_SAM, "iam": SA_IAM}
STATUS = {0: "SA_OK", -1: "SA_ERR_INVALID_ARG", -2: "SA_ERR_CUDA", -3: "SA_ERR_OOM",
          -4: "SA_ERR_SUN_BELOW_HORIZON", -5: "SA_ERR_DEGENERATE", -6: "SA_ERR_TIMEOUT",
          -7: "SA_ERR_INTERNAL", -8: "SA_ERR_UNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class SAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def checked_requested() -> bool:
    """SA_CHECKED=1 in the environment selects the bounds-checked build of the library."""
    return os.environ.get("SA_CHECKED", "0") not in ("", "0")


def lib_path() -> str:
    return _build.LIB_CHECKED if checked_requested() else _build.LIB


def lib():
    """Load (building first if stale) the CUDA library and declare its signatures."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=checked_requested())
            L = ct.CDLL(path)
            P, i32, i64, f32 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_float
            PP = ct.POINTER(ct.c_void_p)
            L.sa_last_error.restype = ct.c_char_p
            L.sa_version.restype = i32
            L.sa_scene_from_mesh.argtypes = [P, i64, P, i64, P, i32, i32, P, PP]
            L.sa_scene_destroy.argtypes = [P]
            L.sa_scene_destroy.restype = None
            L.sa_scene_info.argtypes = [P, P, P, P, P]
            L.sa_sun_create.argtypes = [P, i32, P, i32, i32, P, PP]
            L.sa_sun_destroy.argtypes = [P]
            L.sa_sun_destroy.restype = None
            L.sa_sun_info.argtypes = [P, P, P, P]
            L.sa_receivers_grid.argtypes = [f32, f32, f32, i32, i32, PP]
            L.sa_receivers_points.argtypes = [P, P, i64, i32, P, PP]
            L.sa_receivers_destroy.argtypes = [P]
            L.sa_receivers_destroy.restype = None
            L.sa_receivers_count.argtypes = [P]
            L.sa_receivers_count.restype = i64
            L.sa_accumulate.argtypes = [P, P, P, f32, i32, i32, i32, P, P, P, P]
            L.sa_shadow_masks.argtypes = [P, P, P, i32, i32, P, P]
            L.sa_accumulate_grid_noalloc.argtypes = [P, P, P, f32, i32, P, P, P, P]
            L.sa_work_counters.argtypes = [P, P, P, i32, P, P]
            L.sa_scene_declare_closed.argtypes = [P, i32]
            L.sa_set_option.argtypes = [i32, i32]
            L.sa_batch_create.argtypes = [P, P, P, P, i32, i32, P, PP]
            L.sa_batch_destroy.argtypes = [P]
            L.sa_batch_destroy.restype = None
            L.sa_batch_output_count.argtypes = [P]
            L.sa_batch_output_count.restype = i64
            L.sa_batch_output_offset.argtypes = [P, i32, i32]
            L.sa_batch_output_offset.restype = i64
            L.sa_batch_work_items.argtypes = [P]
            L.sa_batch_work_items.restype = i32
            L.sa_batch_affected_items.argtypes = [P]
            L.sa_batch_affected_items.restype = i32
            L.sa_batch_run.argtypes = [P, P, P, P]
            L.sa_batch_tune.argtypes = [P, P, P, P]
            L.sa_batch_work_counters.argtypes = [P, P, P]
            L.sa_get_option.argtypes = [i32]
            L.sa_get_option.restype = i32
            L.sa_scene_from_footprints.argtypes = [P, P, i32, P, f32, i32, P, PP]
            L.sa_scene_set_heights.argtypes = [P, P, i32, P]
            L.sa_height_grad.argtypes = [P, P, P, f32, P, P, P, P]
            L.sa_kernel_times.argtypes = [P, P, i32]
            L.sa_shadow_area.argtypes = [P, P, i32, P, i32, P, P]
            L.sa_shadow_score.argtypes = [P, P, i32, P, P, P, i32, P, P]
            L.sa_block_partition.argtypes = [P, i32, i32, P, P, P]
            L.sa_scratch_stats.argtypes = [P]
            L.sa_checked_build.restype = i32
            L.sa_check_status.argtypes = [P, P, P]
            L.sa_building_contribution.argtypes = [P, P, P, P, i32, P, P, P, P]
            L.sa_sun_interpolate.argtypes = [P, i32, P, i32, i32, P]
            L.sa_direction_graph.argtypes = [P, i32, P, i32, i32, f32, P, P, P, P, P]
            L.sa_accumulate_graph.argtypes = [P, P, P, i32, i32, f32, f32, P, P, P, P, P]
            for name in ("sa_scene_from_mesh", "sa_scene_info", "sa_sun_create", "sa_sun_info",
                         "sa_receivers_grid", "sa_receivers_points", "sa_accumulate",
                         "sa_shadow_masks", "sa_accumulate_grid_noalloc", "sa_work_counters",
                         "sa_scene_from_footprints", "sa_scene_set_heights", "sa_height_grad",
                         "sa_scene_declare_closed", "sa_set_option", "sa_batch_create",
                         "sa_batch_run", "sa_batch_tune", "sa_batch_work_counters",
                         "sa_kernel_times", "sa_shadow_area", "sa_shadow_score",
                         "sa_block_partition", "sa_scratch_stats", "sa_check_status",
                         "sa_building_contribution",
                         "sa_sun_interpolate", "sa_direction_graph", "sa_accumulate_graph"):
                getattr(L, name).restype = ct.c_int
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise SAError(status, lib().sa_last_error().decode(errors="replace"))


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _host_f32(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float32)


def _host_i32(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ct.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ct.c_void_p)


# ------------------------------------------------------------------------------ handles
class Scene:
    """sa_scene: device copy of the mesh plus its linear BVH."""

    def __init__(self, verts, tris, tri_building=None, n_buildings=None, stream=None,
                 closed: bool = False):
        v, t = _host_f32(verts).reshape(-1, 3), _host_i32(tris).reshape(-1, 3)
        b = None if tri_building is None else _host_i32(tri_building).reshape(-1)
        nb = int(n_buildings if n_buildings is not None else (int(b.max()) + 1 if b is not None and b.size else 1))
        h = ct.c_void_p()
        _check(lib().sa_scene_from_mesh(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(b), nb, 0,
                                        ct.c_void_p(_stream(stream)), ct.byref(h)))
        self.handle = h
        self.n_buildings = nb
        if closed:
            _check(lib().sa_scene_declare_closed(h, 1))

    @classmethod
    def from_footprints(cls, footprints, heights, band_height: float = 0.0, stream=None):
        """Extruded convex CCW footprints (list of [v, 2] arrays) with heights [B]."""
        xy = np.ascontiguousarray(np.concatenate([np.asarray(f, np.float32).reshape(-1, 2)
                                                  for f in footprints]) if len(footprints)
                                  else np.zeros((0, 2), np.float32), dtype=np.float32)
        off = np.zeros(len(footprints) + 1, np.int32)
        off[1:] = np.cumsum([len(f) for f in footprints])
        hs = _host_f32(heights).reshape(-1)
        h = ct.c_void_p()
        _check(lib().sa_scene_from_footprints(_ptr(xy), _ptr(off), len(footprints), _ptr(hs),
                                              float(band_height), 0, ct.c_void_p(_stream(stream)),
                                              ct.byref(h)))
        obj = cls.__new__(cls)
        obj.handle = h
        obj.n_buildings = len(footprints)
        return obj

    def set_heights(self, heights, stream=None):
        """New heights (host array or CUDA tensor [B]); rebuilds mesh and BVH."""
        if isinstance(heights, torch.Tensor) and heights.is_cuda:
            hs = heights.detach().float().contiguous()
            _check(lib().sa_scene_set_heights(self.handle, _ptr(hs), 1, ct.c_void_p(_stream(stream))))
        else:
            hs = _host_f32(heights).reshape(-1)
            _check(lib().sa_scene_set_heights(self.handle, _ptr(hs), 0, ct.c_void_p(_stream(stream))))

    def info(self):
        nt, nn, nb, mz = ct.c_int64(), ct.c_int64(), ct.c_int32(), ct.c_float()
        _check(lib().sa_scene_info(self.handle, ct.byref(nt), ct.byref(nn), ct.byref(nb), ct.byref(mz)))
        return {"n_tris": nt.value, "n_nodes": nn.value, "n_buildings": nb.value, "min_z": mz.value}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sa_scene_destroy(h)
            self.handle = None


class Sun:
    """sa_sun: validated, block-partitioned sun-direction table."""

    def __init__(self, dirs, day_start, block_len: int = 0, stream=None):
        d = _host_f32(dirs).reshape(-1, 3)
        ds = _host_i32(day_start).reshape(-1)
        h = ct.c_void_p()
        _check(lib().sa_sun_create(_ptr(d), d.shape[0], _ptr(ds), ds.shape[0] - 1, int(block_len),
                                   ct.c_void_p(_stream(stream)), ct.byref(h)))
        self.handle = h
        S, D, nb = ct.c_int32(), ct.c_int32(), ct.c_int32()
        _check(lib().sa_sun_info(h, ct.byref(S), ct.byref(D), ct.byref(nb)))
        self.S, self.D, self.n_blocks = S.value, D.value, nb.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sa_sun_destroy(h)
            self.handle = None


def sun_interpolate(dirs, day_start, block_len: int = 0) -> np.ndarray:
    """The paper's short-interval sun (Sec. 3.2, Sec. 4): float32 [S, 3] in which each
    block keeps its first and last directions and the steps between follow the great
    circle through them at a constant angular rate.  Build a `Sun` from it with the same
    block_len to run a method in the paper's mode."""
    d = _host_f32(dirs).reshape(-1, 3)
    ds = _host_i32(day_start).reshape(-1)
    out = np.empty_like(d)
    _check(lib().sa_sun_interpolate(_ptr(d), d.shape[0], _ptr(ds), ds.shape[0] - 1, int(block_len), _ptr(out)))
    return out


class Receivers:
    """sa_receivers: a ground grid (no per-cell storage) or Morton-sorted points."""

    def __init__(self, handle, R, grid=None):
        self.handle = handle
        self.R = int(R)
        self.grid = grid

    @classmethod
    def ground_grid(cls, x0, y0, dx, nx, ny):
        h = ct.c_void_p()
        _check(lib().sa_receivers_grid(float(x0), float(y0), float(dx), int(nx), int(ny), ct.byref(h)))
        return cls(h, int(nx) * int(ny), grid=(x0, y0, dx, nx, ny))

    @classmethod
    def points(cls, pos, normal=None, stream=None):
        if isinstance(pos, torch.Tensor) and pos.is_cuda:
            p = pos.detach().float().contiguous()
            n = None if normal is None else normal.detach().float().contiguous()
            dev = 1
        else:
            p = _host_f32(pos).reshape(-1, 3)
            n = None if normal is None else _host_f32(normal).reshape(-1, 3)
            dev = 0
        h = ct.c_void_p()
        _check(lib().sa_receivers_points(_ptr(p), _ptr(n), p.shape[0], dev,
                                         ct.c_void_p(_stream(stream)), ct.byref(h)))
        return cls(h, p.shape[0])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sa_receivers_destroy(h)
            self.handle = None


# --------------------------------------------------------------------------- the calls
def sa_accumulate(scene: Scene, recv: Receivers, sun: Sun, step_minutes: float, method,
                  iam_levels: int = 0, accumulate_into: bool = False, gross=None, minutes=None,
                  continuous=None, want_minutes=True, want_continuous=True, stream=None):
    """Returns (gross_steps int32, gross_minutes float32 | None, continuous int32 | None) on
    the current CUDA device; pass preallocated tensors to reuse or to accumulate into."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    dev = torch.device("cuda", torch.cuda.current_device())
    R = recv.R
    if gross is None:
        gross = torch.zeros(R, dtype=torch.int32, device=dev)
    if minutes is None and want_minutes:
        minutes = torch.empty(R, dtype=torch.float32, device=dev)
    if continuous is None and want_continuous:
        continuous = torch.zeros(R, dtype=torch.int32, device=dev)
    for t, dt in ((gross, torch.int32), (minutes, torch.float32), (continuous, torch.int32)):
        if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() != R):
            raise ValueError("output tensors must be contiguous CUDA tensors of R elements")
    _check(lib().sa_accumulate(scene.handle, recv.handle, sun.handle, float(step_minutes), m,
                               int(iam_levels), SA_ACCUMULATE_INTO if accumulate_into else 0,
                               _ptr(gross), _ptr(minutes), _ptr(continuous),
                               ct.c_void_p(_stream(stream))))
    return gross, minutes, continuous


def direction_graph(dirs, day_start, block_len: int = 0, bin_deg: float = 5.0):
    """The direction graph of a sun table (Sec. 6): (edge of each block, the block each
    edge's map is computed from -- its middle block --, weight of each edge) as int32
    arrays.  Host only."""
    d = _host_f32(dirs).reshape(-1, 3)
    ds = _host_i32(day_start).reshape(-1)
    nb, ne = ct.c_int32(), ct.c_int32()
    args = (_ptr(d), d.shape[0], _ptr(ds), ds.shape[0] - 1, int(block_len), float(bin_deg))
    _check(lib().sa_direction_graph(*args, ct.byref(nb), ct.byref(ne), None, None, None))
    edge = np.zeros(nb.value, np.int32)
    first = np.zeros(ne.value, np.int32)
    weight = np.zeros(ne.value, np.int32)
    _check(lib().sa_direction_graph(*args, ct.byref(nb), ct.byref(ne), _ptr(edge), _ptr(first), _ptr(weight)))
    return edge, first, weight


def sa_accumulate_graph(scene: Scene, recv: Receivers, sun: Sun, step_minutes: float, method,
                        bin_deg: float = 5.0, iam_levels: int = 0, stream=None):
    """Accumulation through the direction graph (Sec. 6, approximate): one map per edge,
    reused for every block of the edge.  Returns (gross_steps int32, gross_minutes float32,
    continuous int32, number of maps computed)."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    dev = torch.device("cuda", torch.cuda.current_device())
    R = recv.R
    gross = torch.zeros(R, dtype=torch.int32, device=dev)
    minutes = torch.zeros(R, dtype=torch.float32, device=dev)
    continuous = torch.zeros(R, dtype=torch.int32, device=dev)
    ne = ct.c_int32()
    _check(lib().sa_accumulate_graph(scene.handle, recv.handle, sun.handle, m, int(iam_levels), float(bin_deg),
                                     float(step_minutes), _ptr(gross), _ptr(minutes), _ptr(continuous),
                                     ct.byref(ne), ct.c_void_p(_stream(stream))))
    return gross, minutes, continuous, ne.value


def sa_accumulate_grid_noalloc(scene: Scene, grid: Receivers, sun: Sun, step_minutes: float,
                               gross, minutes=None, continuous=None, accumulate_into=False,
                               stream=None):
    """The ground accrual raster with no device allocation: the caller passes every output
    tensor (already allocated); the library's scratch is a fixed array compiled into it."""
    _check(lib().sa_accumulate_grid_noalloc(scene.handle, grid.handle, sun.handle,
                                            float(step_minutes),
                                            SA_ACCUMULATE_INTO if accumulate_into else 0,
                                            _ptr(gross), _ptr(minutes), _ptr(continuous),
                                            ct.c_void_p(_stream(stream))))
    return gross, minutes, continuous


def sa_work_counters(scene: Scene, recv: Receivers, sun: Sun, method, stream=None):
    """Work counters of one accumulation, as four Python ints: box and triangle tests of
    the trace methods; work units, enumerated cells, cell set-ups and cell-step tests of
    the raster ones; pair set-ups and step tests of the light-space map of points (see
    sa_work_counters in the C header)."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    c = torch.zeros(4, dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib().sa_work_counters(scene.handle, recv.handle, sun.handle, m, _ptr(c),
                                  ct.c_void_p(_stream(stream))))
    return [int(x) for x in c.cpu().tolist()]


def sa_checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(lib().sa_checked_build())


def sa_check_status():
    """Synchronises the device and returns the first out-of-range index the checked build
    recorded since the last call, as (site, index, bound), or None if there was none
    (always None for the plain build)."""
    site, idx, bound = ct.c_int32(), ct.c_int64(), ct.c_int64()
    st = lib().sa_check_status(ct.byref(site), ct.byref(idx), ct.byref(bound))
    if st == 0:
        return None
    if st != -7:
        _check(st)
    return site.value, idx.value, bound.value


def sa_scratch_stats():
    """The library's scratch-memory statistics: a dict with the allocations made since
    load and their bytes, and the current device pool's reserved bytes and high-water mark
    of bytes in use."""
    st = (ct.c_uint64 * 4)()
    _check(lib().sa_scratch_stats(st))
    return {"allocations": int(st[0]), "bytes": int(st[1]), "pool_reserved": int(st[2]),
            "pool_used_high": int(st[3])}


SA_OPT_SWEEP_TRAVERSAL, SA_OPT_ACCRUAL_TRAVERSAL, SA_OPT_RASTER_RUN = 1, 2, 3
SA_OPT_KERNEL_TIMING = 4
SA_OPT_POINT_RUN = 5
SA_OPT_BATCH_TILE_SKIP = 6
TRAVERSAL = {"auto": 0, "packet": 1, "lane": 2}
KERNEL_CLASSES = ("raster", "sam_points", "accrual", "sweep", "iam", "graph", "raster_bin", "contrib")


def sa_set_option(key: int, value: int):
    _check(lib().sa_set_option(int(key), int(value)))


def sa_get_option(key: int) -> int:
    return int(lib().sa_get_option(int(key)))


def sa_kernel_times():
    """Launches timed since the last collection (SA_OPT_KERNEL_TIMING on): a dict from
    kernel class to (total milliseconds, launches)."""
    n = len(KERNEL_CLASSES)
    ms = (ct.c_double * n)()
    cnt = (ct.c_int64 * n)()
    _check(lib().sa_kernel_times(ms, cnt, n))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def sa_height_grad(scene: Scene, grid: Receivers, sun: Sun, step_minutes: float, weights=None,
                   stream=None):
    """(dS/dh float32 [B], S float64 scalar tensor) on the current device."""
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.empty(scene.n_buildings, dtype=torch.float32, device=dev)
    S = torch.empty(1, dtype=torch.float64, device=dev)
    w = None if weights is None else torch.as_tensor(weights, dtype=torch.float32, device=dev).contiguous()
    _check(lib().sa_height_grad(scene.handle, grid.handle, sun.handle, float(step_minutes), _ptr(w),
                                _ptr(g), _ptr(S), ct.c_void_p(_stream(stream))))
    return g, S[0]


class _Variants(ct.Structure):
    _fields_ = [("n_variants", ct.c_int32), ("tower_tris", ct.c_void_p), ("tower_off", ct.c_void_p),
                ("removed_ids", ct.c_void_p), ("removed_off", ct.c_void_p), ("regions", ct.c_void_p)]


class Batch:
    """sa_batch: base scene + variants (towers, removed buildings, regions) x intervals."""

    def __init__(self, scene: Scene, grid: Receivers, tower_tris, removed, regions, suns,
                 with_impact: bool = True, stream=None):
        V = len(tower_tris)
        tow = np.ascontiguousarray(np.concatenate([np.asarray(t, np.float32).reshape(-1, 9)
                                                   for t in tower_tris]) if V else
                                   np.zeros((0, 9), np.float32), dtype=np.float32)
        toff = np.zeros(V + 1, np.int32)
        toff[1:] = np.cumsum([np.asarray(t).reshape(-1, 9).shape[0] for t in tower_tris])
        rem = np.ascontiguousarray(np.concatenate([np.asarray(r, np.int32) for r in removed])
                                   if V else np.zeros(0, np.int32), dtype=np.int32)
        roff = np.zeros(V + 1, np.int32)
        roff[1:] = np.cumsum([len(r) for r in removed])
        reg = np.ascontiguousarray(regions, dtype=np.int32).reshape(-1, 4)
        self._keep = (tow, toff, rem, roff, reg, scene, grid, list(suns))
        desc = _Variants(V, tow.ctypes.data, toff.ctypes.data, rem.ctypes.data, roff.ctypes.data,
                         reg.ctypes.data)
        arr = (ct.c_void_p * max(1, len(suns)))(*[s.handle.value for s in suns])
        h = ct.c_void_p()
        _check(lib().sa_batch_create(scene.handle, grid.handle, ct.byref(desc), arr, len(suns),
                                     1 if with_impact else 0, ct.c_void_p(_stream(stream)),
                                     ct.byref(h)))
        self.handle = h
        self.V, self.I = V, len(suns)
        self.n_out = int(lib().sa_batch_output_count(h))
        self.n_items = int(lib().sa_batch_work_items(h))
        self.n_affected = int(lib().sa_batch_affected_items(h))

    def offset(self, interval: int, variant: int) -> int:
        return int(lib().sa_batch_output_offset(self.handle, interval, variant))

    def run(self, counts=None, impact=None, want_impact=True, stream=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        if counts is None:
            counts = torch.empty(max(1, self.n_out), dtype=torch.int32, device=dev)
        if impact is None and want_impact:
            impact = torch.empty(max(1, self.n_out), dtype=torch.int32, device=dev)
        _check(lib().sa_batch_run(self.handle, _ptr(counts), _ptr(impact), ct.c_void_p(_stream(stream))))
        return counts, impact

    def tune(self, stream=None):
        c, r = ct.c_int32(), ct.c_int32()
        _check(lib().sa_batch_tune(self.handle, ct.byref(c), ct.byref(r), ct.c_void_p(_stream(stream))))
        return c.value, r.value

    def work_counters(self, stream=None):
        c = torch.zeros(4, dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
        _check(lib().sa_batch_work_counters(self.handle, _ptr(c), ct.c_void_p(_stream(stream))))
        return [int(x) for x in c.cpu().tolist()]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sa_batch_destroy(h)
            self.handle = None


def sa_shadow_masks(scene: Scene, recv: Receivers, sun: Sun, method, iam_levels: int = 0,
                    masks=None, stream=None):
    """uint64 masks [n_blocks, R] as an int64 tensor (bit k = step k of the block)."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    if masks is None:
        masks = torch.empty((sun.n_blocks, recv.R), dtype=torch.int64,
                            device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib().sa_shadow_masks(scene.handle, recv.handle, sun.handle, m, int(iam_levels),
                                 _ptr(masks), ct.c_void_p(_stream(stream))))
    return masks


def block_partition(day_start, block_len: int = 0):
    """The library's block partition of a sun table's days (sa_block_partition, host
    only): (j0, K) int32 arrays, each block's first step and length; block b is mask
    block b of sa_shadow_masks."""
    ds = _host_i32(day_start).reshape(-1)
    nb = ct.c_int32()
    _check(lib().sa_block_partition(_ptr(ds), ds.shape[0] - 1, int(block_len), ct.byref(nb), None, None))
    j0 = np.zeros(nb.value, np.int32)
    K = np.zeros(nb.value, np.int32)
    _check(lib().sa_block_partition(_ptr(ds), ds.shape[0] - 1, int(block_len), ct.byref(nb),
                                    _ptr(j0), _ptr(K)))
    return j0, K


def sa_shadow_area(grid: Receivers, steps, total_steps: int, polygon, stream=None) -> float:
    """Shadow area (m^2) over a polygon [n, 2] of a ground grid, from per-cell step counts
    (an int32 CUDA tensor in output order) out of total_steps (Sec. 7.2)."""
    if grid.grid is None:
        raise SAError(-1, "sa_shadow_area: receivers must be a ground grid")
    st = steps.detach().to(torch.int32).contiguous()
    poly = _host_f32(polygon).reshape(-1, 2)
    out = ct.c_double()
    _check(lib().sa_shadow_area(grid.handle, _ptr(st), int(total_steps), _ptr(poly), poly.shape[0],
                                ct.c_void_p(_stream(stream)), ct.byref(out)))
    return float(out.value)


def sa_building_contribution(scene: Scene, grid: Receivers, sun: Sun, polygon, stream=None):
    """Per-building shadow over a polygon of a ground grid (Sec. 7.2), in m^2 over the sun
    table's interval: (casting, nearest, stats).  casting[b] is the area building b
    shadows on its own; nearest[b] the area where b is the nearest caster.  stats[0]
    counts cell-steps that met more than 64 buildings (the call then raises),
    stats[1] shadowed cell-steps whose ray grazed past every triangle; sum(nearest) plus
    stats[1] x dx^2 / S is the region's gross shadow area."""
    if grid.grid is None:
        raise SAError(-1, "sa_building_contribution: receivers must be a ground grid")
    poly = _host_f32(polygon).reshape(-1, 2)
    nb = max(int(scene.n_buildings), 1)
    casting = np.zeros(nb, np.float64)
    nearest = np.zeros(nb, np.float64)
    stats = np.zeros(2, np.int64)
    _check(lib().sa_building_contribution(scene.handle, grid.handle, sun.handle, _ptr(poly), poly.shape[0],
                                          ct.c_void_p(_stream(stream)), casting.ctypes.data,
                                          nearest.ctypes.data, stats.ctypes.data))
    n = int(scene.n_buildings)
    return casting[:n], nearest[:n], (int(stats[0]), int(stats[1]))


def sa_shadow_score(grid: Receivers, steps, total_steps, weights, polygon, stream=None) -> float:
    """Shadow score (m^2) over a polygon of a ground grid and several intervals (Sec. 7.2):
    steps is an int32 CUDA tensor [n_intervals, R] (or a list of [R] tensors, stacked on the
    device) of per-cell counts; total_steps and weights (in [-1, 1]) have one entry per
    interval."""
    if grid.grid is None:
        raise SAError(-1, "sa_shadow_score: receivers must be a ground grid")
    if isinstance(steps, (list, tuple)):
        steps = torch.stack([t.detach().to(torch.int32) for t in steps])
    st = steps.detach().to(torch.int32).contiguous()
    n_t = st.shape[0] if st.dim() == 2 else 1
    tot = _host_i32(total_steps).reshape(-1)
    w = _host_f32(weights).reshape(-1)
    if tot.shape[0] != n_t or w.shape[0] != n_t:
        raise SAError(-1, "sa_shadow_score: one total and one weight per interval")
    poly = _host_f32(polygon).reshape(-1, 2)
    out = ct.c_double()
    _check(lib().sa_shadow_score(grid.handle, _ptr(st), n_t, _ptr(tot), _ptr(w), _ptr(poly),
                                 poly.shape[0], ct.c_void_p(_stream(stream)), ct.byref(out)))
    return float(out.value)

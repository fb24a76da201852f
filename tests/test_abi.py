"""C-ABI checks that need no GPU: the library builds, loads, exports every declared symbol,
and rejects bad arguments on the host before touching the device."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sa_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_1907_04435_gb300 import binding
    return binding.lib()


def test_library_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 14
    for n in sorted(names):
        assert hasattr(L, n), f"missing export {n}"


def test_version_and_empty_error(L):
    assert L.sa_version() >> 16 == 1
    assert isinstance(L.sa_last_error(), bytes)


def test_grid_receivers_need_no_device(L):
    from paper_1907_04435_gb300 import binding as B
    r = B.Receivers.ground_grid(0.0, 0.0, 1.0, 7, 5)
    assert L.sa_receivers_count(r.handle) == 35
    h = ct.c_void_p()
    assert L.sa_receivers_grid(0.0, 0.0, 0.0, 3, 3, ct.byref(h)) == -1       # dx = 0
    assert L.sa_receivers_grid(0.0, 0.0, 1.0, -1, 3, ct.byref(h)) == -1
    assert b"grid size" in L.sa_last_error()


def test_sun_validation_happens_on_the_host(L):
    from paper_1907_04435_gb300 import binding as B
    h = ct.c_void_p()
    bad = np.array([[0.6, 0.0, 0.8], [0.8, 0.0, -0.6]], np.float32)
    ds = np.array([0, 2], np.int32)
    assert L.sa_sun_create(B._ptr(bad), 2, B._ptr(ds), 1, 0, None, ct.byref(h)) == -4
    unnorm = np.array([[0.6, 0.0, 0.9]], np.float32)
    assert L.sa_sun_create(B._ptr(unnorm), 1, B._ptr(np.array([0, 1], np.int32)), 1, 0, None,
                           ct.byref(h)) == -1
    ok = np.array([[0.6, 0.0, 0.8]], np.float32)
    assert L.sa_sun_create(B._ptr(ok), 1, B._ptr(np.array([0, 2], np.int32)), 1, 0, None,
                           ct.byref(h)) == -1          # day_start[D] != S
    assert L.sa_sun_create(B._ptr(ok), 1, B._ptr(np.array([0, 1], np.int32)), 1, 65, None,
                           ct.byref(h)) == -1          # block_len > 64


def test_scene_argument_checks_happen_on_the_host(L):
    """Sizes and pointers are checked before any device work (the mesh's contents are
    checked on the device while its BVH is built: `test_gpu_parity.py`)."""
    from paper_1907_04435_gb300 import binding as B
    h = ct.c_void_p()
    v = np.zeros((3, 3), np.float32)
    t = np.array([[0, 1, 2]], np.int32)
    assert L.sa_scene_from_mesh(B._ptr(v), -1, B._ptr(t), 1, None, 1, 0, None, ct.byref(h)) == -1
    assert L.sa_scene_from_mesh(B._ptr(v), 3, B._ptr(t), -2, None, 1, 0, None, ct.byref(h)) == -1
    assert L.sa_scene_from_mesh(None, 3, B._ptr(t), 1, None, 1, 0, None, ct.byref(h)) == -1
    assert L.sa_scene_from_mesh(B._ptr(v), 3, None, 1, None, 1, 0, None, ct.byref(h)) == -1
    assert L.sa_scene_from_mesh(B._ptr(v), 3, B._ptr(t), 1, None, -1, 0, None, ct.byref(h)) == -1
    assert L.sa_scene_from_mesh(B._ptr(v), 3, B._ptr(t), (1 << 30) + 1, None, 1, 0, None, ct.byref(h)) == -1
    assert L.sa_scene_from_mesh(B._ptr(v), 3, B._ptr(t), 1, None, 1, 0, None, None) == -1
    assert not h.value


def test_block_partition_is_the_oracles():
    """sa_block_partition is host code: per day, ceil(n / K) blocks whose sizes differ by
    at most one, the longer first; the same blocks as the oracle's partition."""
    import oracle
    from paper_1907_04435_gb300 import binding as B
    assert B.block_partition([0, 481])[1].tolist() == [54, 54, 54, 54, 53, 53, 53, 53, 53]
    assert B.block_partition([0, 5, 5, 70], 64)[1].tolist() == [5, 33, 32]
    assert B.block_partition([0, 3], 1)[1].tolist() == [1, 1, 1]
    for ds, bl in (([0, 481], 0), ([0, 5, 5, 70], 64), ([0, 1000], 64), ([0, 241, 482, 483], 7),
                   ([0, 0], 0), (list(range(0, 92 * 481 + 1, 481)), 60)):
        j0, K = B.block_partition(ds, bl)
        oj, oK = oracle.block_partition(ds, bl)
        assert np.array_equal(j0, oj) and np.array_equal(K, oK), (ds[:4], bl)
        assert K.sum() == ds[-1] and (K <= (bl or 60)).all()
    with pytest.raises(B.SAError):
        B.block_partition([0, 10], 65)
    with pytest.raises(B.SAError):
        B.block_partition([1, 10], 0)
    with pytest.raises(B.SAError):
        B.block_partition([0, 10, 5], 0)


def test_options_and_kernel_timing_record_need_no_device(L):
    from paper_1907_04435_gb300 import binding as B
    for key, good, bad in ((B.SA_OPT_RASTER_RUN, 8, 33), (B.SA_OPT_KERNEL_TIMING, 1, 2),
                           (B.SA_OPT_ACCRUAL_TRAVERSAL, 0, 3), (B.SA_OPT_POINT_RUN, 4, 33)):
        old = B.sa_get_option(key)
        B.sa_set_option(key, good)
        assert B.sa_get_option(key) == good
        assert L.sa_set_option(key, bad) == -1
        B.sa_set_option(key, old)
    assert B.sa_get_option(99) == -1
    assert L.sa_kernel_times(None, None, -1) == -1
    # nothing launched: the record is empty
    t = B.sa_kernel_times()
    assert set(t) == set(B.KERNEL_CLASSES) and all(v == (0.0, 0) for v in t.values())


def test_interpolated_sun_matches_the_oracle_on_the_host():
    """sa_sun_interpolate is host code: its table equals the oracle's FP64 interpolation to
    FP32 rounding, keeps every block's ends bit for bit, and validates like sa_sun_create."""
    import oracle
    from paper_1907_04435_gb300 import binding as B
    from synth.sun import sun_table
    st = sun_table(40.7, [79, 172, 355], 9.0, 17.0, 1.0)
    for bl in (0, 17, 60, 64):
        got = B.sun_interpolate(st.dirs, st.day_start, bl)
        want = oracle.sun_interpolate(st.dirs, st.day_start, bl)
        assert np.abs(got.astype(np.float64) - want).max() <= 1.2e-7, bl
        j0, K = oracle.block_partition(st.day_start, bl)
        assert np.array_equal(got[j0], st.dirs[j0]) and np.array_equal(got[j0 + K - 1], st.dirs[j0 + K - 1])
    # in place
    d = st.dirs.copy()
    L = B.lib()
    assert L.sa_sun_interpolate(d.ctypes.data, d.shape[0], st.day_start.ctypes.data, st.D, 60, d.ctypes.data) == 0
    assert np.array_equal(d, B.sun_interpolate(st.dirs, st.day_start, 60))
    with pytest.raises(B.SAError):
        B.sun_interpolate(st.dirs * 2.0, st.day_start, 60)
    with pytest.raises(B.SAError):
        B.sun_interpolate(st.dirs, st.day_start, 65)


def test_direction_graph_matches_the_oracle_on_the_host():
    """sa_direction_graph is host code: the same edges, map blocks and weights as the
    oracle's graph, bit for bit, on a season of one-minute steps and on the Fig. 7 case."""
    import oracle
    from paper_1907_04435_gb300 import binding as B
    from synth.sun import sun_table
    st = sun_table(40.7, list(range(172, 264)), 9.0, 17.0, 1.0)
    for bl, bd in ((60, 5.0), (30, 2.5), (64, 10.0), (60, 1e-6)):
        e, f, w = B.direction_graph(st.dirs, st.day_start, bl, bd)
        oe, of, ow = oracle.direction_graph(st.dirs, st.day_start, bl, bd)
        assert np.array_equal(e, oe) and np.array_equal(f, of) and np.array_equal(w, ow), (bl, bd)
    e, f, w = B.direction_graph(st.dirs, st.day_start, 60, 5.0)
    assert len(f) < len(e) / 4 and w.sum() == len(e)
    with pytest.raises(B.SAError):
        B.direction_graph(st.dirs, st.day_start, 60, 0.0)
    with pytest.raises(B.SAError):
        B.direction_graph(st.dirs, st.day_start, 60, 91.0)


def test_binding_reaches_every_declared_entry_point():
    """Every call include/*.h declares has its argument types set in the binding and is
    used by it, so each is reachable from Python."""
    src = open(os.path.join(ROOT, "paper_1907_04435_gb300", "binding.py")).read()
    missing = [n for n in sorted(declared_symbols())
               if f"L.{n}" not in src and f"lib().{n}" not in src and f"_lib.{n}" not in src]
    assert not missing, missing


def test_checked_build_exports_the_same_calls_and_says_so():
    """The bounds-checked variant is built beside the plain library (nvcc cross-compiles
    here), exports every declared call and reports itself; the plain build reports no
    check and its status call needs no device."""
    from paper_1907_04435_gb300 import build as b
    path = b.build(checked=True)
    Lc = ct.CDLL(path)
    for n in sorted(declared_symbols()):
        assert hasattr(Lc, n), f"missing export {n}"
    assert Lc.sa_checked_build() == 1
    from paper_1907_04435_gb300 import binding as B
    Lp = B.lib()
    assert Lp.sa_checked_build() == 0
    site, idx, bound = ct.c_int32(7), ct.c_int64(7), ct.c_int64(7)
    assert Lp.sa_check_status(ct.byref(site), ct.byref(idx), ct.byref(bound)) == 0
    assert (site.value, idx.value, bound.value) == (0, 0, 0)

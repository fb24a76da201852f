"""Accumulation through the direction graph (Sec. 6) on the device against the FP64 oracle's
graph: the same edges, one map per edge from its middle block, Eq. 1 for gross and the
day paths stitched for continuous; bins small enough to keep every block apart give the
exact result bit for bit; and the error of 5 degree bins against the exact counts."""
import numpy as np
import pytest

import oracle
from parity import EPS_RAD, assert_counts_parity
from synth import configs

pytestmark = pytest.mark.gpu

DOYS = (165, 168, 172, 176, 180)


def _case(**kw):
    return configs.district_small(doys=DOYS, step=2.0, **kw)


def _handles(B, w):
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    return scene, sun, grid


_cache = {}


def _oracle_graph(w, pos, nrm, bin_deg, key=None):
    if key is not None and key in _cache:
        return _cache[key]
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    bits = oracle.shadow_bits(t9, tb, pos, nrm, w.sun.dirs)
    near = oracle.near_boundary(t9, tb, pos, nrm, w.sun.dirs, w.sun.day_start, bits, eps=EPS_RAD)
    gb = oracle.graph_bits(bits, w.sun.dirs, w.sun.day_start, 0, bin_deg)
    gn = oracle.graph_bits(near, w.sun.dirs, w.sun.day_start, 0, bin_deg)
    if key is not None:
        _cache[key] = (bits, gb, gn)
    return bits, gb, gn


@pytest.mark.parametrize("method", ["accrual_sam", "accrual_trace"])
def test_graph_ground_matches_the_oracle(cuda_lib, method):
    B = cuda_lib
    w = _case(n_facade=0)
    scene, sun, grid = _handles(B, w)
    gross, minutes, cont, n_edges = B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, method, 5.0)
    _, rep, weight = oracle.direction_graph(w.sun.dirs, w.sun.day_start, 0, 5.0)
    assert n_edges == len(rep) < sun.n_blocks and weight.sum() == sun.n_blocks
    _, gb, gn = _oracle_graph(w, w.ground.positions(), None, 5.0, key="ground")
    g = gross.cpu().numpy()
    assert_counts_parity(g, cont.cpu().numpy(), gb, gn, w.sun.day_start, f"graph {method}")
    assert np.array_equal(minutes.cpu().numpy(), g.astype(np.float32) * np.float32(w.sun.step_minutes))


def test_graph_facades_match_the_oracle(cuda_lib):
    B = cuda_lib
    w = _case()
    scene, sun, _ = _handles(B, w)
    pts = B.Receivers.points(w.facade_pos, w.facade_nrm)
    gross, _, cont, _ = B.sa_accumulate_graph(scene, pts, sun, w.sun.step_minutes, "accrual_sam", 5.0)
    _, gb, gn = _oracle_graph(w, w.facade_pos, w.facade_nrm, 5.0)
    assert_counts_parity(gross.cpu().numpy(), cont.cpu().numpy(), gb, gn, w.sun.day_start, "graph facades")


@pytest.mark.parametrize("method", ["accrual_sam", "sweep_raster", "iam"])
def test_tiny_bins_give_the_exact_counts(cuda_lib, method):
    B = cuda_lib
    w = _case(n_facade=0)
    scene, sun, grid = _handles(B, w)
    ge, _, ce = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, method)
    gg, _, cg, n_edges = B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, method, 1e-6)
    assert n_edges == sun.n_blocks
    assert np.array_equal(gg.cpu().numpy(), ge.cpu().numpy())
    assert np.array_equal(cg.cpu().numpy(), ce.cpu().numpy())


def test_graph_error_against_the_exact_counts(cuda_lib):
    """A week of consecutive days: 5 degree bins compute a fraction of the maps, and the
    device's gross error against the exact counts equals the oracle's up to the pairs near
    a shadow boundary."""
    B = cuda_lib
    w = configs.district_small(doys=tuple(range(172, 179)), step=2.0, n_facade=0)
    scene, sun, grid = _handles(B, w)
    ge, _, _ = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
    gg, _, _, n_edges = B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, "accrual_sam", 5.0)
    ge, gg = ge.cpu().numpy().astype(np.int64), gg.cpu().numpy().astype(np.int64)
    err = np.abs(gg - ge).sum() / ge.sum()
    bits, gb, gn = _oracle_graph(w, w.ground.positions(), None, 5.0)
    oe, _ = oracle.reduce(bits, w.sun.day_start)
    og, _ = oracle.reduce(gb, w.sun.day_start)
    err_o = np.abs(og.astype(np.int64) - oe).sum() / oe.sum()
    near = oracle.near_boundary(w.mesh.tri9(), w.mesh.tri_building, w.ground.positions(), None,
                                w.sun.dirs, w.sun.day_start, bits, eps=EPS_RAD)
    slack = (near.sum() + gn.sum()) / oe.sum()
    print(f"graph: {n_edges} maps for {sun.n_blocks} blocks, gross error {100 * err:.3f} % "
          f"(oracle {100 * err_o:.3f} %)")
    assert n_edges * 3 < sun.n_blocks
    assert err < 0.02 and abs(err - err_o) <= slack


def test_graph_rejects_bad_bins(cuda_lib):
    B = cuda_lib
    w = _case(n_facade=0)
    scene, sun, grid = _handles(B, w)
    for bd in (0.0, -1.0, 120.0, float("nan")):
        with pytest.raises(B.SAError):
            B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, "accrual_sam", bd)


def test_graph_degenerate_inputs(cuda_lib):
    """No receivers, a sun table with no steps, point receivers with a grid-only method,
    and one day (every block its own edge): the exact counts."""
    B = cuda_lib
    w = _case(n_facade=0)
    scene, sun, grid = _handles(B, w)
    empty_grid = B.Receivers.ground_grid(0.0, 0.0, 1.0, 0, 0)
    g, m, c, ne = B.sa_accumulate_graph(scene, empty_grid, sun, w.sun.step_minutes, "accrual_sam")
    assert g.numel() == 0 and ne == len(oracle.direction_graph(w.sun.dirs, w.sun.day_start)[1])
    no_steps = B.Sun(np.zeros((0, 3), np.float32), np.zeros(1, np.int32))
    g, m, c, ne = B.sa_accumulate_graph(scene, grid, no_steps, w.sun.step_minutes, "accrual_sam")
    assert ne == 0 and not g.any() and not c.any() and not m.any()
    pts = B.Receivers.points(np.array([[50.0, 50.0, 0.0]], np.float32))
    with pytest.raises(B.SAError):
        B.sa_accumulate_graph(scene, pts, sun, w.sun.step_minutes, "iam")
    one = configs.district_small(doys=(172,), step=2.0, n_facade=0)
    sc1, sun1, grid1 = _handles(B, one)
    ge, _, ce = B.sa_accumulate(sc1, grid1, sun1, one.sun.step_minutes, "accrual_sam")
    gg, _, cg, ne = B.sa_accumulate_graph(sc1, grid1, sun1, one.sun.step_minutes, "accrual_sam", 5.0)
    assert ne == sun1.n_blocks
    assert np.array_equal(gg.cpu().numpy(), ge.cpu().numpy()) and np.array_equal(cg.cpu().numpy(), ce.cpu().numpy())

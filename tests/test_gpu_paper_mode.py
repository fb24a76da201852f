"""The methods in the paper's short-interval mode (Sec. 3.2, Sec. 4): the sun table rebuilt
from each block's first and last direction (great-circle motion at a constant rate).
Parity against the FP64 oracle run on its own interpolation of the same table, and the
error of the linear-motion assumption measured against the exact table -- the question of
Table 1 asked of shadows instead of directions."""
import numpy as np
import pytest
import torch

import oracle
from parity import EPS_RAD, assert_counts_parity, block_sizes, unpack_masks, workload
from synth import configs

pytestmark = pytest.mark.gpu


def _setup(B, w, block_len=0):
    dirs = B.sun_interpolate(w.sun.dirs, w.sun.day_start, block_len)
    odirs = oracle.sun_interpolate(w.sun.dirs, w.sun.day_start, block_len)
    assert np.abs(dirs.astype(np.float64) - odirs).max() <= 1.2e-7
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(dirs, w.sun.day_start, block_len)
    return scene, sun, odirs


@pytest.mark.parametrize("method", ["accrual_sam", "accrual_trace", "sweep_raster"])
def test_paper_mode_ground_matches_the_oracle(cuda_lib, method):
    B = cuda_lib
    w = workload("district_small")
    g = w.ground
    scene, sun, odirs = _setup(B, w)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    gross, _, cont = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, method)
    t9, tb, pos = w.mesh.tri9(), w.mesh.tri_building, g.positions()
    bits = oracle.shadow_bits(t9, tb, pos, None, odirs)
    near = oracle.near_boundary(t9, tb, pos, None, odirs, w.sun.day_start, bits, eps=EPS_RAD)
    assert_counts_parity(gross.cpu().numpy(), cont.cpu().numpy(), bits, near, w.sun.day_start,
                         f"paper mode {method}")


def test_paper_mode_facades_match_the_oracle(cuda_lib):
    B = cuda_lib
    w = workload("district_small")
    scene, sun, odirs = _setup(B, w)
    pts = B.Receivers.points(w.facade_pos, w.facade_nrm)
    gross, _, cont = B.sa_accumulate(scene, pts, sun, w.sun.step_minutes, "accrual_sam")
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    bits = oracle.shadow_bits(t9, tb, w.facade_pos, w.facade_nrm, odirs)
    near = oracle.near_boundary(t9, tb, w.facade_pos, w.facade_nrm, odirs, w.sun.day_start, bits,
                                eps=EPS_RAD)
    assert_counts_parity(gross.cpu().numpy(), cont.cpu().numpy(), bits, near, w.sun.day_start,
                         "paper mode facades")


@pytest.mark.parametrize("doy", [172, 355])
def test_linear_motion_error_against_the_exact_table(cuda_lib, doy):
    """One-minute steps in hourly blocks: the paper-mode gross counts differ from the
    exact ones by well under 1 % of the shadow, and the device's error equals the oracle's
    up to the pairs near a shadow boundary under either table."""
    B = cuda_lib
    w = configs.district_small(step=1.0, doys=(doy,), n_facade=0)
    g = w.ground
    scene, sun_p, odirs = _setup(B, w)
    sun_e = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    ge, _, _ = B.sa_accumulate(scene, grid, sun_e, w.sun.step_minutes, "accrual_sam")
    gp, _, _ = B.sa_accumulate(scene, grid, sun_p, w.sun.step_minutes, "accrual_sam")
    ge, gp = ge.cpu().numpy().astype(np.int64), gp.cpu().numpy().astype(np.int64)
    err = np.abs(gp - ge).sum() / ge.sum()
    t9, tb, pos = w.mesh.tri9(), w.mesh.tri_building, g.positions()
    be = oracle.shadow_bits(t9, tb, pos, None, w.sun.dirs)
    bp = oracle.shadow_bits(t9, tb, pos, None, odirs)
    ne = oracle.near_boundary(t9, tb, pos, None, w.sun.dirs, w.sun.day_start, be, eps=EPS_RAD)
    np_ = oracle.near_boundary(t9, tb, pos, None, odirs, w.sun.day_start, bp, eps=EPS_RAD)
    oe, _ = oracle.reduce(be, w.sun.day_start)
    op, _ = oracle.reduce(bp, w.sun.day_start)
    err_o = np.abs(op.astype(np.int64) - oe).sum() / oe.sum()
    slack = (ne.sum() + np_.sum()) / oe.sum()
    print(f"doy {doy}: paper-mode gross error {100 * err:.3f} % (oracle {100 * err_o:.3f} %)")
    assert 0 < err < 0.01
    assert abs(err - err_o) <= slack
    torch.cuda.synchronize()


def test_paper_mode_iam_matches_its_restatement(cuda_lib):
    """The inverse accrual map (Sec. 5) on the interpolated table, held to the bar of its
    own parity test: every bit the FP64 supercover map sets for certain is set, none
    outside what it may set within 1 mm of a cell edge, a triangle edge or another source."""
    B = cuda_lib
    w = configs.district_small(dx=1.0, nx=240, ny=180, step=2.0, t0=10.0, t1=15.0)
    g = w.ground
    scene, sun, odirs = _setup(B, w)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    masks = B.sa_shadow_masks(scene, grid, sun, "iam", 3)
    torch.cuda.synchronize()
    gb = unpack_masks(masks, block_sizes(w.sun.day_start, 0))
    must, may = oracle.iam_bounds(w.mesh.tri9(), w.mesh.tri_building, (g.x0, g.y0, g.dx, g.nx, g.ny),
                                  odirs, w.sun.day_start, levels=3, eps_cell=1e-3, eps_src=1e-3,
                                  eps_t=1e-3)
    assert not ((must == 1) & (gb == 0)).any()
    assert not ((may == 0) & (gb == 1)).any()
    assert (may != must).mean() < 1e-3

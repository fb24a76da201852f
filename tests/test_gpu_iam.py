"""GPU inverse accrual map (Sec. 5) against its FP64 restatement and the paper's bar."""
import numpy as np
import pytest
import torch

import oracle
from synth import configs

from parity import block_sizes, unpack_masks

pytestmark = pytest.mark.gpu


def _case():
    return configs.district_small(dx=1.0, nx=240, ny=180, step=2.0, t0=10.0, t1=15.0)


def _gpu_iam(B, w, levels=3, block_len=0):
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    sun = B.Sun(w.sun.dirs, w.sun.day_start, block_len)
    masks = B.sa_shadow_masks(scene, grid, sun, "iam", levels)
    gross, _, cont = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "iam", levels)
    torch.cuda.synchronize()
    bits = unpack_masks(masks, block_sizes(w.sun.day_start, block_len))
    return bits, gross.cpu().numpy(), cont.cpu().numpy()


# Tolerances of the bar, in metres (see iam_bounds): the kernel's sources and shadow-line
# ends are FP32, so a line end may sit a few 1e-5 m from the FP64 one (coordinates of a few
# hundred metres carry FP32 steps of 3e-5 m, and a line end takes three roundings); a
# source ray may pass that close to a triangle's edge, or two sources lie that close in
# distance.  1 mm is ten times the worst of these.
EPS_M = 1e-3


@pytest.mark.parametrize("levels", [1, 3])
def test_iam_matches_its_fp64_restatement(cuda_lib, levels):
    """Every bit the FP64 supercover map sets for certain is set, and no bit outside what
    it may set: only cells a line reaches within 1 mm of their edge or corner, and lines
    of sources within 1 mm of a triangle edge or of another source, may differ."""
    B = cuda_lib
    w = _case()
    g = w.ground
    grid = (g.x0, g.y0, g.dx, g.nx, g.ny)
    must, may = oracle.iam_bounds(w.mesh.tri9(), w.mesh.tri_building, grid, w.sun.dirs,
                                  w.sun.day_start, levels=levels, eps_cell=EPS_M,
                                  eps_src=EPS_M, eps_t=EPS_M)
    gb, gross, cont = _gpu_iam(B, w, levels)
    missing = np.argwhere((must == 1) & (gb == 0))
    extra = np.argwhere((may == 0) & (gb == 1))
    assert missing.shape[0] == 0, f"{missing.shape[0]} certain bits unset, e.g. {missing[:5].tolist()}"
    assert extra.shape[0] == 0, f"{extra.shape[0]} bits set outside the bound, e.g. {extra[:5].tolist()}"
    # the band the bar leaves open is small (so that it can tell the line readings apart)
    assert (may != must).mean() < 1e-3
    assert must.sum() > 0.1 * must.size
    assert np.array_equal(gross, gb.sum(axis=1))


def test_iam_area_error_within_the_paper_bar(cuda_lib):
    """Sec. 8.2: with three source levels the shadow-area error stays below 1 % of the
    area on average (max 2.6 %), measured per hourly block against the exact result."""
    B = cuda_lib
    w = configs.district_small(dx=1.0, nx=300, ny=240, step=1.0, t0=9.0, t1=15.0)
    gb, _, _ = _gpu_iam(B, w, 3)
    exact = oracle.shadow_bits(w.mesh.tri9(), w.mesh.tri_building, w.ground.positions(), None,
                               w.sun.dirs)
    j0, K = oracle.block_partition(w.sun.day_start)
    errs = [abs(gb[:, a:a + k].sum() - exact[:, a:a + k].sum()) / (k * exact.shape[0])
            for a, k in zip(j0, K)]
    assert np.mean(errs) < 0.01 and max(errs) < 0.026, errs


def test_iam_rejects_bad_levels_and_points(cuda_lib):
    B = cuda_lib
    w = configs.boxes16()
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    with pytest.raises(B.SAError):
        B.sa_accumulate(scene, grid, sun, 1.0, "iam", 9)
    pts = B.Receivers.points(g.positions()[:4])
    with pytest.raises(B.SAError) as e:
        B.sa_accumulate(scene, pts, sun, 1.0, "iam", 3)
    assert e.value.status == -8

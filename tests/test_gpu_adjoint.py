"""GPU height gradient of a region's shadow-minutes: closed form, oracle finite differences,
footprint scenes and the autograd.Function."""
import numpy as np
import pytest
import torch

import oracle
from synth import city as C
from synth import configs
from synth.sun import sun_table

from test_oracle_adjoint import closed_form

pytestmark = pytest.mark.gpu


def _fp_scene(B, city, heights=None):
    return B.Scene.from_footprints(city.footprints, city.heights if heights is None else heights,
                                   city.band_height)


def _grid(B, g):
    return B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)


def test_footprint_scene_equals_the_host_extruded_mesh(cuda_lib):
    B = cuda_lib
    w = configs.district_small()
    a = _fp_scene(B, w.city)
    b = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    assert a.info()["n_tris"] == w.mesh.T
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = _grid(B, w.ground)
    for method in ("accrual_sam", "sweep_trace"):
        assert torch.equal(B.sa_shadow_masks(a, grid, sun, method),
                           B.sa_shadow_masks(b, grid, sun, method))


def test_set_heights_rebuilds_the_scene(cuda_lib):
    B = cuda_lib
    w = configs.district_small(n_facade=0)
    h2 = w.city.heights * np.float32(1.3)
    bands = C.band_counts(w.city)
    mesh2 = C.extrude(w.city, heights=h2, bands=bands)
    a = _fp_scene(B, w.city)
    a.set_heights(torch.as_tensor(h2, device="cuda"))
    b = B.Scene(mesh2.verts, mesh2.tris, mesh2.tri_building, w.city.B)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = _grid(B, w.ground)
    assert torch.equal(B.sa_shadow_masks(a, grid, sun, "accrual_sam"),
                       B.sa_shadow_masks(b, grid, sun, "accrual_sam"))


def test_single_box_gradient_matches_the_closed_form(cuda_lib):
    B = cuda_lib
    fp = C.box_footprint(0.0, 0.0, 30.0, 20.0)
    h = 40.0
    city = C.City([fp], np.array([h], np.float32))
    st = sun_table(40.7, [80], 9.0, 17.0, 4.0)
    g = C.GroundGrid(-80.0, -80.0, 1.0, 190, 120)
    S_cf, G_cf = closed_form(fp.astype(np.float32).astype(np.float64), h, g.positions(), st.dirs,
                             st.step_minutes)
    scene = _fp_scene(B, city)
    grad, S = B.sa_height_grad(scene, _grid(B, g), B.Sun(st.dirs, st.day_start), st.step_minutes)
    assert abs(float(S) - S_cf) <= 1e-6 * S_cf
    assert abs(float(grad[0]) - G_cf) <= 1e-4 * abs(G_cf), (float(grad[0]), G_cf)


def flips_per_day(bits, day_start):
    """int [R, D]: status changes between consecutive steps of each day."""
    out = np.zeros((bits.shape[0], len(day_start) - 1), np.int64)
    for k in range(len(day_start) - 1):
        a, b = int(day_start[k]), int(day_start[k + 1])
        out[:, k] = np.abs(np.diff(bits[:, a:b].astype(np.int64), axis=1)).sum(axis=1)
    return out


def test_park_gradient_matches_oracle_finite_differences(cuda_lib):
    """Central differences (h = 0.01 m) of the FP64 oracle's shadow-minutes, per building.

    The objective counts at most one flip per step interval.  A flip that moves across a
    step keeps it continuous (one interval's flip time runs to its end as the next one's
    starts), but a brief shadow or gap that appears or vanishes at a step makes it jump.
    So only receivers whose number of flips in some day differs between h - 0.01 and
    h + 0.01, for some building, are given weight 0 on both sides (the library takes
    per-receiver weights); receivers whose flips merely cross a step are kept."""
    B = cuda_lib
    w = configs.park(width=120.0, depth=80.0, dx=1.0, n_buildings=24, band=100.0, step=4.0)
    pos = w.ground.positions()
    bands = C.band_counts(w.city)

    def mesh(hs):
        return C.extrude(w.city, heights=hs, bands=bands)

    def bits(hs):
        m = mesh(hs)
        return oracle.shadow_bits(m.tri9(), m.tri_building, pos, None, w.sun.dirs)

    pert = []
    jump = np.zeros(pos.shape[0], bool)
    moved = np.zeros(pos.shape[0], bool)
    ds = w.sun.day_start
    for b in range(w.city.B):
        hp, hm = w.city.heights.copy(), w.city.heights.copy()
        hp[b] += np.float32(0.01)
        hm[b] -= np.float32(0.01)
        pert.append((hp, hm))
        bp, bm = bits(hp), bits(hm)
        moved |= (bp != bm).any(axis=1)
        jump |= (flips_per_day(bp, ds) != flips_per_day(bm, ds)).any(axis=1)
    assert jump.mean() < 0.05
    # flips that cross a step under the perturbation are kept, and there are some
    assert (moved & ~jump).sum() > 0
    wts = (~jump).astype(np.float64)

    scene = _fp_scene(B, w.city)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grad, S = B.sa_height_grad(scene, _grid(B, w.ground), sun, w.sun.step_minutes,
                               weights=wts.astype(np.float32))
    grad = grad.cpu().numpy().astype(np.float64)

    def S_or(hs):
        m = mesh(hs)
        return oracle.shadow_integral(m.tri9(), m.tri_building, pos, w.sun.dirs, w.sun.day_start,
                                      w.sun.step_minutes, weights=wts)
    S0 = S_or(w.city.heights)
    assert abs(float(S) - S0) <= 1e-4 * S0, (float(S), S0)
    fd = np.array([(S_or(hp) - S_or(hm)) / (float(hp[b]) - float(hm[b]))
                   for b, (hp, hm) in enumerate(pert)])
    scale = np.abs(fd).max()
    assert scale > 0
    err = np.abs(grad - fd)
    assert err.max() <= 1e-3 * scale, (err.max(), scale)
    big = np.abs(fd) > 0.05 * scale
    assert np.all(err[big] <= 1e-3 * np.abs(fd[big])), (err[big] / np.abs(fd[big])).max()


def test_autograd_function_returns_the_library_gradient(cuda_lib):
    B = cuda_lib
    from paper_1907_04435_gb300.autograd import shadow_minutes
    w = configs.park(width=120.0, depth=80.0, dx=1.0, n_buildings=24, band=100.0, step=6.0)
    scene = _fp_scene(B, w.city)
    grid = _grid(B, w.ground)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    h = torch.tensor(w.city.heights, device="cuda", dtype=torch.float64, requires_grad=True)
    S = shadow_minutes(h, scene, grid, sun, w.sun.step_minutes)
    (gh,) = torch.autograd.grad(S, h)
    g2, S2 = B.sa_height_grad(scene, grid, sun, w.sun.step_minutes)
    assert torch.allclose(gh.float(), g2) and float(S.detach()) == float(S2)
    # lowering the buildings along the gradient reduces the shadow
    with torch.no_grad():
        h2 = (h - 0.5 * gh / gh.abs().max()).clamp_min(1.0)
    S_low = shadow_minutes(h2.detach(), scene, grid, sun, w.sun.step_minutes)
    assert float(S_low) < float(S.detach())

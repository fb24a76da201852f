"""Per-kernel device timing: one event pair per launch of each timed kernel class, and the
timed calls' results unchanged."""
import pytest
import torch

from parity import workload

pytestmark = pytest.mark.gpu


def test_kernel_timing_counts_launches_and_keeps_results(cuda_lib):
    B = cuda_lib
    w = workload("district_small")
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    fac = B.Receivers.points(w.facade_pos, w.facade_nrm)
    ref = [B.sa_accumulate(scene, r, sun, 1.0, m)[0].clone()
           for r, m in ((grid, "accrual_sam"), (fac, "accrual_sam"), (fac, "accrual_trace"),
                        (fac, "sweep_trace"))]
    B.sa_kernel_times()                                   # empty the record
    old = B.sa_get_option(B.SA_OPT_KERNEL_TIMING)
    B.sa_set_option(B.SA_OPT_KERNEL_TIMING, 1)
    try:
        got = [B.sa_accumulate(scene, r, sun, 1.0, m)[0]
               for r, m in ((grid, "accrual_sam"), (fac, "accrual_sam"), (fac, "accrual_trace"),
                            (fac, "sweep_trace"))]
        t = B.sa_kernel_times()
    finally:
        B.sa_set_option(B.SA_OPT_KERNEL_TIMING, old)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    nb = sun.n_blocks
    assert t["raster"][1] == (nb + 63) // 64
    assert t["sam_points"][1] == (nb + 63) // 64          # one launch per chunk of blocks
    assert t["accrual"][1] == 1 and t["sweep"][1] == 1 and t["iam"][1] == 0
    for k in ("raster", "sam_points", "accrual", "sweep"):
        assert t[k][0] > 0.0
    # collected once: the record is empty again, and nothing is recorded with timing off
    B.sa_accumulate(scene, grid, sun, 1.0, "accrual_sam")
    assert all(v == (0.0, 0) for v in B.sa_kernel_times().values())

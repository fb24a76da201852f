"""The receiver split on one GPU: the district-small workload cut into rank shares (bands
of grid rows, ranges of facade points), each share accumulated on its own as a rank
would, gives the unsplit results bit for bit once the shares are concatenated in rank
order.  (The shares run one after another: no kernel of one waits for another.)"""
import numpy as np
import pytest
import torch

from paper_1907_04435_gb300 import shard
from synth import configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("method", ["accrual_sam", "accrual_trace"])
def test_shares_concatenate_to_the_unsplit_result(cuda_lib, world, method):
    B = cuda_lib
    w = configs.district_small()
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = (g.x0, g.y0, g.dx, g.nx, g.ny)
    full_g = [t.cpu().numpy() for t in B.sa_accumulate(scene, B.Receivers.ground_grid(*grid), sun,
                                                       w.sun.step_minutes, method)]
    full_f = [t.cpu().numpy() for t in B.sa_accumulate(scene, B.Receivers.points(w.facade_pos, w.facade_nrm),
                                                       sun, w.sun.step_minutes, method)]
    parts_g, parts_f = [], []
    for rank in range(world):
        x0, y0, dx, nx, rows, _ = shard.grid_band(grid, rank, world)
        parts_g.append([t.cpu().numpy() for t in B.sa_accumulate(
            scene, B.Receivers.ground_grid(x0, y0, dx, nx, rows), sun, w.sun.step_minutes, method)])
        a, b = shard.split(w.facade_pos.shape[0], rank, world)
        parts_f.append([t.cpu().numpy() for t in B.sa_accumulate(
            scene, B.Receivers.points(w.facade_pos[a:b], w.facade_nrm[a:b]), sun, w.sun.step_minutes, method)])
    torch.cuda.synchronize()
    for q in range(3):
        assert np.array_equal(np.concatenate([p[q] for p in parts_g]), full_g[q]), q
        assert np.array_equal(np.concatenate([p[q] for p in parts_f]), full_f[q]), q

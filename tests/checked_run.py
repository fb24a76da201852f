"""Runs every computing call of the library on small workloads and prints, as one JSON line,
a digest of each output plus the bounds-checked build's status.  Used by
test_gpu_checked.py, which runs it under the checked and the plain build in fresh processes
(the build is chosen by SA_CHECKED when the binding loads)."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1907_04435_gb300 import binding as B  # noqa: E402
from synth import configs  # noqa: E402


def digest(*ts):
    h = hashlib.sha256()
    for t in ts:
        if t is None:
            continue
        a = t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def main():
    out = {"checked": B.sa_checked_build()}
    w = configs.district_small()
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    open_scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    fac = B.Receivers.points(w.facade_pos, w.facade_nrm)
    for sc_name, sc in (("closed", scene), ("open", open_scene)):
        for m in ("accrual_sam", "accrual_trace", "sweep_trace", "sweep_raster", "iam"):
            out[f"{sc_name}/ground/{m}"] = digest(*B.sa_accumulate(sc, grid, sun, w.sun.step_minutes, m))
        for m in ("accrual_sam", "accrual_trace", "sweep_trace"):
            out[f"{sc_name}/facades/{m}"] = digest(*B.sa_accumulate(sc, fac, sun, w.sun.step_minutes, m))
    out["masks"] = digest(B.sa_shadow_masks(scene, grid, sun, "accrual_sam"))
    gg = B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, "accrual_sam", 5.0)
    out["graph"] = digest(*gg[:3])
    poly = np.array([[60.0, 40.0], [420.0, 90.0], [480.0, 250.0], [300.0, 330.0]], np.float32)
    c, n, st = B.sa_building_contribution(scene, grid, sun, poly)
    out["contribution"] = digest(c, n, np.asarray(st))
    gr = torch.zeros(grid.R, dtype=torch.int32, device="cuda")
    B.sa_accumulate_grid_noalloc(scene, grid, sun, w.sun.step_minutes, gr)
    out["noalloc"] = digest(gr)
    pk = configs.park(width=120.0, depth=80.0, dx=1.0, n_buildings=24, band=100.0, step=6.0)
    fs = B.Scene.from_footprints(pk.city.footprints, pk.city.heights, pk.city.band_height)
    pg = B.Receivers.ground_grid(pk.ground.x0, pk.ground.y0, pk.ground.dx, pk.ground.nx, pk.ground.ny)
    grad, S = B.sa_height_grad(fs, pg, B.Sun(pk.sun.dirs, pk.sun.day_start), pk.sun.step_minutes)
    out["height_grad"] = digest(grad, S)
    sc4 = configs.scenarios(n_variants=3, days=1, base=w)
    bt = B.Batch(scene, grid, sc4.tower_tris, sc4.removed, [(0, 0, 64, 64)] * 3,
                 [B.Sun(it.dirs, it.day_start) for it in sc4.intervals])
    out["batch"] = digest(*bt.run())
    torch.cuda.synchronize()
    out["status"] = B.sa_check_status()
    print(json.dumps(out))


if __name__ == "__main__":
    main()

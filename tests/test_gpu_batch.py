"""Batched scenarios: one persistent, graph-captured launch over (interval, variant, tile)
items equals per-scenario accumulation on each variant's own mesh, and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from synth import configs

from parity import assert_counts_parity

pytestmark = pytest.mark.gpu


def _small():
    base = configs.district_small(n_facade=0)
    return configs.scenarios(n_variants=6, days=2, step=10.0, base=base,
                             region_sides=(32, 64, 128), centres=(172, 355))


def _batch(B, sc, with_impact=True):
    w = sc.base
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    suns = [B.Sun(it.dirs, it.day_start) for it in sc.intervals]
    bt = B.Batch(scene, grid, sc.tower_tris, sc.removed, sc.regions, suns, with_impact)
    return scene, grid, suns, bt


def _region(arr, reg, g):
    ix0, iy0, nx, ny = reg
    return arr.reshape(g.ny, g.nx)[iy0:iy0 + ny, ix0:ix0 + nx].ravel()


def test_batch_equals_per_scenario_accumulation(cuda_lib):
    B = cuda_lib
    sc = _small()
    scene, grid, suns, bt = _batch(B, sc)
    assert bt.n_items > 0
    counts, impact = bt.run()
    torch.cuda.synchronize()
    counts, impact = counts.cpu().numpy(), impact.cpu().numpy()
    g = sc.base.ground
    base_counts = [B.sa_accumulate(scene, grid, s, 10.0, "accrual_sam")[0].cpu().numpy() for s in suns]
    for v in range(sc.V):
        t9, tb = sc.variant_mesh(v)
        verts = t9.reshape(-1, 3)
        tris = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
        vs = B.Scene(verts, tris, tb, int(tb.max()) + 1, closed=True)
        for i, s in enumerate(suns):
            full = B.sa_accumulate(vs, grid, s, 10.0, "accrual_sam")[0].cpu().numpy()
            o = bt.offset(i, v)
            n = int(sc.regions[v, 2] * sc.regions[v, 3])
            want = _region(full, sc.regions[v], g)
            assert np.array_equal(counts[o:o + n], want), (v, i)
            assert np.array_equal(impact[o:o + n], want - _region(base_counts[i], sc.regions[v], g))


def test_batch_matches_the_oracle_on_sampled_receivers(cuda_lib):
    B = cuda_lib
    sc = _small()
    _, _, _, bt = _batch(B, sc, with_impact=False)
    counts, _ = bt.run(want_impact=False)
    counts = counts.cpu().numpy()
    g = sc.base.ground
    pos = g.positions()
    rng = np.random.default_rng(3)
    it = sc.intervals[0]
    for v in range(sc.V):
        ix0, iy0, nx, ny = sc.regions[v]
        idx = rng.choice(nx * ny, size=min(200, nx * ny), replace=False)
        gl = (iy0 + idx // nx) * g.nx + (ix0 + idx % nx)
        t9, tb = sc.variant_mesh(v)
        bits = oracle.shadow_bits(t9, tb, pos[gl], None, it.dirs)
        near = oracle.near_boundary(t9, tb, pos[gl], None, it.dirs, it.day_start, bits)
        o = bt.offset(0, v)
        assert_counts_parity(counts[o + idx], None, bits, near, it.day_start, f"variant {v}")


def test_batch_tuning_keeps_results_and_reruns_are_stable(cuda_lib):
    B = cuda_lib
    sc = _small()
    _, _, _, bt = _batch(B, sc)
    a, ia = bt.run()
    a, ia = a.clone(), ia.clone()
    ctas, run = bt.tune()
    assert ctas > 0 and run in (8, 16, 24)
    b, ib = bt.run()
    c, ic = bt.run()
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(b, c) and torch.equal(ia, ib)
    w = bt.work_counters()
    assert w[2] > 0 and w[3] >= w[2]

"""Pins of the oracle's direction bins and direction graph (Sec. 6): the worked example of
Fig. 7, the bins' angular bound, exactness when every interval is its own edge, repeated
days (and the middle block as each edge's map), and the weighted gross sum of Eq. 1."""
import os

import numpy as np
import pytest

import oracle
from synth import configs
from synth.sun import sun_table

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "fig7_direction_graph.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            vals[k] = [int(x) for x in v]
    return vals


def _fig7_sun():
    """Two days of one-minute steps from 10:00 to 14:59; the second day repeats the first
    until 13:00 and then follows the sun of another season."""
    a = sun_table(40.7, [172], 10.0, 14.0 + 59 / 60, 1.0).dirs
    b = sun_table(40.7, [110], 10.0, 14.0 + 59 / 60, 1.0).dirs
    assert a.shape == (300, 3)
    day2 = np.concatenate([a[:180], b[180:]])
    return np.concatenate([a, day2]).astype(np.float32), np.array([0, 300, 600], np.int32)


def test_worked_example_of_fig7():
    g = _golden()
    dirs, ds = _fig7_sun()
    edge, rep, weight = oracle.direction_graph(dirs, ds, 60, 5.0)
    assert len(edge) == g["days"][0] * g["intervals_per_day"][0]
    assert len(rep) == g["edges"][0]
    assert sorted(weight.tolist(), reverse=True) == g["weights"]
    # the shared intervals are the first three of each day, in the same edges
    assert edge[:3].tolist() == edge[5:8].tolist() == [0, 1, 2]
    assert weight[:3].tolist() == [2, 2, 2]
    assert rep.tolist() == [0, 1, 2, 3, 4, 8, 9]


def test_bins_bound_both_angles():
    rng = np.random.default_rng(3)
    v = rng.normal(size=(20000, 3))
    v[:, 2] = np.abs(v[:, 2]) + 1e-3
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    for b in (2.5, 5.0, 10.0):
        eb, ab = oracle.direction_bins(v.astype(np.float32), b)
        el = np.degrees(np.arcsin(v[:, 2]))
        az = np.degrees(np.arctan2(v[:, 0], v[:, 1]))
        assert np.all((eb * b <= el + 1e-9) & (el < (eb + 1) * b + 1e-9))
        assert np.all((ab * b <= az + 1e-9) & (az < (ab + 1) * b + 1e-9))
        assert eb.min() >= 0 and eb.max() < int(np.ceil(90 / b))
        assert ab.min() >= -int(np.ceil(180 / b)) and ab.max() < int(np.ceil(180 / b))
    # north, east, south, west at the horizon fall in the sectors starting at 0, 90, 180, -90
    nesw = np.array([[0, 1, 1e-6], [1, 0, 1e-6], [0, -1, 1e-6], [-1, 0, 1e-6]], np.float32)
    assert oracle.direction_bins(nesw, 5.0)[1].tolist() == [0, 18, 36, -18]


def _box_bits(dirs):
    w = configs.boxes16()
    pos = w.ground.positions()[::7]
    return oracle.shadow_bits(w.mesh.tri9(), w.mesh.tri_building, pos, None, dirs)


def test_tiny_bins_give_the_exact_result():
    st = sun_table(40.7, [150, 172, 200], 9.0, 17.0, 2.0)
    edge, rep, weight = oracle.direction_graph(st.dirs, st.day_start, 60, 1e-7)
    assert len(rep) == len(edge) and np.all(weight == 1)
    bits = _box_bits(st.dirs)
    gb = oracle.graph_bits(bits, st.dirs, st.day_start, 60, 1e-7)
    assert np.array_equal(gb, bits)


def test_repeated_days_share_every_edge():
    one = sun_table(40.7, [172], 9.0, 17.0, 2.0)
    d = 4
    dirs = np.tile(one.dirs, (d, 1))
    ds = np.arange(d + 1, dtype=np.int32) * one.S
    edge, rep, weight = oracle.direction_graph(dirs, ds, 60, 5.0)
    nb = len(oracle.block_partition(one.day_start, 60)[0])
    assert len(rep) == nb and np.all(weight == d)
    # each edge's map is computed from its middle block: the second of four days
    assert np.array_equal(rep, np.arange(nb) + nb)
    bits1 = _box_bits(one.dirs)
    g1, c1 = oracle.reduce(bits1, one.day_start)
    gd, cd = oracle.reduce(oracle.graph_bits(_box_bits(dirs), dirs, ds, 60, 5.0), ds)
    assert np.array_equal(gd, d * g1) and np.array_equal(cd, c1)


def test_gross_is_the_weighted_sum_of_edge_maps_and_days_stitch_their_paths():
    """Eq. 1 (gross = sum_j G_j w_j over edges) and the continuous count, stitched along
    each day's path from the edges' prefix / maximum / suffix runs, against the plain
    counts of the substituted bits."""
    st = sun_table(40.7, list(range(160, 200, 3)), 9.0, 17.0, 2.0)
    bits = _box_bits(st.dirs)
    j0, K = oracle.block_partition(st.day_start, 30)
    edge, rep, weight = oracle.direction_graph(st.dirs, st.day_start, 30, 5.0)
    assert len(rep) < len(edge)
    gb = oracle.graph_bits(bits, st.dirs, st.day_start, 30, 5.0)
    g, c = oracle.reduce(gb, st.day_start)
    G = np.stack([bits[:, j0[r]:j0[r] + K[r]].sum(axis=1) for r in rep], axis=1)
    assert np.array_equal(g, G @ weight)

    def runs(x):
        p = int(np.argmin(x)) if not x.all() else len(x)
        s = int(np.argmin(x[::-1])) if not x.all() else len(x)
        best, cur = 0, 0
        for v in x:
            cur = cur + 1 if v else 0
            best = max(best, cur)
        return p, best, s, bool(x.all())

    days = np.searchsorted(j0, st.day_start[:-1])
    days = np.append(days, len(j0))
    for r in range(0, bits.shape[0], 13):
        want = 0
        for q in range(len(days) - 1):
            run, best = 0, 0
            for b in range(days[q], days[q + 1]):
                e = rep[edge[b]]
                p, m, s, full = runs(bits[r, j0[e]:j0[e] + K[e]])
                if full:
                    run += K[e]
                else:
                    best = max(best, run + p, m)
                    run = s
            want = max(want, best, run)
        assert c[r] == want, r


def test_blocks_of_different_lengths_are_different_edges():
    """An edge's map holds one bit per step, so only intervals with as many steps share
    it: a day cut short by ten minutes has 58-step blocks where the full day has 60."""
    a = sun_table(40.7, [172], 10.0, 14.0 + 59 / 60, 1.0).dirs
    dirs = np.concatenate([a, a[:290]]).astype(np.float32)
    ds = np.array([0, 300, 590], np.int32)
    j0, K = oracle.block_partition(ds, 60)
    edge, rep, weight = oracle.direction_graph(dirs, ds, 60, 5.0)
    assert K.tolist() == [60] * 5 + [58] * 5
    assert len(rep) == 10 and np.all(weight == 1)
    eb, ab = oracle.direction_bins(dirs, 5.0)
    same_bins = sum(eb[j0[b]] == eb[j0[b + 5]] and ab[j0[b]] == ab[j0[b + 5]] and
                    eb[j0[b] + 59] == eb[j0[b + 5] + 57] and ab[j0[b] + 59] == ab[j0[b + 5] + 57]
                    for b in range(5))
    assert same_bins >= 2          # without the length in the key these would merge

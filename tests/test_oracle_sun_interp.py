"""Pins of the oracle's endpoint-interpolated sun (Sec. 3.2 and Sec. 4): the steps between a
block's first and last directions rebuilt from those two alone.  Checked against an
independent axis-angle rotation, against the paper's own tangent law on a shadow plane
orthogonal to d_1, and against the true sun at the interval lengths of Table 1."""
import numpy as np
import pytest

import oracle
from synth.sun import sun_table


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _blocks(day_start, block_len):
    j0, K = oracle.block_partition(day_start, block_len)
    return list(zip(j0.tolist(), K.tolist()))


def test_block_ends_and_short_blocks_are_kept():
    st = sun_table(40.7, [172, 355], 9.0, 17.0, 1.0)
    out = oracle.sun_interpolate(st.dirs, st.day_start, 60)
    for a, n in _blocks(st.day_start, 60):
        assert np.array_equal(out[a], st.dirs[a]) and np.array_equal(out[a + n - 1], st.dirs[a + n - 1])
    for bl in (1, 2):
        assert np.array_equal(oracle.sun_interpolate(st.dirs, st.day_start, bl), st.dirs)
    # interior steps are rebuilt: they differ from the true sun somewhere
    assert not np.array_equal(out, st.dirs)


def test_steps_are_rotations_of_d1_about_the_common_normal():
    """Step i = d_1 turned about the axis d_1 x d_n by i' theta / (n - 1) (Rodrigues)."""
    st = sun_table(40.7, [79, 172, 355], 8.0, 16.0, 1.0)
    out = oracle.sun_interpolate(st.dirs, st.day_start, 64).astype(np.float64)
    worst = 0.0
    for a, n in _blocks(st.day_start, 64):
        d1, dn = _unit(st.dirs[a]), _unit(st.dirs[a + n - 1])
        k = np.cross(d1, dn)
        theta = np.arcsin(min(np.linalg.norm(k), 1.0))
        k = k / np.linalg.norm(k)
        for i in range(1, n - 1):
            phi = i * theta / (n - 1)
            r = d1 * np.cos(phi) + np.cross(k, d1) * np.sin(phi) + k * np.dot(k, d1) * (1 - np.cos(phi))
            worst = max(worst, float(np.abs(out[a + i] - r).max()))
    assert worst < 2e-7


def test_the_tangent_law_on_a_plane_orthogonal_to_d1_draws_the_same_steps():
    """Sec. 4: with the shadow plane orthogonal to d_1, a point s projects along d_1 to p_1
    and along d_n to p_n, and at step i to p_1 + (p_n - p_1) tan(i' theta / (n-1)) / tan theta.
    Projecting s along the interpolated direction of step i lands on that point."""
    rng = np.random.default_rng(11)
    # the true sun in 60-minute blocks, plus wide synthetic blocks where the law is far from linear
    st = sun_table(40.7, [172, 355], 9.0, 17.0, 1.0)
    cases = [(st.dirs, st.day_start, 60)]
    for theta_deg, n in ((25.0, 9), (50.0, 17)):
        d1 = _unit([0.3, -0.5, 0.8])
        ax = _unit(np.cross(d1, [0.1, 0.9, 0.2]))
        t = np.radians(theta_deg)
        dn = d1 * np.cos(t) + np.cross(ax, d1) * np.sin(t)
        dirs = np.stack([d1] + [_unit(d1 + 1e-3 * rng.normal(size=3)) for _ in range(n - 2)] + [dn])
        cases.append((dirs.astype(np.float32), np.array([0, n], np.int32), 64))
    for dirs, ds, bl in cases:
        out = oracle.sun_interpolate(dirs, ds, bl).astype(np.float64)
        for a, n in _blocks(ds, bl):
            if n <= 2:
                continue
            d1, dn = _unit(dirs[a]), _unit(dirs[a + n - 1])
            theta = np.arccos(np.clip(np.dot(d1, dn), -1, 1))
            s = np.array([12.0, -7.0, 55.0])
            delta = 80.0                                   # plane beyond s, seen from the light
            p1 = s - delta * d1
            pn = s - (delta / np.dot(d1, dn)) * dn
            for i in range(1, n - 1):
                want = p1 + (pn - p1) * np.tan(i * theta / (n - 1)) / np.tan(theta)
                di = _unit(out[a + i])
                got = s - (delta / np.dot(d1, di)) * di
                assert np.abs(got - want).max() < 2e-4 * (1 + np.abs(pn - p1).max()), (i, n, got, want)


def test_the_interpolated_sun_stays_close_to_the_true_one_as_in_table_1():
    """Table 1: the interpolated direction stays within a cosine of 0.99999 of the true
    one on average for hourly intervals, and the error grows with the interval length."""
    st = sun_table(40.7, list(range(1, 366, 5)), 7.0, 17.0, 1.0)
    truth = _unit(st.dirs)
    mean_cos = {}
    for bl in (10, 30, 60):
        out = _unit(oracle.sun_interpolate(st.dirs, st.day_start, bl))
        cs = np.sum(out * truth, axis=1)
        mean_cos[bl] = float(cs.mean())
        assert np.degrees(np.arccos(np.clip(cs.min(), -1, 1))) < 0.25
    assert mean_cos[60] > 0.99999
    assert mean_cos[10] > mean_cos[30] > mean_cos[60]

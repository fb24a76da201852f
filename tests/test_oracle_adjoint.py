"""Pins of the oracle's continuous-time shadow integral, used for finite differences of the
height gradient, against the single-box closed form computed here independently (numpy).

For a convex prism (footprint F, height h) a ground point p is in shadow for direction d
exactly when the line p + z u, u = d_xy / d_z, meets F for some z in [0, h]: the edge
constraints A_e + z B_e >= 0 give an interval of z.  A flip caused by roof edge e happens
where the entry height equals h, so  A_e + h B_e(a) = 0  and  da/dh = -B_e / (h B_e'(a)).
"""
import numpy as np

import oracle
from synth import city as C
from synth.sun import sun_table


def _slerp(a, b, al):
    th = np.arccos(np.clip(a @ b, -1, 1))
    d = (np.sin((1 - al) * th)[..., None] * a + np.sin(al * th)[..., None] * b) / np.sin(th)
    return d / np.linalg.norm(d, axis=-1, keepdims=True), th


def _interval(fp, h, p, u):
    """Entry/exit heights of the line p + z u through the CCW footprint, vectorised."""
    zlo = np.zeros(p.shape[0])
    zhi = np.full(p.shape[0], h)
    elo = np.full(p.shape[0], -1)
    ok = np.ones(p.shape[0], bool)
    n = fp.shape[0]
    for e in range(n):
        a, b = fp[e], fp[(e + 1) % n]
        c = b - a
        A = c[0] * (p[:, 1] - a[1]) - c[1] * (p[:, 0] - a[0])
        Bc = c[0] * u[:, 1] - c[1] * u[:, 0]
        with np.errstate(divide="ignore", invalid="ignore"):
            z = -A / Bc
        up = Bc > 0
        better = up & (z > zlo)
        zlo = np.where(better, z, zlo)
        elo = np.where(better, e, elo)
        zhi = np.where(Bc < 0, np.minimum(zhi, z), zhi)
        ok &= ~((Bc == 0) & (A < 0))
    return ok & (zlo <= zhi), zlo, zhi, elo


def closed_form(fp, h, pos, dirs, step_minutes):
    """(S, dS/dh) of one prism over consecutive steps of one day, flips by bisection."""
    p = pos[:, :2].astype(np.float64)
    S = 0.0
    G = 0.0
    d = dirs.astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for j in range(d.shape[0] - 1):
        a, b = d[j], d[j + 1]
        def inside(al):
            dd, _ = _slerp(a, b, np.asarray(al, np.float64))
            dd = np.broadcast_to(dd, (p.shape[0], 3))
            return _interval(fp, h, p, dd[:, :2] / dd[:, 2:3])[0]
        c0, c1 = inside(0.0), inside(1.0)
        S += step_minutes * np.sum(c0 & c1)
        f = np.nonzero(c0 != c1)[0]
        if f.size == 0:
            continue
        lo, hi = np.zeros(f.size), np.ones(f.size)
        pf = p[f]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            dd, _ = _slerp(a, b, mid)
            ins = _interval(fp, h, pf, dd[:, :2] / dd[:, 2:3])[0]
            same = ins == c0[f]
            lo, hi = np.where(same, mid, lo), np.where(same, hi, mid)
        al = 0.5 * (lo + hi)
        S += step_minutes * np.sum(np.where(c0[f], al, 1 - al))
        dd, th = _slerp(a, b, al)
        ddd = th * (-np.cos((1 - al) * th)[:, None] * a + np.cos(al * th)[:, None] * b) / np.sin(th)
        u = dd[:, :2] / dd[:, 2:3]
        du = (ddd[:, :2] * dd[:, 2:3] - dd[:, :2] * ddd[:, 2:3]) / dd[:, 2:3] ** 2
        ok, zlo, zhi, elo = _interval(fp, h, pf, u)
        roof = (elo >= 0) & (np.abs(zlo - h) <= 1e-6 * (h + 1)) & (zhi >= h - 1e-6 * (h + 1))
        for i in np.nonzero(roof)[0]:
            e = elo[i]
            c = fp[(e + 1) % fp.shape[0]] - fp[e]
            Bc = c[0] * u[i, 1] - c[1] * u[i, 0]
            dB = c[0] * du[i, 1] - c[1] * du[i, 0]
            G += step_minutes * (1.0 if c0[f][i] else -1.0) * (-Bc / (h * dB))
    return S, G


def test_shadow_integral_and_its_height_derivative_match_the_single_box_closed_form():
    fp = C.box_footprint(0.0, 0.0, 30.0, 20.0)
    h = 40.0
    city = C.City([fp], np.array([h], np.float32))
    st = sun_table(40.7, [80], 9.0, 17.0, 4.0)
    g = C.GroundGrid(-80.0, -80.0, 1.0, 190, 120)
    pos = g.positions()
    fp32 = fp.astype(np.float32).astype(np.float64)
    S_cf, G_cf = closed_form(fp32, h, pos, st.dirs, st.step_minutes)

    def S(hh):
        m = C.extrude(city, heights=np.array([hh], np.float32))
        return oracle.shadow_integral(m.tri9(), m.tri_building, pos, st.dirs, st.day_start,
                                      st.step_minutes)
    S0 = S(h)
    assert abs(S0 - S_cf) <= 1e-6 * S_cf, (S0, S_cf)
    hp, hm = float(np.float32(h + 0.01)), float(np.float32(h - 0.01))
    fd = (S(hp) - S(hm)) / (hp - hm)
    assert abs(fd - G_cf) <= 1e-3 * abs(G_cf), (fd, G_cf)
    assert G_cf > 0


def test_shadow_integral_counts_whole_steps_without_flips():
    """Zenith-like high sun over a receiver under the roof: every interval counts fully."""
    fp = C.box_footprint(0.0, 0.0, 30.0, 20.0)
    m = C.extrude(C.City([fp], np.array([40.0], np.float32)))
    st = sun_table(40.7, [172], 11.0, 13.0, 10.0)
    pos = np.array([[15.0, 10.0, 0.0], [500.0, 500.0, 0.0]], np.float32)
    S, per = oracle.shadow_integral(m.tri9(), m.tri_building, pos, st.dirs, st.day_start,
                                    st.step_minutes, per_receiver=True)
    assert per[0] == (st.S - 1) * st.step_minutes and per[1] == 0.0
    w = np.array([2.0, 5.0])
    assert oracle.shadow_integral(m.tri9(), m.tri_building, pos, st.dirs, st.day_start,
                                  st.step_minutes, weights=w) == 2.0 * per[0]


def test_shadow_integral_follows_the_great_circle_between_hourly_steps():
    """Steps an hour apart (about 15 degrees): between them the sun moves on the great
    circle at a constant rate, which a straight-line interpolation of the directions would
    miss by a measurable part of the step at every flip."""
    fp = C.box_footprint(0.0, 0.0, 30.0, 20.0)
    h = 40.0
    city = C.City([fp], np.array([h], np.float32))
    st = sun_table(40.7, [80], 9.0, 17.0, 60.0)
    g = C.GroundGrid(-80.0, -80.0, 1.0, 190, 120)
    pos = g.positions()
    fp32 = fp.astype(np.float32).astype(np.float64)
    S_cf, _ = closed_form(fp32, h, pos, st.dirs, st.step_minutes)
    m = C.extrude(city)
    S = oracle.shadow_integral(m.tri9(), m.tri_building, pos, st.dirs, st.day_start, st.step_minutes)
    assert abs(S - S_cf) <= 1e-6 * S_cf, (S, S_cf)
    assert st.S == 9

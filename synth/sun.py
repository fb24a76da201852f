"""Seeded-free, deterministic sun-direction tables (harness input, not part of the method).

The paper treats the sun as a directional light (Sec. 3.2) and tracks its motion over
the interval of interest; it does not say which solar-position algorithm it used.
Here the per-step direction table is computed with Spencer's (1971) Fourier series for
the solar declination, with the hour angle taken in local apparent solar time, so the
equation of time is not needed.  Both the CUDA path and the oracle consume the same
FP32 table, so the choice of solar algorithm cannot affect parity.

Frame: ENU metres (x = east, y = north, z = up).  Every vector points TOWARD the sun;
light travels along -d.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# 2019 is not a leap year: doy 172 = 21 June, doy 263 = 20 September.
DAYS_PER_YEAR = 365


def declination(doy: np.ndarray | float) -> np.ndarray:
    """Solar declination in radians, Spencer (1971) series in the day angle."""
    g = 2.0 * math.pi * (np.asarray(doy, dtype=np.float64) - 1.0) / DAYS_PER_YEAR
    return (0.006918 - 0.399912 * np.cos(g) + 0.070257 * np.sin(g)
            - 0.006758 * np.cos(2 * g) + 0.000907 * np.sin(2 * g)
            - 0.002697 * np.cos(3 * g) + 0.00148 * np.sin(3 * g))


def sun_direction(lat_deg: float, doy, solar_hour) -> np.ndarray:
    """Unit vector toward the sun (FP64), shape (..., 3), for apparent solar time `solar_hour`."""
    phi = math.radians(lat_deg)
    dec = declination(doy)
    omega = np.radians(15.0 * (np.asarray(solar_hour, dtype=np.float64) - 12.0))
    east = -np.cos(dec) * np.sin(omega)
    north = np.sin(dec) * math.cos(phi) - np.cos(dec) * np.cos(omega) * math.sin(phi)
    up = np.sin(dec) * math.sin(phi) + np.cos(dec) * np.cos(omega) * math.cos(phi)
    d = np.stack(np.broadcast_arrays(east, north, up), axis=-1)
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


@dataclass
class SunTable:
    """Per-step directions for D days, grouped by day.

    dirs:      float32 [S, 3]   unit vectors toward the sun (all with d_z > 0)
    day_start: int32   [D + 1]  steps of day k are dirs[day_start[k]:day_start[k+1]]
    step_minutes: length of one step (minutes)
    doys, hours: metadata per step (float64) for diagnostics
    """
    dirs: np.ndarray
    day_start: np.ndarray
    step_minutes: float
    doys: np.ndarray
    hours: np.ndarray

    @property
    def S(self) -> int:
        return int(self.dirs.shape[0])

    @property
    def D(self) -> int:
        return int(self.day_start.shape[0] - 1)


def sun_table(lat_deg: float, doys, t_start_h: float, t_end_h: float, step_minutes: float,
              min_elevation_deg: float = 0.5) -> SunTable:
    """Inclusive time grid t_start..t_end per day; steps at or below `min_elevation_deg` dropped.

    09:00-17:00 at 2 min gives 241 steps, at 1 min 481 steps (both ends inclusive).
    Directions are renormalised after the FP32 cast so |d| is within 1e-6 of 1.
    """
    doys = list(np.atleast_1d(doys))
    n = int(round((t_end_h - t_start_h) * 60.0 / step_minutes)) + 1
    hours = t_start_h + np.arange(n) * (step_minutes / 60.0)
    all_dirs, starts, all_doy, all_h = [], [0], [], []
    for doy in doys:
        d = sun_direction(lat_deg, doy, hours)
        keep = d[:, 2] > math.sin(math.radians(min_elevation_deg))
        d = d[keep]
        all_dirs.append(d)
        all_doy.append(np.full(d.shape[0], float(doy)))
        all_h.append(hours[keep])
        starts.append(starts[-1] + d.shape[0])
    dirs = np.concatenate(all_dirs).astype(np.float32)
    dirs /= np.linalg.norm(dirs.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    return SunTable(dirs=np.ascontiguousarray(dirs, dtype=np.float32),
                    day_start=np.asarray(starts, dtype=np.int32),
                    step_minutes=float(step_minutes),
                    doys=np.concatenate(all_doy), hours=np.concatenate(all_h))

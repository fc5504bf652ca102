"""Oracle: baseline coordinates (u, v, w) from antenna positions.

Test infrastructure only (see ``oracle/__init__``).

The paper's measurement equation (Eq. ME) takes the baseline vector b_ij in
wavelengths in the frame of the phase centre: u towards east, v towards
north on the sky, w towards the source.  Here the antennas are given in the
local horizon frame (east, north, up) at latitude phi, the source at
declination delta and hour angle H.  Two rotations take a local vector there:
about the east axis by (pi/2 - phi), which gives the equatorial frame (X to
the meridian on the equator, Y east, Z to the pole), then the one that
brings the source direction (H, delta) onto the third axis.  Written out as
matrices and applied to b_ij = x_j - x_i (metres), one row per baseline in
the order (0,1), (0,2), ..., (1,2), ...
"""
from __future__ import annotations

import math

import numpy as np


def horizon_to_equatorial(lat_rad: float) -> np.ndarray:
    """3x3 matrix: (east, north, up) -> (X, Y, Z)."""
    s, c = math.sin(lat_rad), math.cos(lat_rad)
    return np.array([[0.0, -s, c],
                     [1.0, 0.0, 0.0],
                     [0.0, c, s]])


def equatorial_to_uvw(ha_rad: float, dec_rad: float) -> np.ndarray:
    """3x3 matrix: (X, Y, Z) -> (u, v, w) for a source at hour angle H and declination delta."""
    sh, ch = math.sin(ha_rad), math.cos(ha_rad)
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    return np.array([[sh, ch, 0.0],
                     [-sd * ch, sd * sh, cd],
                     [cd * ch, -cd * sh, sd]])


def uvw(enu_m, lat_rad: float, dec_rad: float, ha_rad) -> np.ndarray:
    """float64 [n_time][n_bl][3] baseline coordinates in metres."""
    enu = np.asarray(enu_m, dtype=np.float64)
    n = enu.shape[0]
    ij = [(i, j) for i in range(n) for j in range(i + 1, n)]
    b = np.array([enu[j] - enu[i] for i, j in ij])                 # [n_bl][3] horizon frame
    E = horizon_to_equatorial(lat_rad)
    out = []
    for h in np.atleast_1d(np.asarray(ha_rad, dtype=np.float64)):
        M = equatorial_to_uvw(float(h), dec_rad) @ E
        out.append(b @ M.T)
    return np.asarray(out)

"""Pins of the oracle's (u, v, w) from antenna positions (oracle/geometry.py)
against what the rotation must preserve and cases with a known answer."""
import math

import numpy as np

from oracle import geometry as G

DEG = math.pi / 180.0


def test_rotations_preserve_baseline_lengths():
    rng = np.random.default_rng(1)
    enu = rng.normal(0.0, 500.0, (6, 3))
    u = G.uvw(enu, 34 * DEG, 30 * DEG, np.linspace(-1.0, 1.0, 7))
    ij = [(i, j) for i in range(6) for j in range(i + 1, 6)]
    lens = np.array([np.linalg.norm(enu[j] - enu[i]) for i, j in ij])
    assert np.allclose(np.linalg.norm(u, axis=-1), lens[None, :], rtol=1e-13)


def test_known_cases():
    enu = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0], [0.0, 200.0, 0.0], [0.0, 0.0, 50.0]])
    # an east-west baseline at transit lies along u for any latitude and declination
    for lat, dec in ((34.0, 30.0), (-20.0, -60.0), (0.0, 0.0)):
        u = G.uvw(enu, lat * DEG, dec * DEG, [0.0])[0]
        assert np.allclose(u[0], [100.0, 0.0, 0.0], atol=1e-12)
    # at the pole, looking at the pole: up is w, and (east, north) turn with H
    for h in (0.0, 0.4, -1.1):
        u = G.uvw(enu, 90 * DEG, 90 * DEG, [h])[0]
        assert np.allclose(u[2], [0.0, 0.0, 50.0], atol=1e-12)               # (0, 3): up
        e_uv = u[0][:2] / 100.0                                              # (0, 1): east
        n_uv = u[1][:2] / 200.0                                              # (0, 2): north
        # X = -north, Y = east at the pole; u = sin H X + cos H Y, v = -cos H X + sin H Y
        assert np.allclose(e_uv, [math.cos(h), math.sin(h)], atol=1e-12)
        assert np.allclose(n_uv, [-math.sin(h), math.cos(h)], atol=1e-12)
    # on the equator, a source at the zenith (dec 0, H 0): north is v, up is w
    u = G.uvw(enu, 0.0, 0.0, [0.0])[0]
    assert np.allclose(u[1], [0.0, 200.0, 0.0], atol=1e-12)
    assert np.allclose(u[2], [0.0, 0.0, 50.0], atol=1e-12)


def test_baseline_order_and_antisymmetry():
    rng = np.random.default_rng(2)
    enu = rng.normal(0.0, 300.0, (4, 3))
    u = G.uvw(enu, 34 * DEG, 30 * DEG, [0.3])[0]
    rev = G.uvw(enu[::-1], 34 * DEG, 30 * DEG, [0.3])[0]
    # reversing the antennas turns (i, j) into (n-1-j, n-1-i): same pairs, opposite sign
    ij = [(i, j) for i in range(4) for j in range(i + 1, 4)]
    for k, (i, j) in enumerate(ij):
        kr = ij.index((3 - j, 3 - i))
        assert np.allclose(rev[kr], -u[k], atol=1e-10)

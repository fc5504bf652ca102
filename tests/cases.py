"""Tiny seeded problems shared by the oracle pins and the GPU parity tests.

Inputs come from ``paper_1709_08681_gb300.inputs``; the oracle is used only
to turn them into expected values (model grid, predicted visibilities).
"""
import math

import numpy as np

from paper_1709_08681_gb300 import inputs as I


def geometry(n_ant=6, extent_m=300.0, n_time=6, span_h=1.0, freqs=(1.4e9,), seed=1):
    enu = I.y_layout(n_ant, extent_m, seed)
    ha = np.linspace(-span_h / 2, span_h / 2, n_time) * 15 * I.DEG if n_time > 1 else np.zeros(1)
    uvw = I.uvw_tracks(enu, 34 * I.DEG, 30 * I.DEG, ha)
    return uvw, np.asarray(freqs, dtype=np.float64)


# (kind, N, cell arcsec, Ng): grids with the kernel inside S=32 taps and the
# primary beam's periodic aliases far outside the image.
GAUSS_SMALL = ("gauss", 64, 41.25, 360)
DISK_SMALL = ("disk", 64, 24.0, 1024)


def problem(spec=DISK_SMALL, n_ant=6, n_time=6, freqs=(1.4e9,), n_src=8, sigma_arcsec=20.0,
            seed=1, support=32, decorrelation=1, extent_m=300.0):
    """(oracle Model, sky [n][3], true offsets [n_ant][2], image)."""
    from oracle import model_grid, psc
    kind, N, cell_as, Ng = spec
    uvw, freq = geometry(n_ant, extent_m, n_time, 1.0, freqs, seed)
    cell = cell_as * I.ARCSEC
    sky = I.sky_points(n_src, 12.0 * I.ARCMIN, N, cell, ("loguniform", 0.1, 1.0), seed)
    img = I.sky_image(sky, N, cell)
    lm = I.true_offsets(n_ant, sigma_arcsec * I.ARCSEC, seed)
    grid = model_grid.grid_from_image(img, Ng)
    m = psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=n_ant, grid=grid, cell_rad=cell, support=support,
                  oversample=20, ap_kind=kind, diam_m=25.0,
                  alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=decorrelation)
    return m, sky, lm, img


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))

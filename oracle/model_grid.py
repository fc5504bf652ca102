"""Oracle: the model grid V° = F[I^M] (Algorithm 1, first pre-compute; Eq. MEDD).

Test infrastructure only (see ``oracle/__init__``).

Convention (Eq. ME uses exp(+2 pi i s.b)): image pixel (row, col) sits at
l = (col - N/2) dl, m = (row - N/2) dl; grid cell (gy, gx) at
u = (gx - Ng/2) du, v = (gy - Ng/2) du with du = 1 / (Ng dl).  Then

    G[gy, gx] = sum_{row, col} I[row, col] exp(+2 pi i ((gx - Ng/2)(col - N/2)
                                                       + (gy - Ng/2)(row - N/2)) / Ng)

which is the unnormalised DFT of the image zero-padded to Ng x Ng.  It is
written as two matrix products with the DFT matrix E[g, c]; the phase index
(g - Ng/2)(c - N/2) is reduced modulo Ng in exact integer arithmetic.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n_grid: int, n_img: int) -> np.ndarray:
    g = np.arange(n_grid, dtype=np.int64) - n_grid // 2
    c = np.arange(n_img, dtype=np.int64) - n_img // 2
    k = np.mod(np.outer(g, c), n_grid)
    return np.exp(2j * np.pi * k.astype(np.float64) / n_grid)


def grid_from_image(image: np.ndarray, n_grid: int) -> np.ndarray:
    """complex128 [Ng][Ng] grid of the N x N image (see module docstring)."""
    image = np.asarray(image, dtype=np.float64)
    E = dft_matrix(n_grid, image.shape[0])
    return (E @ image) @ E.T


def grid_from_components(src: np.ndarray, n_grid: int, du: float, flux=None) -> np.ndarray:
    """Same grid from point components (l, m, S): G = sum_k S_k exp(+2 pi i (u l_k + v m_k)).
    ``flux`` (optional, complex) replaces the column S."""
    g = (np.arange(n_grid, dtype=np.float64) - n_grid // 2) * du
    ex = np.exp(2j * np.pi * np.outer(g, src[:, 0]))
    ey = np.exp(2j * np.pi * np.outer(g, src[:, 1]))
    s = src[:, 2] if flux is None else np.asarray(flux)
    return (ey * s[None, :]) @ ex.T

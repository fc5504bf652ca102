"""Seeded synthetic inputs shaped like the paper's simulated observations.

This module holds no step of the Pointing SelfCal arithmetic.  It draws the
*inputs* of the method: antenna layouts, uvw tracks from standard
interferometer geometry, channel frequencies, point-source skies (and their
pixel images), true pointing offsets and thermal-noise samples.  The oracle
tests and the GPU path both take their inputs from here, so neither side's
arithmetic can leak into the other through the generator.

The sizes follow the paper's VLA simulation (Sec. 4.1: 27 antennas, L band,
offsets of order 20 arcsec, a sky spread across the primary beam) and the
workload table of this project (see ``WORKLOADS``).  Every draw comes from
``numpy.random.Generator(PCG64)`` seeded by ``(seed, stream)``, which gives the
same numbers on x86-64 and aarch64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0          # m/s
ARCSEC = math.pi / (180.0 * 3600.0)
ARCMIN = 60.0 * ARCSEC
DEG = math.pi / 180.0

# Gaussian EFP parameter matched to the uniform-disk (Airy) power beam's
# half-power width, per unit aperture diameter in wavelengths:
#   alpha = ALPHA_PER_DLAMBDA_DISK * D/lambda.
# The Airy power pattern (2 J1(x)/x)^2 falls to 1/2 at x_h = 1.6163399...
# (x = pi D_lambda rho), and a Gaussian power beam exp(-2 alpha^2 rho^2)
# falls to 1/2 at rho = sqrt(ln2 / 2) / alpha, so
#   alpha / D_lambda = pi sqrt(ln 2 / 2) / x_h.
# The value is an input parameter of the disk model; a CPU test recomputes it
# from the Bessel function.
ALPHA_PER_DLAMBDA_DISK = 1.1442341324495227


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


# ---------------------------------------------------------------- layouts

def y_layout(n_ant: int, arm_m: float, seed: int) -> np.ndarray:
    """ENU positions (m) of a Y-shaped array: three arms 120 deg apart, the
    radii of each arm's antennas drawn U(0.02, 1) * arm and sorted."""
    rng = _rng(seed, 1)
    per = [n_ant // 3 + (1 if k < n_ant % 3 else 0) for k in range(3)]
    pos = []
    for k in range(3):
        az = (5.0 + 120.0 * k) * DEG
        r = np.sort(rng.uniform(0.02, 1.0, per[k])) * arm_m
        for rr in r:
            pos.append((rr * math.sin(az), rr * math.cos(az), 0.0))
    return np.asarray(pos, dtype=np.float64)


def disk_layout(n_ant: int, radius_m: float, seed: int) -> np.ndarray:
    """ENU positions (m) of a centrally concentrated random array: half of the
    antennas uniform within 0.2 R, the rest uniform in the annulus to R."""
    rng = _rng(seed, 2)
    n_in = n_ant // 2
    r_in = 0.2 * radius_m * np.sqrt(rng.uniform(0.0, 1.0, n_in))
    u = rng.uniform(0.0, 1.0, n_ant - n_in)
    r_out = radius_m * np.sqrt(0.04 + (1.0 - 0.04) * u)
    r = np.concatenate([r_in, r_out])
    th = rng.uniform(0.0, 2.0 * math.pi, n_ant)
    return np.stack([r * np.sin(th), r * np.cos(th), np.zeros(n_ant)], axis=1)


def baselines(n_ant: int) -> np.ndarray:
    """Antenna pairs (i, j), i < j, in lexicographic order: (0,1), (0,2), ..."""
    return np.asarray([(i, j) for i in range(n_ant) for j in range(i + 1, n_ant)], dtype=np.int32)


def uvw_tracks(enu_m: np.ndarray, lat_rad: float, dec_rad: float,
               hour_angles_rad: np.ndarray) -> np.ndarray:
    """Baseline coordinates (m) ``[n_time][n_bl][3]`` for b_ij = x_j - x_i.

    Standard conversion: local ENU to equatorial XYZ at latitude ``lat``, then
    the (u, v, w) rotation for hour angle H and declination dec.
    """
    e, n, up = enu_m[:, 0], enu_m[:, 1], enu_m[:, 2]
    sl, cl = math.sin(lat_rad), math.cos(lat_rad)
    X = -sl * n + cl * up
    Y = e
    Z = cl * n + sl * up
    bl = baselines(enu_m.shape[0])
    bx = X[bl[:, 1]] - X[bl[:, 0]]
    by = Y[bl[:, 1]] - Y[bl[:, 0]]
    bz = Z[bl[:, 1]] - Z[bl[:, 0]]
    H = np.asarray(hour_angles_rad, dtype=np.float64)[:, None]
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    sH, cH = np.sin(H), np.cos(H)
    u = sH * bx + cH * by
    v = -sd * cH * bx + sd * sH * by + cd * bz
    w = cd * cH * bx - cd * sH * by + sd * bz
    return np.ascontiguousarray(np.stack([u, v, w], axis=-1))


# ---------------------------------------------------------------- skies

def sky_points(n_src: int, radius_rad: float, n_img: int, cell_rad: float,
               flux: tuple, seed: int) -> np.ndarray:
    """Point sources ``[n_src][3]`` = (l, m, S), uniform in a disc of radius
    ``radius_rad`` intersected with the image, snapped to pixel centres
    (l = (col - N/2) cell, m = (row - N/2) cell), so that the pixel image and
    the component list describe the same sky.

    ``flux`` is ("loguniform", smin, smax) or ("powerlaw", smin, smax, index):
    p(S) ~ S^index.
    """
    rng = _rng(seed, 3)
    half = (n_img // 2 - 1) * cell_rad
    out = []
    while len(out) < n_src:
        r = radius_rad * math.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2.0 * math.pi)
        l, m = r * math.cos(th), r * math.sin(th)
        if abs(l) > half or abs(m) > half:
            continue
        out.append((round(l / cell_rad) * cell_rad, round(m / cell_rad) * cell_rad))
    lm = np.asarray(out)
    u = rng.uniform(0.0, 1.0, n_src)
    if flux[0] == "loguniform":
        s = np.exp(math.log(flux[1]) + u * (math.log(flux[2]) - math.log(flux[1])))
    elif flux[0] == "powerlaw":
        a = 1.0 + flux[3]
        s = (flux[1] ** a + u * (flux[2] ** a - flux[1] ** a)) ** (1.0 / a)
    else:
        raise ValueError(flux)
    return np.concatenate([lm, s[:, None]], axis=1)


def sky_image(src: np.ndarray, n_img: int, cell_rad: float) -> np.ndarray:
    """Pixel image (float32, Jy/pixel) of point sources on pixel centres:
    pixel (row, col) holds the flux at l = (col - N/2) cell, m = (row - N/2) cell."""
    img = np.zeros((n_img, n_img), dtype=np.float64)
    col = np.rint(src[:, 0] / cell_rad).astype(np.int64) + n_img // 2
    row = np.rint(src[:, 1] / cell_rad).astype(np.int64) + n_img // 2
    np.add.at(img, (row, col), src[:, 2])
    return img.astype(np.float32)


def true_offsets(n_ant: int, sigma_rad: float, seed: int, stream: int = 4) -> np.ndarray:
    """Pointing offsets ``[n_ant][2]`` (rad), Gaussian per antenna per axis."""
    return _rng(seed, stream).normal(0.0, sigma_rad, (n_ant, 2))


def drifting_offsets(n_ant: int, n_steps: int, sigma_mean_rad: float, step_rad: float, seed: int,
                     stream: int = 6) -> np.ndarray:
    """Pointing that drifts: per antenna a mean offset, Gaussian sigma_mean per
    axis, plus a random walk whose steps (one per solution interval) are
    Gaussian step_rad per axis; the offset is constant within an interval.
    Returns [n_steps][n_ant][2] (rad)."""
    rng = _rng(seed, stream)
    mean = rng.normal(0.0, sigma_mean_rad, (n_ant, 2))
    steps = rng.normal(0.0, step_rad, (n_steps, n_ant, 2))
    steps[0] = 0.0
    return mean[None] + np.cumsum(steps, axis=0)


def squinted_offsets(n_ant: int, sigma_mech_rad: float, squint_rad: float, seed: int, stream: int = 7):
    """Pointing of the two parallel-hand polarisations (R, L) of each antenna:
    a mechanical offset, Gaussian sigma_mech per axis, and a beam squint of
    length squint_rad in a random direction per antenna that displaces the R
    beam by +squint/2 and the L beam by -squint/2.  Returns (mech [n_ant][2],
    squint [n_ant][2], lm_R, lm_L) in rad."""
    rng = _rng(seed, stream)
    mech = rng.normal(0.0, sigma_mech_rad, (n_ant, 2))
    th = rng.uniform(0.0, 2.0 * math.pi, n_ant)
    sq = squint_rad * np.stack([np.cos(th), np.sin(th)], axis=1)
    return mech, sq, mech + 0.5 * sq, mech - 0.5 * sq


def complex_noise(shape, sigma: float, seed: int, stream: int = 5) -> np.ndarray:
    """Complex Gaussian noise, real and imaginary parts each N(0, sigma^2)."""
    g = _rng(seed, stream).normal(0.0, sigma, tuple(shape) + (2,))
    return (g[..., 0] + 1j * g[..., 1]).astype(np.complex64)


# ---------------------------------------------------------------- workloads

@dataclasses.dataclass
class Workload:
    """Everything a solve needs except the observed visibilities.

    Visibilities are ``[n_time][n_bl][n_chan]`` complex64; uvw ``[n_time][n_bl][3]``
    float64 metres; the image ``[N][N]`` float32 with l = (col - N/2) cell.
    ``intervals`` splits the time axis into solution intervals (t0, nt).
    """
    name: str
    enu_m: np.ndarray
    uvw_m: np.ndarray
    freq_hz: np.ndarray
    sky: np.ndarray
    image: np.ndarray
    cell_rad: float
    n_grid: int
    support: int
    oversample: int
    ap_kind: str           # "disk" or "gauss"
    diam_m: float
    alpha_per_dlambda: float
    decorrelation: int
    lm_true: np.ndarray    # [n_interval][n_ant][2]
    sigma_pt: float        # rms of the true offsets per axis (rad)
    sigma_noise: float
    intervals: list
    seed: int

    @property
    def n_ant(self):
        return self.enu_m.shape[0]

    @property
    def n_bl(self):
        return self.n_ant * (self.n_ant - 1) // 2

    @property
    def n_time(self):
        return self.uvw_m.shape[0]

    @property
    def n_chan(self):
        return self.freq_hz.shape[0]

    @property
    def n_vis(self):
        return self.n_time * self.n_bl * self.n_chan

    def noise(self, stream: int = 5) -> np.ndarray:
        return complex_noise((self.n_time, self.n_bl, self.n_chan), self.sigma_noise, self.seed, stream)


def _hour_angles(r: dict) -> np.ndarray:
    """Hour angles (rad): ``n_time`` samples evenly spread over ``span_h``
    hours, or spaced ``dt_s`` seconds apart, centred on transit."""
    n_t = r["n_time"]
    centre = r.get("ha_centre_h", 0.0) * 15.0 * DEG
    if "dt_s" in r:
        return centre + (np.arange(n_t) - (n_t - 1) / 2.0) * r["dt_s"] / 3600.0 * 15.0 * DEG
    if n_t == 1:
        return np.full(1, centre)
    return centre + np.linspace(-r["span_h"] / 2, r["span_h"] / 2, n_t) * 15.0 * DEG


def make_workload(name: str, seed: int = 0, **over) -> Workload:
    """Build one of the named workloads (see ``WORKLOADS``); keyword
    arguments override entries of the recipe (for reduced test sizes)."""
    r = dict(WORKLOADS[name])
    r.update(over)
    if r["layout"] == "y":
        enu = y_layout(r["n_ant"], r["extent_m"], seed)
    else:
        enu = disk_layout(r["n_ant"], r["extent_m"], seed)
    ha = _hour_angles(r)
    uvw = uvw_tracks(enu, r["lat_deg"] * DEG, r["dec_deg"] * DEG, ha)
    nc = r["n_chan"]
    if nc == 1:
        freq = np.asarray([r["f_lo"]], dtype=np.float64)
    else:
        freq = r["f_lo"] + (np.arange(nc) + 0.5) * (r["f_hi"] - r["f_lo"]) / nc
    cell = r["cell_arcsec"] * ARCSEC
    sky = sky_points(r["n_src"], r["src_radius_arcmin"] * ARCMIN, r["n_img"], cell, r["flux"], seed)
    img = sky_image(sky, r["n_img"], cell)
    n_int = r["n_interval"]
    nt = r["n_time"] // n_int
    intervals = [(k * nt, nt) for k in range(n_int)]
    if r.get("pointing") == "walk":
        lm_true = drifting_offsets(r["n_ant"], n_int, r["sigma_pt_arcsec"] * ARCSEC,
                                   r["walk_arcsec_per_step"] * ARCSEC, seed)
    else:
        lm_true = np.stack([true_offsets(r["n_ant"], r["sigma_pt_arcsec"] * ARCSEC, seed, 100 + k)
                            for k in range(n_int)])
    return Workload(
        name=name, enu_m=enu, uvw_m=uvw, freq_hz=np.asarray(freq, dtype=np.float64), sky=sky,
        image=img, cell_rad=cell, n_grid=r["n_img"] * r["pad"], support=r["support"],
        oversample=r["oversample"], ap_kind=r["ap_kind"], diam_m=r["diam_m"],
        alpha_per_dlambda=r.get("alpha_per_dlambda", ALPHA_PER_DLAMBDA_DISK),
        decorrelation=r["decorrelation"], lm_true=lm_true, sigma_pt=r["sigma_pt_arcsec"] * ARCSEC,
        sigma_noise=r["noise_jy"],
        intervals=intervals, seed=seed)


# Recipes.  "disk64_l16ch": the learned-initialiser case (64 antennas of
# 13.5 m in a centrally concentrated disk of 4 km radius, 16 channels over
# 1.3-1.5 GHz, 60 x 10 s, offsets sigma 30", 0.5 mJy noise, 200 sources in
# the primary beam on a 2048^2 image of 2.5" padded to 8192^2);
# "vla27_l1ch": the small plain-method case (27 antennas, one
# channel at 1.4 GHz, 60 x 10 s over +-1 h, 50 sources on a 256^2 image at
# 6"); "vla27_l64ch": the precision-study case (64 channels over 1-2 GHz,
# 600 x 2 s in 4 solution intervals, 2000 sources on a 2048^2 image).
# "drift197_l128ch": the full-scale case (197 antennas of 15 m in a random
# disk of 8 km radius, 128 channels over 0.95-1.76 GHz, 1800 x 1 s, a 4096^2
# image at 1" padded to 8192^2 with 10^4 sources; pointing = a 30" mean plus
# a random walk of 2" per minute, solved every 60 s: 30 intervals).
WORKLOADS = {
    "drift197_l128ch": dict(
        layout="disk", n_ant=197, extent_m=8000.0, lat_deg=34.0, dec_deg=30.0,
        n_time=1800, dt_s=1.0, n_chan=128, f_lo=0.95e9, f_hi=1.76e9,
        n_src=10000, src_radius_arcmin=30.0, flux=("powerlaw", 1e-4, 1.0, -1.5),
        n_img=4096, cell_arcsec=1.0, pad=2, support=32, oversample=20,
        ap_kind="disk", diam_m=15.0, decorrelation=1,
        sigma_pt_arcsec=30.0, walk_arcsec_per_step=2.0, pointing="walk", noise_jy=1e-3, n_interval=30),
    "disk64_l16ch": dict(
        layout="disk", n_ant=64, extent_m=4000.0, lat_deg=34.0, dec_deg=30.0,
        n_time=60, dt_s=10.0, n_chan=16, f_lo=1.3e9, f_hi=1.5e9,
        n_src=200, src_radius_arcmin=30.0, flux=("powerlaw", 1e-4, 1.0, -1.5),
        n_img=2048, cell_arcsec=2.5, pad=4, support=32, oversample=20,
        ap_kind="disk", diam_m=13.5, decorrelation=1,
        sigma_pt_arcsec=30.0, noise_jy=5e-4, n_interval=1),
    "vla27_l1ch": dict(
        layout="y", n_ant=27, extent_m=1000.0, lat_deg=34.0, dec_deg=30.0,
        n_time=60, span_h=2.0, n_chan=1, f_lo=1.4e9, f_hi=1.4e9,
        n_src=50, src_radius_arcmin=15.0, flux=("loguniform", 1e-3, 1.0),
        n_img=256, cell_arcsec=6.0, pad=16, support=32, oversample=20,
        ap_kind="disk", diam_m=25.0, decorrelation=1,
        sigma_pt_arcsec=20.0, noise_jy=1e-3, n_interval=1),
    "vla27_l64ch": dict(
        layout="y", n_ant=27, extent_m=1000.0, lat_deg=34.0, dec_deg=30.0,
        n_time=600, dt_s=2.0, n_chan=64, f_lo=1.0e9, f_hi=2.0e9,
        n_src=2000, src_radius_arcmin=21.0, flux=("powerlaw", 1e-4, 2.0, -1.5),
        n_img=2048, cell_arcsec=8.0, pad=1, support=32, oversample=20,
        ap_kind="disk", diam_m=25.0, decorrelation=1,
        sigma_pt_arcsec=20.0, noise_jy=1e-3, n_interval=4),
}


# ---------------------------------------------------------------- mixed batches

# Array types of the batched-solve workload: 16 channels over 1.3-1.5 GHz,
# 10 s samples; per type a layout, dish, sky and grid.  Pixel size about
# 1 / (2.2 u_max), the image covering about 1.5 primary-beam widths.
MIXED_ARRAYS = {
    "y27": dict(layout="y", n_ant=27, extent_m=1000.0, diam_m=25.0, n_img=256, cell_arcsec=11.0, pad=4,
                n_src=50, src_radius_arcmin=15.0),
    "disk64": dict(layout="disk", n_ant=64, extent_m=4000.0, diam_m=13.5, n_img=2048, cell_arcsec=2.5, pad=4,
                   n_src=200, src_radius_arcmin=30.0),
    "disk197": dict(layout="disk", n_ant=197, extent_m=8000.0, diam_m=15.0, n_img=4096, cell_arcsec=1.2, pad=2,
                    n_src=400, src_radius_arcmin=27.0),
}
MIXED_COMMON = dict(lat_deg=34.0, dec_deg=30.0, dt_s=10.0, n_chan=16, f_lo=1.3e9, f_hi=1.5e9, support=32,
                    oversample=20, ap_kind="disk", decorrelation=1, noise_jy=1e-3,
                    flux=("powerlaw", 1e-4, 1.0, -1.5))


@dataclasses.dataclass
class MixedArray:
    """One array type of a mixed batch: geometry, channels, sky and grid."""
    name: str
    enu_m: np.ndarray
    freq_hz: np.ndarray
    sky: np.ndarray
    image: np.ndarray
    cell_rad: float
    n_grid: int
    support: int
    oversample: int
    ap_kind: str
    diam_m: float
    alpha_per_dlambda: float
    decorrelation: int
    sigma_noise: float
    lat_rad: float
    dec_rad: float

    @property
    def n_ant(self):
        return self.enu_m.shape[0]

    @property
    def n_bl(self):
        return self.n_ant * (self.n_ant - 1) // 2


@dataclasses.dataclass
class MixedInterval:
    """One solution interval of a mixed batch."""
    array: str
    hour_angles: np.ndarray    # [n_time] rad
    lm_true: np.ndarray        # [n_ant][2] rad
    sigma_pt: float            # rad
    outliers: np.ndarray       # antennas whose offset is an outlier
    noise_seed: int

    @property
    def n_time(self):
        return self.hour_angles.shape[0]


def mixed_arrays(seed: int = 0, names=("y27", "disk64", "disk197")) -> dict:
    out = {}
    c = MIXED_COMMON
    nc = c["n_chan"]
    freq = c["f_lo"] + (np.arange(nc) + 0.5) * (c["f_hi"] - c["f_lo"]) / nc
    for k, name in enumerate(names):
        a = MIXED_ARRAYS[name]
        s = seed * 7 + k
        enu = y_layout(a["n_ant"], a["extent_m"], s) if a["layout"] == "y" else disk_layout(a["n_ant"], a["extent_m"], s)
        cell = a["cell_arcsec"] * ARCSEC
        sky = sky_points(a["n_src"], a["src_radius_arcmin"] * ARCMIN, a["n_img"], cell, c["flux"], s)
        out[name] = MixedArray(
            name=name, enu_m=enu, freq_hz=freq.astype(np.float64), sky=sky, image=sky_image(sky, a["n_img"], cell),
            cell_rad=cell, n_grid=a["n_img"] * a["pad"], support=c["support"], oversample=c["oversample"],
            ap_kind=c["ap_kind"], diam_m=a["diam_m"], alpha_per_dlambda=ALPHA_PER_DLAMBDA_DISK,
            decorrelation=c["decorrelation"], sigma_noise=c["noise_jy"], lat_rad=c["lat_deg"] * DEG,
            dec_rad=c["dec_deg"] * DEG)
    return out


def mixed_intervals(arrays: dict, n_intervals: int = 256, seed: int = 0, t_range=(30, 600),
                    sigma_range_arcsec=(10.0, 60.0), outlier_frac: float = 0.05,
                    outlier_arcsec: float = 120.0) -> list:
    """Intervals of uneven length on arrays drawn uniformly from ``arrays``:
    n_time ~ U{t_range}, a start hour angle U(-4 h, 4 h - length), offsets
    Gaussian with sigma ~ U(sigma_range) per interval, and each antenna with
    probability ``outlier_frac`` an outlier of ``outlier_arcsec`` in a random
    direction instead."""
    rng = _rng(seed, 50)
    names = list(arrays)
    dt = MIXED_COMMON["dt_s"]
    out = []
    for k in range(n_intervals):
        name = names[int(rng.integers(len(names)))]
        n_ant = arrays[name].n_ant
        nt = int(rng.integers(t_range[0], t_range[1] + 1))
        span_h = nt * dt / 3600.0
        h0 = rng.uniform(-4.0, 4.0 - span_h)
        ha = (h0 + np.arange(nt) * dt / 3600.0) * 15.0 * DEG
        sig = rng.uniform(*sigma_range_arcsec) * ARCSEC
        lm = rng.normal(0.0, sig, (n_ant, 2))
        out_mask = rng.uniform(0.0, 1.0, n_ant) < outlier_frac
        th = rng.uniform(0.0, 2.0 * math.pi, n_ant)
        lm[out_mask, 0] = outlier_arcsec * ARCSEC * np.cos(th[out_mask])
        lm[out_mask, 1] = outlier_arcsec * ARCSEC * np.sin(th[out_mask])
        out.append(MixedInterval(array=name, hour_angles=ha, lm_true=lm, sigma_pt=sig,
                                 outliers=np.nonzero(out_mask)[0], noise_seed=int(seed) * 100003 + k))
    return out


def mixed_uvw(arr: MixedArray, iv: MixedInterval) -> np.ndarray:
    return uvw_tracks(arr.enu_m, arr.lat_rad, arr.dec_rad, iv.hour_angles)

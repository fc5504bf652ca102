"""ctypes binding of ``libpsc.so`` (declared in ``include/psc.h``).

Argument marshalling only: every step of the Pointing SelfCal path runs in
the CUDA library.  Device buffers are passed as torch CUDA tensors (or raw
integer device addresses); host buffers as numpy arrays.  Functions carry the
C names and raise ``PscError`` on any status other than ``PSC_OK``.  There is
no CPU fallback: if the library cannot be loaded the import-time ``lib()``
call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PSC_OK, PSC_ERR_ARG, PSC_ERR_CUDA, PSC_ERR_OOM = 0, 1, 2, 3
PSC_ERR_NOT_CONVERGED, PSC_ERR_TIMEOUT, PSC_ERR_NUMERIC, PSC_ERR_DEVICE = 4, 5, 6, 7
PSC_AP_DISK, PSC_AP_GAUSS, PSC_AP_TABLE = 0, 1, 2
PSC_GRID_F32, PSC_GRID_BF16 = 0, 1
PSC_STAGE_AUTO, PSC_STAGE_NEVER = 0, 1
PSC_KERNEL_GAUSS, PSC_KERNEL_EXACT_DISK = 0, 1
PSC_ORDER_BASELINE, PSC_ORDER_UV = 0, 1
PSC_LM_FULL, PSC_LM_BLOCK = 0, 1
STOP_REASONS = {0: "none", 1: "step", 2: "chi2", 3: "lambda", 4: "max_iter", 5: "numeric"}

EXPORTS = ("psc_solve_opts_default", "psc_model_grid", "psc_model_grid_components", "psc_snapshot_plane",
           "psc_snapshot_components", "psc_wstack_components", "psc_wstack_range", "psc_model_grid_wstack",
           "psc_set_wstack", "psc_create", "psc_destroy", "psc_last_error",
           "psc_predict", "psc_residual_grad", "psc_solve_offsets", "psc_lm_begin", "psc_lm_iterate",
           "psc_lm_end", "psc_lm_restart", "psc_set_tiling", "psc_set_grid_precision", "psc_set_staging",
           "psc_set_kernel_model", "psc_set_flat_tiling", "psc_set_track_tiling", "psc_set_wait_limit",
           "psc_get_wait_limit", "psc_features_batch", "psc_features_batch_work", "psc_predict_dev", "psc_uvw", "psc_set_brick_order", "psc_fp32_fma_rate", "psc_profile", "psc_profile_read",
           "psc_residual_grad_noalloc", "psc_batch_create", "psc_batch_destroy", "psc_batch_last_error",
           "psc_batch_autotune", "psc_batch_begin", "psc_batch_restart", "psc_batch_kernel", "psc_batch_iterate", "psc_batch_end",
           "psc_solve_batch", "psc_batch_profile", "psc_batch_profile_read", "psc_features",
           "psc_mlp_n_params", "psc_mlp_create", "psc_mlp_destroy", "psc_mlp_set_params", "psc_mlp_get_params",
           "psc_mlp_forward", "psc_mlp_grad", "psc_mlp_train_step", "psc_mlp_infer_offsets", "psc_learned_init")


class PscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("psc status %d: %s" % (status, msg))
        self.status = status


class psc_grid_desc(ctypes.Structure):
    _fields_ = [("n_img", ctypes.c_int), ("n_grid", ctypes.c_int), ("cell_rad", ctypes.c_double),
                ("support", ctypes.c_int), ("oversample", ctypes.c_int)]


class psc_aperture(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("diam_m", ctypes.c_double), ("alpha_per_dlambda", ctypes.c_double),
                ("decorrelation", ctypes.c_int), ("table", ctypes.POINTER(ctypes.c_double)),
                ("table_len", ctypes.c_int)]


def make_aperture(ap_kind, diam_m, alpha_per_dlambda, decorrelation=1, table=None):
    """psc_aperture for "disk", "gauss" or "table" (table: the caller's radial
    A° samples, see PSC_AP_TABLE); returns (struct, the array it points at)."""
    kind = {"disk": PSC_AP_DISK, "gauss": PSC_AP_GAUSS, "table": PSC_AP_TABLE}.get(ap_kind, ap_kind)
    tab = None
    ap = psc_aperture(int(kind), float(diam_m), float(alpha_per_dlambda), int(decorrelation), None, 0)
    if table is not None:
        tab = np.ascontiguousarray(table, dtype=np.float64)
        ap.table = tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        ap.table_len = int(tab.size)
    return ap, tab


class psc_obs(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("n_time", ctypes.c_int), ("n_chan", ctypes.c_int),
                ("uvw_dev", ctypes.c_void_p), ("freq_hz", ctypes.POINTER(ctypes.c_double))]


class psc_solve_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("mode", ctypes.c_int), ("lam0", ctypes.c_double),
                ("lam_max", ctypes.c_double), ("lam_min", ctypes.c_double), ("step_tol_rad", ctypes.c_double),
                ("chi2_rtol", ctypes.c_double), ("block_gain", ctypes.c_double)]


class psc_solve_report(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int), ("n_eval", ctypes.c_int), ("reason", ctypes.c_int),
                ("chi2", ctypes.c_double), ("lam", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_V = ctypes.c_void_p


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "psc_solve_opts_default": (None, [ctypes.POINTER(psc_solve_opts)]),
            "psc_model_grid": (ctypes.c_int, [ctypes.POINTER(psc_grid_desc), _V, _V, _V]),
            "psc_model_grid_components": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_int, ctypes.c_double, _V, _V]),
            "psc_snapshot_plane": (ctypes.c_int, [_V, ctypes.c_longlong, _D, _D, _V]),
            "psc_snapshot_components": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                                       ctypes.POINTER(psc_aperture), ctypes.c_double, _D]),
            "psc_wstack_components": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                                     ctypes.POINTER(psc_aperture), ctypes.c_double, _D]),
            "psc_wstack_range": (ctypes.c_int, [_V, ctypes.c_longlong, ctypes.c_double, ctypes.c_double, _D, _D, _V]),
            "psc_model_grid_wstack": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                     ctypes.c_double, ctypes.c_double, _V, _V]),
            "psc_set_wstack": (ctypes.c_int, [_V, _V, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double]),
            "psc_create": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.POINTER(psc_obs), ctypes.POINTER(psc_aperture),
                                          ctypes.POINTER(psc_grid_desc), _V, _V]),
            "psc_destroy": (None, [_V]),
            "psc_last_error": (ctypes.c_char_p, [_V]),
            "psc_predict": (ctypes.c_int, [_V, _D, _V, _V]),
            "psc_residual_grad": (ctypes.c_int, [_V, _D, _V, _V, ctypes.c_double, _D, _D, _D, _D]),
            "psc_solve_offsets": (ctypes.c_int, [_V, _V, _V, ctypes.c_double, ctypes.POINTER(psc_solve_opts), _D,
                                                 ctypes.POINTER(psc_solve_report)]),
            "psc_lm_begin": (ctypes.c_int, [_V, _D, ctypes.POINTER(psc_solve_opts)]),
            "psc_lm_iterate": (ctypes.c_int, [_V, _V, _V, ctypes.c_double, ctypes.c_int]),
            "psc_lm_end": (ctypes.c_int, [_V, _D, ctypes.POINTER(psc_solve_report)]),
            "psc_lm_restart": (ctypes.c_int, [_V]),
            "psc_set_tiling": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "psc_set_grid_precision": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_set_staging": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_set_kernel_model": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_set_flat_tiling": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int]),
            "psc_set_brick_order": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_fp32_fma_rate": (ctypes.c_int, [_D, _V]),
            "psc_profile": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_profile_read": (ctypes.c_int, [_V, _D, ctypes.POINTER(ctypes.c_int)]),
            "psc_residual_grad_noalloc": (ctypes.c_int, [ctypes.POINTER(psc_obs), ctypes.POINTER(psc_aperture),
                                                         ctypes.POINTER(psc_grid_desc), _V, _D, _V, _V, ctypes.c_double,
                                                         _D, _D, _D, _D, _V]),
            "psc_batch_create": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.POINTER(_V), ctypes.c_int,
                                                ctypes.POINTER(_V), ctypes.POINTER(_V), _D, _V]),
            "psc_batch_destroy": (None, [_V]),
            "psc_batch_last_error": (ctypes.c_char_p, [_V]),
            "psc_batch_autotune": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int)]),
            "psc_batch_begin": (ctypes.c_int, [_V, _D, ctypes.POINTER(psc_solve_opts)]),
            "psc_batch_restart": (ctypes.c_int, [_V]),
            "psc_batch_kernel": (ctypes.c_char_p, [_V]),
            "psc_set_track_tiling": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_set_wait_limit": (ctypes.c_int, [ctypes.c_longlong]),
            "psc_get_wait_limit": (ctypes.c_longlong, []),
            "psc_features_batch": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, ctypes.POINTER(_V),
                                                  ctypes.POINTER(_V), _D, ctypes.c_double, ctypes.c_int, _V,
                                                  ctypes.c_size_t, _V, _V]),
            "psc_predict_dev": (ctypes.c_int, [_V, _V, _V, _V]),
            "psc_uvw": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _V, _V]),
            "psc_features_batch_work": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_int,
                                                       ctypes.POINTER(ctypes.c_size_t)]),
            "psc_batch_iterate": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_batch_end": (ctypes.c_int, [_V, _D, ctypes.POINTER(psc_solve_report)]),
            "psc_mlp_n_params": (ctypes.c_int, []),
            "psc_mlp_create": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, _V]),
            "psc_mlp_destroy": (None, [_V]),
            "psc_mlp_set_params": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_float)]),
            "psc_mlp_get_params": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_float)]),
            "psc_mlp_forward": (ctypes.c_int, [_V, _V, ctypes.c_int, _V]),
            "psc_mlp_grad": (ctypes.c_int, [_V, _V, _V, ctypes.c_int, ctypes.POINTER(ctypes.c_float), _D]),
            "psc_mlp_train_step": (ctypes.c_int, [_V, _V, _V, ctypes.c_int, ctypes.c_double, _D]),
            "psc_mlp_infer_offsets": (ctypes.c_int, [_V, _V, ctypes.c_int, ctypes.c_double, _D]),
            "psc_learned_init": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]),
            "psc_features": (ctypes.c_int, [_V, _V, _V, ctypes.c_double, ctypes.c_double, ctypes.c_int, _V]),
            "psc_batch_profile": (ctypes.c_int, [_V, ctypes.c_int]),
            "psc_batch_profile_read": (ctypes.c_int, [_V, _D, ctypes.POINTER(ctypes.c_int)]),
            "psc_solve_batch": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, ctypes.POINTER(_V),
                                               ctypes.POINTER(_V), _D, ctypes.POINTER(psc_solve_opts), _D,
                                               ctypes.POINTER(psc_solve_report)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Device address of a torch tensor (or an int address, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _dp(a):
    return a.ctypes.data_as(_D)


def _check(st, ctx=None):
    if st != PSC_OK:
        msg = lib().psc_last_error(ctx)
        raise PscError(st, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def psc_set_wait_limit(polls):
    """Polls of one bounded mbarrier wait of the track kernel (< 0: default;
    0: every wait gives up at once, for testing the error path)."""
    _check(lib().psc_set_wait_limit(int(polls)))


def psc_get_wait_limit():
    return int(lib().psc_get_wait_limit())


def psc_uvw(ant_enu_m, lat_rad, dec_rad, ha_rad, uvw_out, stream=None):
    """Baseline coordinates into uvw_out (device float64 [n_time][n_bl][3])."""
    enu = np.ascontiguousarray(ant_enu_m, dtype=np.float64)
    ha = np.ascontiguousarray(np.atleast_1d(ha_rad), dtype=np.float64)
    n_ant = enu.shape[0]
    if enu.shape != (n_ant, 3):
        raise ValueError("ant_enu_m must be [n_ant][3]")
    need = ha.size * (n_ant * (n_ant - 1) // 2) * 3
    if uvw_out.numel() < need:
        raise ValueError("uvw_out holds %d values; %d needed" % (uvw_out.numel(), need))
    _check(lib().psc_uvw(int(n_ant), _dp(enu), float(lat_rad), float(dec_rad), int(ha.size), _dp(ha), _ptr(uvw_out),
                         _stream(stream)))
    return uvw_out


def psc_solve_opts_default() -> psc_solve_opts:
    o = psc_solve_opts()
    lib().psc_solve_opts_default(ctypes.byref(o))
    return o


def psc_model_grid(n_img, n_grid, cell_rad, support, oversample, image_dev, grid_out, stream=None):
    gd = psc_grid_desc(n_img, n_grid, cell_rad, support, oversample)
    _check(lib().psc_model_grid(ctypes.byref(gd), _ptr(image_dev), _ptr(grid_out), _stream(stream)))


def psc_model_grid_components(comp_lmS, n_grid, cell_rad, grid_out, stream=None):
    """V° of point components (host array [n][3] = l, m, S) into grid_out."""
    comp = np.ascontiguousarray(comp_lmS, dtype=np.float64).reshape(-1, 3)
    _check(lib().psc_model_grid_components(comp.shape[0], _dp(comp), int(n_grid), float(cell_rad), _ptr(grid_out),
                                           _stream(stream)))


def psc_snapshot_plane(uvw_dev, n_rows, stream=None):
    """(a, b) of the least-squares plane w = a u + b v of n_rows device uvw rows."""
    a = np.zeros(1)
    b = np.zeros(1)
    _check(lib().psc_snapshot_plane(_ptr(uvw_dev), int(n_rows), _dp(a), _dp(b), _stream(stream)))
    return float(a[0]), float(b[0])


def psc_snapshot_components(comp_lmS, a, b, ap_kind, diam_m, alpha_per_dlambda, freq_hz):
    """Components moved to the snapshot frame of plane (a, b), fluxes rescaled
    by the beam ratio at freq_hz (host [n][3] in, new array out)."""
    comp = np.ascontiguousarray(comp_lmS, dtype=np.float64).reshape(-1, 3)
    out = np.empty_like(comp)
    ap, _tab = make_aperture(ap_kind, diam_m, alpha_per_dlambda, 1)
    _check(lib().psc_snapshot_components(comp.shape[0], _dp(comp), float(a), float(b), ctypes.byref(ap),
                                         float(freq_hz), _dp(out)))
    return out


def psc_wstack_components(comp_lmS, a, b, ap_kind, diam_m, alpha_per_dlambda, freq_hz):
    """(l', m', S', n - 1) per component (host [n][3] true l, m, S in, [n][4] out)."""
    comp = np.ascontiguousarray(comp_lmS, dtype=np.float64).reshape(-1, 3)
    out = np.empty((comp.shape[0], 4))
    ap, _tab = make_aperture(ap_kind, diam_m, alpha_per_dlambda, 1)
    _check(lib().psc_wstack_components(comp.shape[0], _dp(comp), float(a), float(b), ctypes.byref(ap),
                                       float(freq_hz), _dp(out)))
    return out


def psc_wstack_range(uvw_dev, n_rows, a, b, stream=None):
    """(least, greatest) w - a u - b v in metres over n_rows device uvw rows."""
    lo = np.zeros(1)
    hi = np.zeros(1)
    _check(lib().psc_wstack_range(_ptr(uvw_dev), int(n_rows), float(a), float(b), _dp(lo), _dp(hi), _stream(stream)))
    return float(lo[0]), float(hi[0])


def psc_model_grid_wstack(comp_lmSn, n_grid, cell_rad, n_planes, w0, dw, grids_out, stream=None):
    """The n_planes grids of a residual-w stack (components [n][4]) into grids_out."""
    comp = np.ascontiguousarray(comp_lmSn, dtype=np.float64).reshape(-1, 4)
    _check(lib().psc_model_grid_wstack(comp.shape[0], _dp(comp), int(n_grid), float(cell_rad), int(n_planes),
                                       float(w0), float(dw), _ptr(grids_out), _stream(stream)))


def psc_residual_grad_noalloc(n_ant, n_time, n_chan, uvw_dev, freq_hz, ap_kind, diam_m, alpha_per_dlambda,
                              decorrelation, n_img, n_grid, cell_rad, support, oversample, grid_dev, lm, vis_obs,
                              w=None, w_scale=1.0, cross=False, stream=None, ap_table=None):
    """Allocation-free fused evaluation (no psc_ctx; scratch in the
    library's static device array).  Returns (chi2, g, H[, X]).

    Device tensors are checked against the problem's sizes before the call,
    so a short buffer raises here instead of being read past its end."""
    freq = np.ascontiguousarray(freq_hz, dtype=np.float64)
    n_ant, n_time, n_chan = int(n_ant), int(n_time), int(n_chan)
    n_vis = n_time * (n_ant * (n_ant - 1) // 2) * n_chan
    if freq.shape != (n_chan,):
        raise ValueError("freq_hz must hold n_chan values")
    if np.shape(lm) != (n_ant, 2):
        raise ValueError("lm must be [n_ant][2]")
    for name, x, need in (("uvw_dev", uvw_dev, 3 * n_vis // max(n_chan, 1)), ("vis_obs", vis_obs, n_vis),
                          ("w", w, n_vis), ("grid_dev", grid_dev, int(n_grid) ** 2)):
        if x is not None and not isinstance(x, int) and x.numel() < need:
            raise ValueError("%s holds %d elements; the problem needs %d" % (name, x.numel(), need))
    obs = psc_obs(int(n_ant), int(n_time), int(n_chan), _ptr(uvw_dev), _dp(freq))
    ap, _tab = make_aperture(ap_kind, diam_m, alpha_per_dlambda, decorrelation, ap_table)
    gd = psc_grid_desc(int(n_img), int(n_grid), float(cell_rad), int(support), int(oversample))
    lm = np.ascontiguousarray(lm, dtype=np.float64)
    n_bl = int(n_ant) * (int(n_ant) - 1) // 2
    chi2 = np.zeros(1)
    g = np.zeros((int(n_ant), 2))
    H = np.zeros((int(n_ant), 3))
    X = np.zeros((n_bl, 4)) if cross else None
    _check(lib().psc_residual_grad_noalloc(ctypes.byref(obs), ctypes.byref(ap), ctypes.byref(gd), _ptr(grid_dev),
                                           _dp(lm), _ptr(vis_obs), _ptr(w), float(w_scale), _dp(chi2), _dp(g),
                                           _dp(H), _dp(X) if cross else None, _stream(stream)))
    return (float(chi2[0]), g, H, X) if cross else (float(chi2[0]), g, H)


class Context:
    """Owns one ``psc_ctx``; ``uvw_dev`` and ``grid_dev`` must outlive it."""

    def __init__(self, n_ant, n_time, n_chan, uvw_dev, freq_hz, ap_kind, diam_m, alpha_per_dlambda,
                 decorrelation, n_img, n_grid, cell_rad, support, oversample, grid_dev, stream=None, ap_table=None):
        self._keep = (uvw_dev, grid_dev)
        self.n_ant, self.n_time, self.n_chan = int(n_ant), int(n_time), int(n_chan)
        self.n_bl = self.n_ant * (self.n_ant - 1) // 2
        self._freq = np.ascontiguousarray(freq_hz, dtype=np.float64)
        obs = psc_obs(self.n_ant, self.n_time, self.n_chan, _ptr(uvw_dev), _dp(self._freq))
        ap, _tab = make_aperture(ap_kind, diam_m, alpha_per_dlambda, decorrelation, ap_table)
        gd = psc_grid_desc(int(n_img), int(n_grid), float(cell_rad), int(support), int(oversample))
        h = _V()
        _check(lib().psc_create(ctypes.byref(h), ctypes.byref(obs), ctypes.byref(ap), ctypes.byref(gd),
                                _ptr(grid_dev), _stream(stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().psc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _lm(self, lm):
        lm = np.ascontiguousarray(lm, dtype=np.float64)
        if lm.shape != (self.n_ant, 2):
            raise ValueError("lm must be [n_ant][2]")
        return lm

    def psc_set_tiling(self, t_tile=0, c_group=0, vis_per_thread=0):
        _check(lib().psc_set_tiling(self.h, int(t_tile), int(c_group), int(vis_per_thread)), self.h)

    def psc_set_staging(self, mode):
        _check(lib().psc_set_staging(self.h, int(mode)), self.h)

    def psc_set_brick_order(self, order):
        _check(lib().psc_set_brick_order(self.h, int(order)), self.h)

    def psc_set_flat_tiling(self, items, vis_per_thread):
        _check(lib().psc_set_flat_tiling(self.h, int(items), int(vis_per_thread)), self.h)

    def psc_set_track_tiling(self, vis_per_lane):
        _check(lib().psc_set_track_tiling(self.h, int(vis_per_lane)), self.h)

    def psc_set_kernel_model(self, model):
        _check(lib().psc_set_kernel_model(self.h, int(model)), self.h)

    def psc_set_grid_precision(self, precision):
        _check(lib().psc_set_grid_precision(self.h, int(precision)), self.h)

    def psc_set_wstack(self, grids, n_planes, w0=0.0, dw=1.0, a=0.0, b=0.0):
        """Degrid from a residual-w stack (n_planes = 0: the context's own grid)."""
        _check(lib().psc_set_wstack(self.h, _ptr(grids), int(n_planes), float(w0), float(dw), float(a), float(b)),
               self.h)
        self._wstack = grids if n_planes else None          # borrowed: keep it alive

    def psc_predict(self, lm, vis_out, dvis_out=None):
        lm = self._lm(lm)
        _check(lib().psc_predict(self.h, _dp(lm), _ptr(vis_out), _ptr(dvis_out)), self.h)

    def psc_predict_dev(self, lm_dev, vis_out, dvis_out=None):
        """psc_predict with device offsets (float64 [n_ant][2]); enqueued, no synchronisation."""
        _check(lib().psc_predict_dev(self.h, _ptr(lm_dev), _ptr(vis_out), _ptr(dvis_out)), self.h)

    def psc_residual_grad(self, lm, vis_obs, w=None, w_scale=1.0, cross=False):
        lm = self._lm(lm)
        chi2 = np.zeros(1)
        g = np.zeros((self.n_ant, 2))
        H = np.zeros((self.n_ant, 3))
        X = np.zeros((self.n_bl, 4)) if cross else None
        _check(lib().psc_residual_grad(self.h, _dp(lm), _ptr(vis_obs), _ptr(w), float(w_scale), _dp(chi2), _dp(g),
                                       _dp(H), _dp(X) if cross else None), self.h)
        return (float(chi2[0]), g, H, X) if cross else (float(chi2[0]), g, H)

    def psc_solve_offsets(self, vis_obs, w=None, w_scale=1.0, lm0=None, opts=None):
        lm = self._lm(np.zeros((self.n_ant, 2)) if lm0 is None else lm0).copy()
        rep = psc_solve_report()
        _check(lib().psc_solve_offsets(self.h, _ptr(vis_obs), _ptr(w), float(w_scale),
                                       ctypes.byref(opts) if opts is not None else None, _dp(lm),
                                       ctypes.byref(rep)), self.h)
        return lm, rep

    def psc_lm_begin(self, lm0, opts=None):
        self._lm0 = self._lm(lm0)
        _check(lib().psc_lm_begin(self.h, _dp(self._lm0), ctypes.byref(opts) if opts is not None else None), self.h)

    def psc_lm_iterate(self, vis_obs, w=None, w_scale=1.0, n_iter=1):
        _check(lib().psc_lm_iterate(self.h, _ptr(vis_obs), _ptr(w), float(w_scale), int(n_iter)), self.h)

    def psc_features(self, vis_obs, w=None, w_scale=1.0, sigma_prior=30.0 * 4.84813681109536e-06, time_stride=1,
                     out=None):
        """Features [n_ant][52] (torch float32 on the device of vis_obs)."""
        import torch
        if out is None:
            out = torch.empty((self.n_ant, 52), dtype=torch.float32, device=vis_obs.device)
        _check(lib().psc_features(self.h, _ptr(vis_obs), _ptr(w), float(w_scale), float(sigma_prior),
                                  int(time_stride), _ptr(out)), self.h)
        return out

    def psc_learned_init(self, mlp, vis_obs, w=None, w_scale=1.0, sigma_prior=30.0 * 4.84813681109536e-06,
                         time_stride=1):
        lm = np.zeros((self.n_ant, 2))
        _check(lib().psc_learned_init(self.h, mlp.h, _ptr(vis_obs), _ptr(w), float(w_scale), float(sigma_prior),
                                      int(time_stride), _dp(lm)), self.h)
        return lm

    def psc_lm_restart(self):
        _check(lib().psc_lm_restart(self.h), self.h)

    def psc_profile(self, enable=True):
        _check(lib().psc_profile(self.h, int(bool(enable))), self.h)

    def psc_profile_read(self):
        ms = np.zeros(1)
        n = ctypes.c_int(0)
        _check(lib().psc_profile_read(self.h, _dp(ms), ctypes.byref(n)), self.h)
        return float(ms[0]), int(n.value)

    def psc_lm_end(self):
        lm = np.zeros((self.n_ant, 2))
        rep = psc_solve_report()
        _check(lib().psc_lm_end(self.h, _dp(lm), ctypes.byref(rep)), self.h)
        return lm, rep


def _ptr_array(items):
    arr = (_V * len(items))()
    for k, x in enumerate(items):
        arr[k] = _ptr(x)
    return arr


def _bcheck(st, b):
    if st != PSC_OK:
        msg = lib().psc_batch_last_error(b)
        raise PscError(st, msg.decode() if msg else "")


class Batch:
    """Owns one ``psc_batch`` over ``contexts`` (``Context`` objects) and their
    per-context observed data; all of them must outlive the batch."""

    def __init__(self, contexts, vis_obs, w=None, w_scale=None, stream=None):
        self.contexts = list(contexts)
        n = len(self.contexts)
        self._keep = (list(vis_obs), list(w) if w is not None else None)
        hs = (_V * n)(*[c.h.value for c in self.contexts])
        self._hs = hs
        ws = np.ascontiguousarray(np.ones(n) if w_scale is None else w_scale, dtype=np.float64)
        self._ws = ws
        h = _V()
        _bcheck(lib().psc_batch_create(ctypes.byref(h), hs, n, _ptr_array(vis_obs),
                                       _ptr_array(w) if w is not None else None, _dp(ws), _stream(stream)), None)
        self.h = h
        self.n_ant = [c.n_ant for c in self.contexts]

    def close(self):
        if getattr(self, "h", None):
            lib().psc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _concat(self, lm_list):
        return np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in lm_list]))

    def _split(self, flat):
        out, off = [], 0
        for n in self.n_ant:
            out.append(flat[off:off + 2 * n].reshape(n, 2))
            off += 2 * n
        return out

    def psc_batch_autotune(self):
        """Chosen (t_tile, c_group, vis_per_thread, staging mode) of every context."""
        t = (ctypes.c_int * (4 * len(self.contexts)))()
        _bcheck(lib().psc_batch_autotune(self.h, t), self.h)
        return [tuple(t[4 * k:4 * k + 4]) for k in range(len(self.contexts))]

    def psc_batch_begin(self, lm0_list, opts=None):
        self._lm0 = self._concat(lm0_list)
        _bcheck(lib().psc_batch_begin(self.h, _dp(self._lm0), ctypes.byref(opts) if opts is not None else None),
                self.h)

    def psc_batch_kernel(self):
        """Name of the fused kernel the batch's persistent launch runs."""
        return lib().psc_batch_kernel(self.h).decode()

    def psc_batch_restart(self):
        _bcheck(lib().psc_batch_restart(self.h), self.h)

    def psc_batch_iterate(self, n_iter=1):
        _bcheck(lib().psc_batch_iterate(self.h, int(n_iter)), self.h)

    def psc_batch_profile(self, enable=True):
        _bcheck(lib().psc_batch_profile(self.h, int(bool(enable))), self.h)

    def psc_batch_profile_read(self):
        ms = np.zeros(1)
        n = ctypes.c_int(0)
        _bcheck(lib().psc_batch_profile_read(self.h, _dp(ms), ctypes.byref(n)), self.h)
        return float(ms[0]), int(n.value)

    def psc_batch_end(self):
        flat = np.zeros(2 * sum(self.n_ant))
        reps = (psc_solve_report * len(self.contexts))()
        _bcheck(lib().psc_batch_end(self.h, _dp(flat), reps), self.h)
        return self._split(flat), list(reps)


def psc_fp32_fma_rate(stream=None):
    """Measured FP32 FMA throughput of the device (TFLOP/s)."""
    out = np.zeros(1)
    _check(lib().psc_fp32_fma_rate(_dp(out), _stream(stream)))
    return float(out[0])


def psc_features_batch_work(contexts, time_stride):
    """Workspace bytes of psc_features_batch for these contexts (one per pair)."""
    n = len(contexts)
    hs = (_V * n)(*[c.h.value for c in contexts])
    b = ctypes.c_size_t(0)
    _check(lib().psc_features_batch_work(hs, n, int(time_stride), ctypes.byref(b)))
    return int(b.value)


def psc_features_batch(contexts, vis_obs, w_scale, sigma_prior, time_stride, work, out, w=None, stream=None):
    """Features of every (context, data) pair into out (device float32
    [sum n_ant][52]); work: device scratch of psc_features_batch_work bytes."""
    n = len(contexts)
    hs = (_V * n)(*[c.h.value for c in contexts])
    ws = np.ascontiguousarray(np.broadcast_to(np.asarray(w_scale, dtype=np.float64), (n,)))
    need = sum(c.n_ant for c in contexts) * 52
    if out.numel() < need or out.dtype != torch_float32():
        raise ValueError("out must be float32 with at least %d elements" % need)
    _check(lib().psc_features_batch(hs, n, _ptr_array(vis_obs), _ptr_array(w) if w is not None else None, _dp(ws),
                                    float(sigma_prior), int(time_stride), _ptr(work), int(work.numel() * work.element_size()),
                                    _ptr(out), _stream(stream)))
    return out


def torch_float32():
    import torch
    return torch.float32


def psc_solve_batch(contexts, vis_obs, w=None, w_scale=None, lm0_list=None, opts=None):
    """Solves all contexts in one batch; returns (list of lm, list of reports)."""
    n = len(contexts)
    hs = (_V * n)(*[c.h.value for c in contexts])
    n_ant = [c.n_ant for c in contexts]
    if lm0_list is None:
        lm0_list = [np.zeros((a, 2)) for a in n_ant]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in lm0_list]))
    ws = np.ascontiguousarray(np.ones(n) if w_scale is None else w_scale, dtype=np.float64)
    reps = (psc_solve_report * n)()
    _check(lib().psc_solve_batch(hs, n, _ptr_array(vis_obs), _ptr_array(w) if w is not None else None, _dp(ws),
                                 ctypes.byref(opts) if opts is not None else None, _dp(flat), reps))
    out, off = [], 0
    for a in n_ant:
        out.append(flat[off:off + 2 * a].reshape(a, 2))
        off += 2 * a
    return out, list(reps)


class Mlp:
    """Owns one ``psc_mlp`` (the learned initial estimate's network)."""

    def __init__(self, max_batch, stream=None):
        h = _V()
        _check(lib().psc_mlp_create(ctypes.byref(h), int(max_batch), _stream(stream)))
        self.h = h
        self.n_params = lib().psc_mlp_n_params()
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "h", None):
            lib().psc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def psc_mlp_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError("params must have %d entries" % self.n_params)
        _check(lib().psc_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def psc_mlp_get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().psc_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def psc_mlp_forward(self, x_dev, out=None):
        import torch
        B = x_dev.shape[0]
        if out is None:
            out = torch.empty((B, 2), dtype=torch.float32, device=x_dev.device)
        _check(lib().psc_mlp_forward(self.h, _ptr(x_dev), int(B), _ptr(out)))
        return out

    def psc_mlp_grad(self, x_dev, t_dev):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = np.zeros(1)
        _check(lib().psc_mlp_grad(self.h, _ptr(x_dev), _ptr(t_dev), int(x_dev.shape[0]),
                                  g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(loss)))
        return float(loss[0]), g

    def psc_mlp_train_step(self, x_dev, t_dev, lr, want_loss=False):
        loss = np.zeros(1)
        _check(lib().psc_mlp_train_step(self.h, _ptr(x_dev), _ptr(t_dev), int(x_dev.shape[0]), float(lr),
                                        _dp(loss) if want_loss else None))
        return float(loss[0]) if want_loss else None

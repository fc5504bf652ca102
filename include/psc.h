/*
 * psc.h -- Pointing SelfCal hot path on one NVIDIA GB300 (sm_103a): the C ABI.
 *
 * The library solves for antenna pointing offsets (l_i, m_i) of an aperture
 * synthesis array, following Bhatnagar & Cornwell 2017, "The Pointing Self
 * Calibration algorithm for aperture synthesis radio telescopes":
 *
 *   Algorithm 1      pre-compute V° = F[I^M] and A°, then iterate: degrid
 *                    V^M = A_ij * V° and grad V^M = grad A_ij * V°, form the
 *                    residuals, accumulate chi^2 and its gradient, update l_i.
 *   Eq. AIJPOINTING  A_ij = A° exp(-(l_i-l_j)^2 alpha^2/2) exp(i pi u (l_i+l_j))
 *   Eq. DAIJPOINTING dA_ij/dl_i = A_ij [(l_j - l_i) alpha^2 + i pi u]
 *                    (both extended to m the same way, Sec. 3)
 *   Eq. DCHIDD       d chi^2/d a_i = -2 sum_j Re(R_ij^dag W_ij grad_i V^M_ij)
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: offsets in radians, uvw in metres, frequencies in Hz.
 * Baselines: antenna pairs i < j in lexicographic order (0,1),(0,2),...,(1,2),...;
 *   n_bl = n_ant (n_ant - 1) / 2.  uvw of baseline (i, j) is x_j - x_i.
 * Visibilities: complex64 (interleaved float re, im), layout [n_time][n_bl][n_chan].
 * Image / grid: image pixel (row, col) is at l = (col - N/2) cell,
 *   m = (row - N/2) cell; grid cell (gy, gx) at u = (gx - Ng/2) du,
 *   v = (gy - Ng/2) du, du = 1 / (Ng cell).  Fourier sign exp(+2 pi i), Eq. ME.
 * Parameter vectors: lm[n_ant][2] = (l_a, m_a); gradient grad[n_ant][2];
 *   normal blocks normal[n_ant][3] = (H_ll, H_lm, H_mm) of antenna a;
 *   cross blocks cross[n_bl][4] = (H_{l_i l_j}, H_{l_i m_j}, H_{m_i l_j}, H_{m_i m_j}).
 *   H_pq = 2 sum w Re(conj(dV/dp) dV/dq) (Gauss-Newton); chi^2 = sum w |R|^2
 *   over the measured baselines i < j.
 * Memory: "device" pointers are CUDA global memory of the current device and
 *   "host" pointers are ordinary host memory; the caller owns every buffer it
 *   passes.  A psc_ctx owns its internal workspace and frees it in psc_destroy.
 * Streams: work is enqueued on the stream given to psc_create (a cudaStream_t
 *   passed as void*, NULL = legacy default stream).  Calls that return host
 *   results synchronise that stream before returning; psc_lm_iterate does not.
 * Errors: every call returns a psc_status and never throws or aborts; the
 *   message of the last failure is available from psc_last_error().  Device
 *   side failures (a non-finite chi^2 or LM step) are reported as
 *   PSC_ERR_NUMERIC by the next synchronising call.
 * Threads: a psc_ctx must not be used by two host threads at once.
 */
#ifndef PSC_H
#define PSC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSC_OK = 0,
    PSC_ERR_ARG = 1,            /* an argument is NULL, out of range or inconsistent */
    PSC_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    PSC_ERR_OOM = 3,            /* device allocation failed */
    PSC_ERR_NOT_CONVERGED = 4,  /* reserved: a solve hit max_iter (reported in psc_solve_report) */
    PSC_ERR_TIMEOUT = 5,        /* reserved for bounded device waits */
    PSC_ERR_NUMERIC = 6,        /* non-finite chi^2 / normals in the solver */
    PSC_ERR_DEVICE = 7          /* a device-side consistency check failed */
} psc_status;

enum { PSC_AP_DISK = 0, PSC_AP_GAUSS = 1, PSC_AP_TABLE = 2 };
enum { PSC_GRID_F32 = 0, PSC_GRID_BF16 = 1 };
enum { PSC_STAGE_AUTO = 0, PSC_STAGE_NEVER = 1 };
enum { PSC_KERNEL_GAUSS = 0, PSC_KERNEL_EXACT_DISK = 1 };
enum { PSC_ORDER_BASELINE = 0, PSC_ORDER_UV = 1 };
enum { PSC_LM_FULL = 0, PSC_LM_BLOCK = 1 };
enum { PSC_STOP_NONE = 0, PSC_STOP_STEP = 1, PSC_STOP_CHI2 = 2, PSC_STOP_LAMBDA = 3,
       PSC_STOP_MAX_ITER = 4, PSC_STOP_NUMERIC = 5 };

typedef struct psc_ctx psc_ctx;

/* Model grid and tap geometry (Algorithm 1 pre-computes; Eq. MEDD).
 * Tap window of a visibility at grid coordinate x = u/du + Ng/2:
 * x0 = floor(x) - S/2 + 1, taps x0 .. x0 + S - 1 (same for y); cells outside
 * [0, Ng) contribute nothing. */
typedef struct {
    int    n_img;        /* N: the model image is N x N (N even, 2..8192) */
    int    n_grid;       /* Ng: padded grid size (even, N <= Ng <= 16384) */
    double cell_rad;     /* image pixel size (rad) */
    int    support;      /* S: taps per axis (even, 2..64) */
    int    oversample;   /* radial table samples per grid cell (1..64; 20 is the usual) */
} psc_grid_desc;

/* A-priori aperture kernel A° (Sec. 3: the pre-computed, pointing-free part
 * of A_ij) for a homogeneous array of circularly symmetric antennas.
 *   PSC_AP_DISK : uniform disk of diameter diam_m; A° is the disk's
 *                 autocorrelation over its area squared (transform of the
 *                 Airy power beam, integral 1).
 *   PSC_AP_GAUSS: Gaussian voltage pattern exp(-alpha^2 rho^2) (Sec. 3);
 *                 A°(q) = (pi / 2 alpha^2) exp(-pi^2 q^2 / (2 alpha^2)).
 *   PSC_AP_TABLE: a caller's radial A° (Sec. 3 and Alg. 1's second
 *                 pre-compute: A° may carry a-priori primary-beam effects,
 *                 such as a tapered illumination or blockage), given on the
 *                 scale of the dish: table[k] = A°(q) D_lambda^2 at
 *                 q / D_lambda = k / (table_len - 1), k = 0 .. table_len - 1,
 *                 linear between samples, A° = 0 from q = D_lambda on (an
 *                 aperture's autocorrelation ends at one diameter).  The
 *                 samples are used as given: 2 pi int_0^1 T(x) x dx is the
 *                 beam's PB(0) (1 for a normalised beam).  For the uniform
 *                 disk T(x) = (8 / pi^2) (acos x - x sqrt(1 - x^2)).
 * alpha = alpha_per_dlambda * diam_m * nu / c at every channel.  For the disk,
 * alpha only enters the decorrelation factor (1.1442341... matches the Airy
 * half-power width).  A° is applied through a radial table at `oversample`
 * samples per cell, linearly interpolated:
 *   t = rho*ov, n = floor(t), f = t - n, A° = (1-f) tab[n] + f tab[n+1]
 *   if n + 1 < len, else 0;  tab[n] = A°(n du / ov) du^2,
 *   len = floor(ov * rho_max) + 2, rho_max = D_lambda/du (disk, table), (S/2)sqrt(2) (Gaussian).
 * psc_create copies the table (the caller's array may be freed after it). */
typedef struct {
    int    kind;               /* PSC_AP_DISK, PSC_AP_GAUSS or PSC_AP_TABLE */
    double diam_m;             /* aperture diameter (m), > 0 */
    double alpha_per_dlambda;  /* alpha / D_lambda, > 0 */
    int    decorrelation;      /* 1: keep exp(-alpha^2 |p_i - p_j|^2 / 2) of Eq. AIJPOINTING; 0: drop it */
    const double *table;       /* PSC_AP_TABLE: host [table_len], finite; otherwise unused (NULL) */
    int    table_len;          /* PSC_AP_TABLE: 2 .. 65536 */
} psc_aperture;

/* One block of observation (normally one solution interval, Algorithm 1's
 * (tau_sol, dnu_sol)).  uvw_dev is borrowed for the lifetime of the ctx and
 * must not change: psc_create also keeps a copy of (u, v) split into FP32
 * high and low parts (16 bytes per time and baseline), which the fused
 * kernel reads instead of FP64. */
typedef struct {
    int           n_ant;     /* 2..512 */
    int           n_time;    /* >= 1 */
    int           n_chan;    /* 1..4096 */
    const double *uvw_dev;   /* device [n_time][n_bl][3] (m) */
    const double *freq_hz;   /* host [n_chan] (Hz), > 0 */
} psc_obs;

/* Levenberg-Marquardt options: f() and Terminate() of Algorithm 1, left to
 * the minimiser by the paper (Sec. 2.2).  Damped system
 * (H + lam diag(H)) delta = -g over all 2 n_ant parameters (PSC_LM_FULL) or
 * per antenna with step scaled by block_gain (PSC_LM_BLOCK).  A trial that
 * lowers chi^2 is accepted (lam /= 10, floored at lam_min), else rejected
 * (lam *= 10).  Stops: max |delta| < step_tol_rad; a rejected trial whose
 * step max |delta| was below 10 step_tol_rad (reason PSC_STOP_STEP: the minimum
 * is found to within that, and raising lam would only shrink the step to the
 * tolerance); an accepted relative chi^2 decrease < chi2_rtol; lam > lam_max;
 * max_iter iterations. */
typedef struct {
    int    max_iter;       /* 50 */
    int    mode;           /* PSC_LM_FULL */
    double lam0;           /* 1e-3 */
    double lam_max;        /* 1e10 */
    double lam_min;        /* 1e-12 */
    double step_tol_rad;   /* 1e-4 arcsec */
    double chi2_rtol;      /* 1e-10 */
    double block_gain;     /* 0.5 */
} psc_solve_opts;

typedef struct {
    int    n_iter;         /* iterations taken */
    int    n_eval;         /* fused evaluations (= n_iter + 1 unless stopped on a step) */
    int    reason;         /* PSC_STOP_* */
    double chi2;           /* chi^2 at the returned offsets */
    double lam;            /* final damping */
} psc_solve_report;

/* Fills *opts with the defaults listed above. */
void psc_solve_opts_default(psc_solve_opts *opts);

/* Observation geometry: the baseline coordinates (u, v, w) of Eq. ME, in
 * metres, from antenna positions.  ant_enu_m: host [n_ant][3] (east, north,
 * up, metres) in the horizon frame at latitude lat_rad; the phase centre at
 * declination dec_rad; ha_rad: host [n_time] hour angles (local sidereal time
 * minus right ascension).  Writes uvw_out (device, caller-owned,
 * [n_time][n_bl][3] float64) with b_ij = x_j - x_i for the baselines in the
 * order (0,1), (0,2), ..., (1,2), ..., u east, v north, w towards the phase
 * centre -- the layout psc_obs.uvw_dev takes.  FP64.  Synchronises.  Errors:
 * PSC_ERR_ARG (sizes, NULL or non-finite inputs), PSC_ERR_CUDA. */
psc_status psc_uvw(int n_ant, const double *ant_enu_m, double lat_rad, double dec_rad, int n_time, const double *ha_rad,
                   void *uvw_out, void *stream);

/* V° = F[I^M] (Algorithm 1, first pre-compute): the unnormalised DFT of the
 * image zero-padded to Ng x Ng, G[gy][gx] = sum I[row][col]
 * exp(+2 pi i ((gx-Ng/2)(col-N/2) + (gy-Ng/2)(row-N/2)) / Ng).
 * image_dev: device float [N][N]; grid_out: device complex64 [Ng][Ng];
 * stream: cudaStream_t or NULL.  For N % 8 == 0 the two matrix products run
 * on the tensor cores in split bfloat16 (each FP32 operand as three bfloat16
 * parts, FP32 accumulation; error at FP32 rounding level; operands staged by
 * TMA) and need a temporary workspace of 6 N K + 24 Ng K bytes, K = N rounded
 * up to a multiple of 32; otherwise FP32 SIMT with a temporary complex64
 * [N][Ng].  Synchronises the stream before freeing the
 * workspace and returning; PSC_ERR_TIMEOUT if a tensor-core wait ran out. */
psc_status psc_model_grid(const psc_grid_desc *gd, const float *image_dev, void *grid_out,
                          void *stream);

/* V° of a model given as n_comp point components (comp_lmS: host
 * [n_comp][3] = l, m (radians), S (Jy)): G[gy][gx] = sum_k S_k
 * exp(+2 pi i ((gx-Ng/2) du l_k + (gy-Ng/2) du m_k)), du = 1 / (n_grid
 * cell_rad) -- for sources at pixel centres the same grid as psc_model_grid
 * of their image.  One complex matrix product on the tensor cores (split
 * bfloat16 as psc_model_grid; operands from FP64 sincospi; the component
 * count padded to a multiple of 32 with zero flux).  grid_out: device
 * complex64 [n_grid][n_grid].  Temporary workspace of 24 n_grid K bytes, K
 * the padded count.  Synchronises.  Errors: PSC_ERR_ARG (sizes, NULL or
 * non-finite input), PSC_ERR_CUDA / PSC_ERR_OOM, PSC_ERR_TIMEOUT (a
 * tensor-core wait ran out). */
psc_status psc_model_grid_components(int n_comp, const double *comp_lmS, int n_grid, double cell_rad,
                                     void *grid_out, void *stream);

/* W-snapshots (Sec. 6.1: for short solution intervals the array may be
 * treated as co-planar).  psc_snapshot_plane fits the plane w = a u + b v to
 * n_rows baselines (uvw_dev: device double [n_rows][3], metres) by least
 * squares (FP64 sums on the GPU, 2 x 2 solve on the host); synchronises;
 * PSC_ERR_NUMERIC when the (u, v) are collinear.
 * psc_snapshot_components moves each component (host [n_comp][3] = l, m, S)
 * to the snapshot frame of that plane, l' = l + a (n-1), m' = m + b (n-1),
 * n = sqrt(1 - l^2 - m^2), where the co-planar degridding reproduces the
 * w-term exactly for baselines on the plane, and rescales its flux by
 * PB(l) / PB(l'), PB the aperture's pointing-free power pattern at freq_hz
 * (the degridding kernel weights a source by the beam at its grid position);
 * comp_out may equal comp_in.  Feed the result to psc_model_grid_components
 * and give each interval's context its own grid.  What the method neglects is
 * the interval's departure w - a u - b v from the plane, and the beam ratio's
 * change across the band away from freq_hz.  Errors: PSC_ERR_ARG (NULL,
 * aperture, a component outside the unit disk), PSC_ERR_NUMERIC (a moved
 * component on a beam null). */
psc_status psc_snapshot_plane(const double *uvw_dev, long long n_rows, double *a, double *b, void *stream);
psc_status psc_snapshot_components(int n_comp, const double *comp_in, double a, double b, const psc_aperture *ap,
                                   double freq_hz, double *comp_out);

/* Residual w of long intervals (Sec. 6.1 and the conclusions: an array that is
 * not co-planar over a solution interval makes the w-term cost; W-snapshots
 * remove the plane, these calls the rest).  After the plane fit each
 * visibility keeps w_r = (w - a u - b v) nu / c wavelengths of w, which
 * multiplies component k by exp(2 pi i w_r (n_k - 1)), n_k from its true
 * direction.  The model grid becomes a stack of n_planes grids at
 * w_p = w0 + p dw (wavelengths): plane p is the grid of the snapshot-frame
 * components with fluxes S'_k exp(2 pi i w_p (n_k - 1)).  A visibility
 * degrids (1 - f) G_p + f G_{p+1} with q = (w_r - w0) / dw,
 * p = min(floor(q), n_planes - 2), f = q - p: linear interpolation in w of
 * each source's w-phase, in error by at most (2 pi |n_k - 1| dw)^2 / 8 of its
 * flux.  The pointing derivatives keep their form (the w-phase belongs to the
 * sky, not to the antennas).
 *
 * psc_wstack_components (host): comp_in [n_comp][3] = (l, m, S) at their true
 * directions -> comp_out [n_comp][4] = (l', m', S', n - 1): the result of
 * psc_snapshot_components plus n - 1.  The arrays must not overlap.  Errors as
 * psc_snapshot_components.
 * psc_wstack_range: the least and greatest w - a u - b v (metres) over n_rows
 * baselines of uvw_dev (device double [n_rows][3]); scale by the lowest and
 * highest nu / c to size a stack.  Synchronises.  PSC_ERR_NUMERIC for
 * non-finite uvw.
 * psc_model_grid_wstack: the n_planes (>= 2) grids, each as
 * psc_model_grid_components with the plane's complex fluxes, into grids_out
 * (device complex64 [n_planes][n_grid][n_grid], caller-owned).  Temporary
 * workspace as psc_model_grid_components.  Synchronises.  Errors as
 * psc_model_grid_components, plus PSC_ERR_ARG for n_planes or dw.
 * psc_set_wstack: the context degrids from the stack (borrowed like the grid of
 * psc_create, planes [n_planes][Ng][Ng] of the context's grid size) instead of
 * its grid, for every evaluation (predict, residual_grad, the solvers);
 * n_planes = 0 returns to its grid.  It checks on the GPU that the stack
 * covers the residual w of every baseline, time and channel of the context,
 * and refuses with PSC_ERR_ARG otherwise (the message gives both ranges).
 * Taps then read two planes each from global memory (the grid is never
 * staged).  Gaussian kernel model and FP32 grid only: this call refuses a
 * context with the exact kernel or the BF16 grid copy, psc_set_kernel_model
 * and psc_set_grid_precision refuse those while a stack is set.  A batch
 * takes either only stacked contexts (its persistent launch then runs the
 * stacked kernel) or none.  psc_features reads the context's own grid.
 * Synchronises. */
psc_status psc_wstack_components(int n_comp, const double *comp_in, double a, double b, const psc_aperture *ap,
                                 double freq_hz, double *comp_out);
psc_status psc_wstack_range(const double *uvw_dev, long long n_rows, double a, double b, double *wmin_m,
                            double *wmax_m, void *stream);
psc_status psc_model_grid_wstack(int n_comp, const double *comp_lmSn, int n_grid, double cell_rad, int n_planes,
                                 double w0, double dw, void *grids_out, void *stream);
psc_status psc_set_wstack(psc_ctx *ctx, const void *grids, int n_planes, double w0, double dw, double a, double b);

/* Creates a context for one observation block: copies the channel list,
 * builds the A° tables on the device (Algorithm 1, second pre-compute) and
 * allocates the workspace.  grid_dev (complex64 [Ng][Ng], from
 * psc_model_grid or the caller) is borrowed, like obs->uvw_dev; several
 * contexts may share one grid.  On failure *out is NULL. */
psc_status psc_create(psc_ctx **out, const psc_obs *obs, const psc_aperture *ap,
                      const psc_grid_desc *gd, const void *grid_dev, void *stream);

/* Frees the context's workspace.  NULL is ignored. */
void psc_destroy(psc_ctx *ctx);

/* Message of the last failure on ctx (or of the last failed psc_create /
 * psc_model_grid when ctx is NULL).  Valid until the next call on ctx. */
const char *psc_last_error(const psc_ctx *ctx);

/* Model visibilities at offsets lm (host [n_ant][2]) -- Algorithm 1's
 * V^M_ij = A_ij * V° and grad_i V^M_ij = grad_i A_ij * V°.
 * vis_out: device complex64 [n_time][n_bl][n_chan].
 * dvis_out: NULL, or device complex64 [4][n_time][n_bl][n_chan] holding
 * dV/dl_i, dV/dm_i, dV/dl_j, dV/dm_j of each baseline (i, j).  Synchronises. */
psc_status psc_predict(psc_ctx *ctx, const double *lm, void *vis_out, void *dvis_out);

/* psc_predict with the offsets in device memory (lm_dev, [n_ant][2] radians,
 * read by the kernel) and without synchronising: the launch is only
 * enqueued on the context's stream, so that a caller simulating many
 * intervals (one set of offsets each) pays no host round trip per interval.
 * lm_dev must stay valid until the launch has run. */
psc_status psc_predict_dev(psc_ctx *ctx, const double *lm_dev, void *vis_out, void *dvis_out);

/* One fused evaluation at offsets lm (host [n_ant][2]) of the residuals
 * R = V^Obs - V^M, chi^2 (Eq. Chisq), the gradient (Eq. DCHIDD) and the
 * Gauss-Newton normal blocks.  vis_obs: device complex64 [n_time][n_bl][n_chan];
 * w: device float weights of the same shape, or NULL for all ones; each
 * weight is multiplied by w_scale (> 0).  Outputs are host buffers: chi2 (1),
 * grad [n_ant][2], normal [n_ant][3], cross [n_bl][4] (NULL to skip).
 * Synchronises. */
psc_status psc_residual_grad(psc_ctx *ctx, const double *lm, const void *vis_obs, const float *w,
                             double w_scale, double *chi2, double *grad, double *normal,
                             double *cross);

/* Solves for the offsets (Algorithm 1's iteration loop, LM as described at
 * psc_solve_opts), starting from lm_inout (host [n_ant][2]) and writing the
 * solution back there.  opts NULL = defaults; rep may be NULL.  All
 * iterations run on the device; synchronises once at the end. */
psc_status psc_solve_offsets(psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale,
                             const psc_solve_opts *opts, double *lm_inout, psc_solve_report *rep);

/* The solve split into device-resident steps, for callers that pipeline or
 * time the loop: psc_lm_begin uploads lm0 (host [n_ant][2]) and resets the
 * solver state (no synchronisation); psc_lm_iterate enqueues n_iter
 * iterations -- one fused evaluation and one LM update each; iterations after
 * a stop are skipped on the device -- without synchronising; psc_lm_end
 * synchronises and copies out the current offsets (host [n_ant][2]) and report
 * (either may be NULL). */
psc_status psc_lm_begin(psc_ctx *ctx, const double *lm0, const psc_solve_opts *opts);
psc_status psc_lm_iterate(psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale,
                          int n_iter);
psc_status psc_lm_end(psc_ctx *ctx, double *lm_out, psc_solve_report *rep);

/* Resets the solver to the start given by the last psc_lm_begin (offsets,
 * options, damping) with one device kernel, no host transfer and no
 * synchronisation, so that a pipelined caller can run many solves from the
 * same start.  Fails with PSC_ERR_ARG if psc_lm_begin was never called. */
psc_status psc_lm_restart(psc_ctx *ctx);

/* Launch-shape knobs of the fused kernel; 0 keeps the current value.  A
 * thread block holds c_group channels and, per channel, t_tile threads that
 * each own vis_per_thread visibilities at consecutive time steps (a block
 * covers t_tile * vis_per_thread time steps; its size is t_tile * c_group
 * rounded up to a multiple of 32).  t_tile in [1, 256], c_group in [1, 8],
 * t_tile * c_group <= 256, vis_per_thread in {1, 2}.  vis_per_thread = 2
 * shares each staged grid cell between the thread's two visibilities; it is
 * refused (PSC_ERR_ARG) unless every channel's aperture lies inside the
 * S x S tap window and consecutive time steps move a baseline by at most 4
 * grid cells at the highest frequency.  Results do not depend on the shape
 * beyond FP32 summation order. */
psc_status psc_set_tiling(psc_ctx *ctx, int t_tile, int c_group, int vis_per_thread);

/* Flat bricks: the fused kernel's work items of a baseline are its (channel,
 * group of vis_per_thread consecutive time steps) pairs in channel-major
 * order, and a thread block takes `items` consecutive ones (one per thread),
 * so only the baseline's last block has idle lanes -- unlike the (t_tile x
 * c_group) blocks of psc_set_tiling, which idle whole warps when t_tile *
 * c_group falls short of a multiple of 32 and when the channel or time count
 * is not a multiple of the group.  A block may then span several channels
 * (at most 8).  items in {32, 64, ..., 256}; vis_per_thread as for
 * psc_set_tiling.  psc_set_tiling switches back.  Under PSC_KERNEL_EXACT_DISK
 * vis_per_thread must be 1 (psc_set_kernel_model resets the shape to
 * rectangular bricks; set flat bricks after it).  Errors:
 * PSC_ERR_ARG for out-of-range values or a brick spanning more than 8
 * channels (fewer time steps per channel than items / 7). */
psc_status psc_set_flat_tiling(psc_ctx *ctx, int items, int vis_per_thread);

/* Track kernel (Alg. 1's inner loop, Eqs. AIJPOINTING, DAIJPOINTING, Chisq,
 * DCHIDD; the same arithmetic as the brick kernel, for small apertures of a
 * few to a few tens of taps per visibility).  vis_per_lane in {1, 2} makes
 * every later reduce-mode evaluation of ctx (psc_residual_grad, the solver,
 * batches) run one warp per (baseline, 32 x vis_per_lane consecutive time
 * steps) that loops over all channels; each channel's grid box (the cells
 * within the aperture of the warp's visibilities, at most 32 cells wide and
 * 512 cells in all) and A° table are copied into shared memory by TMA
 * (cp.async.bulk.tensor) one channel ahead, and the cell half of the phase
 * ramp is applied there.  Boxes beyond that size read the grid from global
 * memory instead.  chi^2 and the gradient are summed with compensated FP32
 * (TwoSum) per lane and across the warp, then in FP64.  Predictions
 * (psc_predict) keep the brick kernel.  0 switches back to the brick kernel;
 * so do psc_set_tiling, psc_set_flat_tiling, psc_set_kernel_model,
 * psc_set_grid_precision(PSC_GRID_BF16) and psc_set_wstack.  The first call
 * with vis_per_lane > 0 builds the tensor maps of the grid and per-channel
 * tables (a few KB; synchronises the stream).  Errors: PSC_ERR_ARG when the
 * context uses the exact kernel, a residual-w stack or the BF16 grid copy, a
 * grid not 16-byte aligned, an aperture reaching outside the S x S window,
 * or (vis_per_lane 2) consecutive time steps more than 4 cells apart.
 * Results equal the brick kernel's up to FP32 summation order. */
psc_status psc_set_track_tiling(psc_ctx *ctx, int vis_per_lane);

/* Polls of one bounded mbarrier wait of the track kernel (psc_set_track_tiling),
 * each poll suspending the warp for up to about a microsecond.  A wait that
 * runs out makes the warp record a flag, wait with a fixed larger bound for
 * its own copies still in flight and stop; the synchronising call that
 * consumes the evaluation (psc_residual_grad, psc_lm_end, psc_solve_offsets,
 * psc_batch_end, psc_solve_batch) then reports PSC_ERR_TIMEOUT, and the
 * context stays usable.  polls < 0 restores the default (2^24, far beyond any
 * wait that completes); 0 makes every wait give up at once, which exercises
 * that error path.  The limit is process-wide and read when a launch is
 * enqueued (batches capture it in their graph: recreate the batch after a
 * change).  The model-grid and network kernels keep their own fixed bound.
 * psc_get_wait_limit returns the current value.  Never fails. */
psc_status psc_set_wait_limit(long long polls);
long long psc_get_wait_limit(void);

/* Measured FP32 FMA throughput of the current device (TFLOP/s, an FMA counted
 * as 2 flops): eight independent FMA chains per thread on 8 blocks of 256
 * threads per SM, timed with CUDA events.  A check of the FP32 peak that the
 * fused kernel's roofline divides by.  Synchronises.  Errors: PSC_ERR_ARG,
 * PSC_ERR_CUDA (psc_last_error(NULL)). */
psc_status psc_fp32_fma_rate(double *tflops, void *stream);

/* Grid access of the fused kernel.  PSC_STAGE_AUTO (default): a thread
 * block copies the grid cells its visibilities touch (with the per-cell half
 * of the pointing ramp applied) into shared memory when they fit a 64 x 64
 * tile, else reads them from global memory.  PSC_STAGE_NEVER: always read
 * from global memory (pays off for small apertures and long baselines, where
 * a brick's visibilities share few cells).  Results are the same up to FP32
 * summation order.  Errors: PSC_ERR_ARG for an unknown mode. */
psc_status psc_set_staging(psc_ctx *ctx, int mode);

/* Launch order of the fused kernel's bricks.  PSC_ORDER_BASELINE: baselines
 * in (i, j) order.  PSC_ORDER_UV: baselines in Morton (Z-curve) order of
 * their (u, v) at the interval's middle time step, so that the bricks running
 * together read nearby grid cells (L2 reuse when the grid is larger than L2).
 * psc_create picks PSC_ORDER_UV for grids of more than 128 MB, else
 * PSC_ORDER_BASELINE.  Results are identical: each brick's partial sums keep
 * their place, and the reductions run in the same order.  Used by the
 * Gaussian-model kernel (single launches and batches).  Errors: PSC_ERR_ARG. */
psc_status psc_set_brick_order(psc_ctx *ctx, int order);

/* Aperture kernel model of psc_predict, psc_residual_grad, psc_lm_* and
 * psc_solve_offsets on this context.
 *
 * PSC_KERNEL_GAUSS (default): Eq. AIJPOINTING -- A° times the Gaussian
 * decorrelation factor exp(-alpha^2 |l_i - l_j|^2 / 2) (dropped when the
 * aperture's decorrelation is 0) times the phase ramp exp(i pi du.(l_i+l_j)).
 *
 * PSC_KERNEL_EXACT_DISK (uniform-disk apertures only): the exact transform of
 * the product of the two antennas' disk patterns, each shifted by its offset
 * (Sec. 3: a more accurate pattern in place of the Gaussian main lobe):
 *   A_ij(du) = exp(i pi du.(l_i + l_j)) O(du; l_i - l_j) / (pi R^2)^2,
 *   O = integral of cos(2 pi w.(l_i - l_j)) over the lens where the two
 *       apertures of radius R = D_lambda / 2, centred du apart, overlap,
 * with its exact derivatives.  At l_i = l_j it equals A° times the ramp.  The
 * GPU evaluates O by its Taylor series in (2 pi w.(l_i - l_j)) up to the 6th
 * power, from per-channel lens moments computed once (FP64 quadrature) by this
 * call: with x = pi D_lambda |l_i - l_j| the relative truncation error is at
 * most x^8/8! for O and x^6/(7!/8) for its derivative (1e-7 at x = 0.3, i.e.
 * 2 arcmin of offset difference for a 25 m dish at 1.5 GHz), growing fast
 * beyond x = 1.  It runs one visibility per thread (the tiling's
 * vis_per_thread becomes 1; psc_set_tiling refuses 2), reads the FP32 grid
 * (not the BF16 copy) and the FP64 uvw.  Batches (psc_batch_create,
 * psc_solve_batch) refuse contexts in this mode; psc_features and the
 * learned initialiser keep the Gaussian model.
 *
 * Errors: PSC_ERR_ARG (unknown model, non-disk aperture, aperture table too
 * long for shared memory), PSC_ERR_CUDA / PSC_ERR_OOM (moment tables). */
psc_status psc_set_kernel_model(psc_ctx *ctx, int model);

/* Storage precision of the model grid V° that the fused evaluation reads
 * (psc_predict, psc_residual_grad, the solvers and batches; the feature pass
 * of psc_features always reads the FP32 grid).  PSC_GRID_F32 (default) reads
 * the caller's complex64 grid.  PSC_GRID_BF16 takes a copy of that grid
 * with both parts rounded to bfloat16 (nearest even), owned by the context
 * (n_grid^2 * 4 bytes), and reads it instead; all arithmetic stays FP32 with
 * FP64 sums as before.  The copy is taken at this call: call again after the
 * caller's grid changes.  Errors: PSC_ERR_ARG for an unknown precision,
 * PSC_ERR_OOM / PSC_ERR_CUDA.  Synchronises. */
psc_status psc_set_grid_precision(psc_ctx *ctx, int precision);

/* Input features of the learned initial estimate (an addition to the
 * paper's method: the paper starts the minimiser from zero or from previous
 * solutions).  For each antenna i, 52 floats in feat_dev (device
 * [n_ant][52]), all from the time steps t with t % time_stride == 0:
 *   [0..1]   the block Newton step -H_ii^{-1} g_i at zero offsets (Eq. DCHIDD
 *            gradient, Gauss-Newton 2x2 block), divided by sigma_prior_rad;
 *   [2..26]  A_i(s) = sum w Re(conj(V_obs) V_s) / sum w |V_s|^2,
 *   [27..51] C_i(s) = (chi2_i(delta_s) - chi2_i(0)) / sum w |V_0|^2,
 * for the 25 trial offsets delta_s = sigma_prior_rad (a, b), a, b = -2..2
 * (row-major over b, then a; a moves l, b moves m), applied to antenna i
 * alone, with V_s the model of Eq. AIJPOINTING and sums over the baselines
 * of i.  One strided pass of one kernel.  Asynchronous (enqueued on the
 * context's stream). */
psc_status psc_features(psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale, double sigma_prior_rad,
                        int time_stride, float *feat_dev);

/* The features of psc_features for n (context, data) pairs in three launches
 * (one stencil pass over all pairs' bricks, the per-baseline sums, the
 * per-antenna features).  A context may appear in several pairs (for example
 * one context per observation geometry serving many simulated intervals).
 * vis_obs[j] / w[j] (NULL for all ones; w itself may be NULL) / w_scale[j]
 * (NULL for 1) are pair j's data as for psc_features; the features of pair j
 * go to feat_dev (device) from row sum_{i<j} n_ant_i, [n_ant_j][52] each.
 * Every pair needs the same brick shape: contexts of the same number of time
 * steps and channels.  work is caller-owned device scratch of at least the
 * bytes psc_features_batch_work reports for the same contexts and stride
 * (the argument tables, then per pair 56 * 8 bytes per brick and per
 * baseline).  Runs on `stream` and synchronises it (the argument tables are
 * copied from host memory).  Errors: PSC_ERR_ARG (NULL pointers, a workspace
 * that is too small, mixed brick shapes), PSC_ERR_CUDA. */
psc_status psc_features_batch(psc_ctx *const *ctxs, int n, const void *const *vis_obs, const float *const *w,
                              const double *w_scale, double sigma_prior_rad, int time_stride, void *work,
                              size_t work_bytes, float *feat_dev, void *stream);
psc_status psc_features_batch_work(psc_ctx *const *ctxs, int n, int time_stride, size_t *bytes);

/* ---- The learned initial estimate's network (an addition to the method) ----
 * MLP 52 -> 256 -> 256 -> 256 -> 2 with GELU after the hidden layers, input
 * standardised by fixed (mu, s), output the offsets in units of sigma_prior.
 * Flat FP32 parameter vector of psc_mlp_n_params() floats:
 *   W1 [52][256], b1 [256], W2 [256][256], b2 [256], W3 [256][256], b3 [256],
 *   W4 [256][2], b4 [2], mu [52], s [52]   (y = x W + b; W stored [in][out]).
 * GEMM operands are bfloat16 on the tensor cores with FP32 accumulation;
 * master weights, biases and AdamW state are FP32.  The caller draws the
 * initial weights and sets them with psc_mlp_set_params (which also clears
 * the AdamW state).  Loss: (1/B) sum_b sum_o (y_bo - t_bo)^2.
 * x_dev [batch][52], t_dev and y_dev [batch][2] are device FP32; batch is
 * 1..max_batch.  All calls enqueue on the stream given to psc_mlp_create;
 * those with host outputs synchronise it.  The GEMMs run on the tensor cores
 * (tcgen05.mma); if one gives up waiting for its MMAs (a bounded wait), the
 * next synchronising call returns PSC_ERR_TIMEOUT.  Errors: psc_last_error(NULL). */
typedef struct psc_mlp psc_mlp;
int psc_mlp_n_params(void);
psc_status psc_mlp_create(psc_mlp **out, int max_batch, void *stream);
void psc_mlp_destroy(psc_mlp *m);
psc_status psc_mlp_set_params(psc_mlp *m, const float *params);     /* host [n_params] */
psc_status psc_mlp_get_params(psc_mlp *m, float *params);           /* host [n_params] */
psc_status psc_mlp_forward(psc_mlp *m, const float *x_dev, int batch, float *y_dev);
/* Gradient of the loss at the current parameters (no update): grad_host
 * [n_params] (zero for mu and s) and loss, either NULL to skip. */
psc_status psc_mlp_grad(psc_mlp *m, const float *x_dev, const float *t_dev, int batch, float *grad_host,
                        double *loss);
/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, weight decay 1e-4, learning
 * rate lr) on the trained parameters; loss (before the step) if non-NULL. */
psc_status psc_mlp_train_step(psc_mlp *m, const float *x_dev, const float *t_dev, int batch, double lr,
                              double *loss);
/* Offsets (rad, host [n_ant][2]) from features feat_dev [n_ant][52]:
 * network output times sigma_prior_rad. */
psc_status psc_mlp_infer_offsets(psc_mlp *m, const float *feat_dev, int n_ant, double sigma_prior_rad,
                                 double *lm_out);
/* The learned initial estimate of a context: psc_features then
 * psc_mlp_infer_offsets (max_batch >= n_ant).  lm_out host [n_ant][2]. */
psc_status psc_learned_init(psc_ctx *ctx, psc_mlp *m, const void *vis_obs, const float *w, double w_scale,
                            double sigma_prior_rad, int time_stride, double *lm_out);

/* ---- Batches of solution intervals (Algorithm 1's loop over all data) ----
 * A batch groups contexts -- normally one per solution interval, of any
 * array, length and channel set -- with their observed data, so that one LM
 * iteration of all of them is one persistent fused launch: thread blocks pull
 * (baseline, channel group, time tile) bricks of every context from one
 * device work queue, so intervals of uneven size share the GPU.  The
 * reductions and the LM updates of all contexts follow as one launch each,
 * and the iteration is captured once in a CUDA graph and replayed (unless the
 * batch runs on the legacy NULL stream).  Contexts whose solver stopped skip
 * their bricks.  The persistent launch uses the block size of the widest
 * context's shape (t_tile * c_group rounded up to a multiple of 32); narrower
 * contexts leave the extra lanes idle.
 * The contexts must all use the Gaussian kernel model, and either all read
 * a residual-w stack (psc_set_wstack) or none; each context's settings are
 * read when the batch is created or autotuned (PSC_ERR_ARG otherwise).
 * vis_obs[k], w[k] (NULL = ones) and w_scale[k] (NULL = all 1) are the data
 * of ctxs[k], borrowed like the contexts for the batch's lifetime.  The
 * offsets of all contexts are concatenated in the order of ctxs: lm0,
 * lm_out, lm_inout are host [sum n_ant_k][2]; reps is [n_ctx]. */
typedef struct psc_batch psc_batch;

psc_status psc_batch_create(psc_batch **out, psc_ctx *const *ctxs, int n_ctx, const void *const *vis_obs,
                            const float *const *w, const double *w_scale, void *stream);
void psc_batch_destroy(psc_batch *b);
const char *psc_batch_last_error(const psc_batch *b);

/* Name of the fused kernel that the batch's persistent launch runs
 * ("eval_kernel<...>" for brick tilings, "track_kernel<kv>" when every
 * context has the track tiling).  Static storage; never NULL. */
const char *psc_batch_kernel(const psc_batch *b);

/* Picks each context's launch shape by timing the fused kernel on its own
 * data: for blocks of 128 and 256 threads and vis_per_thread 1 and (where
 * psc_set_tiling accepts it) 2, the three channel groups whose smallest
 * fitting time tile leaves the fewest lanes idle (ragged time and channel
 * tails count as idle), plus (32, 4, 1), plus flat bricks of 64, 128, 192
 * and 256 items (psc_set_flat_tiling); the fastest is kept, then contexts
 * narrower than the widest choice take their fastest shape of that width (one
 * block size serves the persistent launch); the winner is also timed with
 * PSC_STAGE_NEVER and the faster grid access kept.  Contexts of the same
 * array, channels and grid reuse the first one's choice, with the time tile
 * refitted to their own length (flat bricks need no refit).  The fused
 * kernel is then chosen on the whole batch: one persistent launch with these
 * brick shapes, and one with the track kernel (psc_set_track_tiling) for each
 * of 1 and 2 visibilities per lane that every context allows, each timed; the
 * fastest is kept.  Each context's trial offsets and solver state are saved
 * before those launches and restored after them.  Writes the chosen (t_tile,
 * c_group, vis_per_thread, staging mode) of context k to tiling_out[4k..4k+3]
 * (NULL to skip); flat
 * bricks are written as (items, 0, vis_per_thread, staging mode) and the
 * track tiling as (-1, 0, vis_per_lane, PSC_STAGE_AUTO).  Synchronises. */
psc_status psc_batch_autotune(psc_batch *b, int *tiling_out);

/* Start (host offsets, options as for psc_lm_begin), restart on the device,
 * n_iter device-resident iterations (graph replays, no synchronisation) and
 * the synchronising read-out, mirroring psc_lm_begin / psc_lm_restart /
 * psc_lm_iterate / psc_lm_end. */
psc_status psc_batch_begin(psc_batch *b, const double *lm0, const psc_solve_opts *opts);
psc_status psc_batch_restart(psc_batch *b);
psc_status psc_batch_iterate(psc_batch *b, int n_iter);
psc_status psc_batch_end(psc_batch *b, double *lm_out, psc_solve_report *reps);

/* Timing of the batch's persistent fused launch: while enabled,
 * psc_batch_iterate launches each iteration directly (not through the graph)
 * with a pair of CUDA events around the fused launch; psc_batch_profile_read
 * synchronises, returns the summed duration (ms) and count, and clears them. */
psc_status psc_batch_profile(psc_batch *b, int enable);
psc_status psc_batch_profile_read(psc_batch *b, double *total_ms, int *n_launches);

/* Solves every context in one batch (created and destroyed inside, on the
 * first context's stream) from lm_inout, writing the solutions back; stops
 * when every solver has stopped or after max_iter + 1 evaluations. */
psc_status psc_solve_batch(psc_ctx *const *ctxs, int n_ctx, const void *const *vis_obs, const float *const *w,
                           const double *w_scale, const psc_solve_opts *opts, double *lm_inout,
                           psc_solve_report *reps);

/* Allocation-free variant of psc_residual_grad.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- because their device memory belongs to another allocator (a
 * framework's caching pool, an arena sized once at start-up) or because they
 * run in a real-time loop where cudaMalloc / cudaFree, which can synchronise
 * the whole device, are not acceptable.  It needs no psc_ctx and allocates
 * no memory: its working memory (channel constants, A° tables, antenna
 * pairs, the FP32 split of the baseline coordinates, per-brick partial sums,
 * per-baseline sums, the packed result) lives in one file-scope device array
 * of 16 MiB that every GPU which loads the library holds until the process
 * exits.
 * Inputs and outputs are those of psc_create + psc_residual_grad: obs,
 * ap and gd as for psc_create; grid_dev device complex64 [Ng][Ng]; lm host
 * [n_ant][2]; vis_obs device complex64 [n_time][n_bl][n_chan]; w device float
 * of the same shape or NULL (all ones), scaled by w_scale > 0; outputs on the
 * host: chi2 (1), grad [n_ant][2], normal [n_ant][3], cross [n_bl][4] (NULL
 * to skip).  The fused kernel runs with t_tile 32, c_group 4, one visibility
 * per thread and staging on, on the same inputs as a context's, so the
 * results equal bit for bit those of psc_residual_grad with that tiling.
 * Limits: a problem whose scratch exceeds 16 MiB -- about 15 * 8 bytes per
 * (baseline, 4 channels, 32 time steps) brick plus 16 bytes per (time step,
 * baseline) plus the tables -- is rejected with PSC_ERR_ARG and a message
 * giving the size it needed; for example 351 baselines x 64 channels x 150
 * time steps needs about 4.4 MB.  Tables of 4 channels that do not fit the
 * fused kernel's shared memory are rejected with PSC_ERR_ARG too.  Both
 * checks come before any work is queued.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and raises the fused kernel's shared-memory limit,
 * with that device current; make that first call before any stream capture.
 * Every call shares the one array and overwrites what it reads, so nothing
 * needs clearing, but calls that overlap on the GPU (different streams or host
 * threads) race on it and must be serialised by the caller.  The call copies
 * lm from pageable host memory, runs on `stream` (cudaStream_t or NULL) and
 * returns after synchronising it, with the outputs on the host.
 * Errors are reported through psc_last_error(NULL). */
psc_status psc_residual_grad_noalloc(const psc_obs *obs, const psc_aperture *ap, const psc_grid_desc *gd,
                                     const void *grid_dev, const double *lm, const void *vis_obs,
                                     const float *w, double w_scale, double *chi2, double *grad,
                                     double *normal, double *cross, void *stream);

/* Timing of the fused evaluation kernel (the dominant launch of every
 * iteration).  psc_profile(ctx, 1) makes every later fused launch on ctx's
 * stream record a pair of CUDA events around it; psc_profile(ctx, 0) stops
 * recording.  psc_profile_read synchronises the stream, returns the summed
 * duration (ms) and count of the recorded launches, and clears the record.
 * This is instrumentation only; it does not change any result. */
psc_status psc_profile(psc_ctx *ctx, int enable);
psc_status psc_profile_read(psc_ctx *ctx, double *total_ms, int *n_launches);

#ifdef __cplusplus
}
#endif
#endif /* PSC_H */

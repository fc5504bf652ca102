// Internal declarations of the Pointing SelfCal CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "psc.h"

namespace psc {

constexpr double kC = 299792458.0;
constexpr int kTile = 64;          // staged grid tile: kTile x kTile complex64 cells
constexpr int kRed = 15;           // per-baseline sums: chi2, g_i(2), g_j(2), H_ii(3), H_jj(3), H_ij(4)
constexpr int kMaxThreads = 256;   // fused-kernel block size upper bound

// Per-channel constants, built once per context.
struct ChanConst {
    double uv_scale;   // nu / (c du): metres of baseline -> grid cells
    float sc_hi, sc_lo;  // uv_scale split into two floats (sc_hi + sc_lo = uv_scale to ~2^-48)
    float alpha2;      // alpha(nu)^2 (rad^-2)
    float rho_max;     // (len - 1) / ov: taps at rho >= rho_max (cells) get A° = 0
    int tab_off;       // first table entry (float2 units)
    int tab_len;       // len
};

// Arguments of the fused evaluation kernel (one launch covers one context).
struct EvalArgs {
    const double *uvw;         // [nt][nbl][3] metres
    const float4 *uvs;         // nullptr or [nt][nbl] (u_hi, u_lo, v_hi, v_lo) metres: the FP32 split of uvw, read instead
    const float2 *grid;        // [ng][ng] V° (complex64)
    const unsigned *grid_bf16; // nullptr or [ng][ng] V° as bfloat16 pairs (re in the low half), read instead
    const ChanConst *chan;     // [nc]
    const float2 *tabs;        // radial tables: (A°(n), A°(n+1) - A°(n)) pairs
    const int2 *pairs;         // [nbl] antenna (i, j)
    const double *lm;          // [n_ant][2] offsets of this evaluation
    const float2 *vis_obs;     // reduce mode: [nt][nbl][nc]
    const float *w;            // reduce mode: weights or nullptr (= 1)
    float w_scale;
    float2 *vis_out;           // predict mode: [nt][nbl][nc]
    float2 *dvis_out;          // predict mode: nullptr or [4][nt][nbl][nc]
    double *partials;          // reduce mode: [n_bricks][kRed]
    const int *skip;           // nullptr or device flag: nonzero = solver stopped, do nothing
    int n_bl, nt, nc, ng, support, ov;
    float du;                  // grid cell (wavelengths)
    int t_tile, c_group, n_tt, n_cg;   // n_tt = ceil(nt / (t_tile * kv))
    int kv;                    // visibilities per thread at consecutive times: 1 or 2
    int no_stage;              // 1: never stage the grid (taps read it from L1/L2)
    int decorrelation;
    int max_tab_len;           // longest table among the channels
    int tab_stride;            // staged entries per channel: max_tab_len + zero padding
    long long n_bricks;        // n_bl * n_cg * n_tt (partials are [kRed][n_bricks])
    const float *kmom;         // exact disk kernel: [table entries][10] lens-moment combinations
    int exact;                 // 1: exact disk kernel (exact.cu) instead of Eq. AIJPOINTING's
    // Flat bricks (flat > 0; t_tile, c_group, n_tt, n_cg unused): the items of a
    // baseline are its (channel, group of kv consecutive time steps) pairs in
    // channel-major order, n_tp groups per channel; brick b of the baseline
    // holds items [b flat, (b + 1) flat), so bpb bricks per baseline, each
    // spanning at most ch_span channels.
    int flat, n_tp, bpb, ch_span;
    // nullptr, or [n_bl]: the baseline of each group of bpb consecutive bricks in
    // launch order (partials stay indexed by baseline: brick = bl * bpb + j)
    const int *bl_order;
    // Residual-w stack (wp_n >= 2): grid holds wp_n planes of ng^2 cells.  A
    // visibility at q = (w - wp_a u - wp_b v) uv_scale wp_scale - wp_q0 (uvw in
    // metres, q clamped to [0, wp_n - 1]) reads (1 - f) plane p + f plane p + 1,
    // p = min(floor(q), wp_n - 2), f = q - p.  Taps read the planes unstaged.
    int wp_n;
    double wp_a, wp_b, wp_scale, wp_q0;
    // Track kernel (track.cu; trk_kv > 0, reduce mode only): one warp per item
    // (baseline, chunk of 32 trk_kv consecutive time steps), looping over the
    // channels; each channel's grid box and table are staged by TMA into the
    // warp's double buffer.  Partials are [kRed][n_bricks] with
    // n_bricks = n_bl trk_chunks (bpb = trk_chunks).
    int trk_kv;                // 0: brick kernel (eval_kernel); 1 or 2: visibilities per lane
    int trk_chunks;            // time chunks per baseline: ceil(nt / (32 trk_kv))
    int trk_cap;               // staged tile capacity of one buffer (cells)
    int trk_stride;            // entries per channel in tabs_cs (even)
    int trk_pad;               // zero entries past a channel's table that a lane can reach
    int trk_tabc;              // table capacity of a warp buffer (entries, multiple of 16): the longest copy
    float trk_spread;          // largest move of a baseline between consecutive time steps (cells, top channel)
    const float2 *tabs_cs;     // [nc][trk_stride]: (A°(n) - n s_n, s_n), s_n = A°(n+1) - A°(n), zero padded
    const void *tmap;          // 3 CUtensorMaps over the grid (8-byte cells), boxes 8, 16, 32 wide x 8 rows
    int *err;                  // device flag, set when a bounded wait ran out (the results are then invalid)
    long long wait_limit;      // polls of one bounded mbarrier wait
};

// Arguments of the stencil-feature kernel (learned initial estimate).
struct StencilArgs {
    const double *uvw;
    const float2 *grid;
    const ChanConst *chan;
    const float2 *tabs;
    const float2 *vis_obs;
    const float *w;
    float w_scale;
    double *partials;          // [56][n_bricks]
    int n_bl, nt, nc, ng, support, ov;
    float du;
    int t_tile, c_group, n_tt, n_cg, time_stride;   // n_tt counts the kept (strided) time steps
    int decorrelation;
    int max_tab_len;
    int stage;                 // 1: stage the grid cells of a brick in shared memory when they fit
    long long n_bricks;
    float sigma;               // stencil spacing (rad)
    int wpb;                   // 1: one brick per block; 4: bricks of one warp, four per block (shared tables)
};

// Per-pair outputs of a batched feature pass (psc_features_batch).
struct FeatPair {
    const double *partials;    // [56][n_bl * bpb]
    double *blsum;             // [n_bl][56]
    float *feat;               // [n_ant][52]
    int n_bl, bpb, n_ant;
};

// Arguments of the second-stage reductions of one context.
struct RedArgs {
    const double *partials;    // [kRed][n_bl * bpb]
    double *blsum;             // [n_bl][kRed]
    double *ev;                // chi2 | g[2n] | H[3n] | X[4 nbl]
    const int *skip;           // nullptr or the solver's stop flag
    int n_bl, bpb, n_ant;
};

// Solver state kept on the device between iterations.
struct LMState {
    int n_iter, n_eval, reason, done;
    double lam, chi2;
    // options
    int max_iter, mode;
    double lam_max, lam_min, step_tol, chi2_rtol, block_gain;
};

// Workspace pointers of the solver (device).
struct LMArgs {
    LMState *st;
    double *lm_cur;            // [n_ant][2] accepted offsets
    double *lm_trial;          // [n_ant][2] offsets of the next evaluation (EvalArgs::lm)
    const double *ev;          // evaluation at lm_trial: chi2 | g[2n] | H[3n] | X[4 nbl]
    double *cur;               // same layout, accepted evaluation
    double *mat;               // [2n][2n] scratch for the damped full system (large systems)
    float *mat32;              // [2n][2n] FP32 factor (large systems)
    double *rhs;               // [2n] scratch
    const int2 *pairs;
    int n_ant, n_bl;
    int *err;                  // the context's bounded-wait flag (read and cleared by psc_batch_end)
};

__host__ __device__ inline size_t ev_len(int n_ant, int n_bl) { return 1 + 2 * (size_t)n_ant + 3 * (size_t)n_ant + 4 * (size_t)n_bl; }

// Track kernel (track.cu): dynamic shared memory of one block for tile
// capacity cap and table capacity tabc (cells / entries per buffer), its
// attribute, occupancy, single-context and persistent launches, the per-channel
// (intercept, slope) tables and the grid's tensor maps (3 x 128 bytes, device).
constexpr int kTrkThreads = 128;
size_t track_dyn_smem(int cap, int tabc);
cudaError_t set_track_smem(size_t dyn);
cudaError_t track_occupancy(int kv, size_t dyn, int *blocks_per_sm);
cudaError_t launch_track(const EvalArgs &a, cudaStream_t s);
cudaError_t launch_track_batch(const EvalArgs *args_dev, const long long *prefix_dev, int n_ctx,
                               unsigned long long *queue, int kv, int cap, int tabc, int grid, cudaStream_t s);
cudaError_t launch_track_tables(const ChanConst *chan, const float2 *tabs, int nc, int stride, float2 *out,
                                cudaStream_t s);
cudaError_t make_grid_maps(const float2 *grid, int ng, void *maps_dev, cudaStream_t s);
// Polls of a bounded mbarrier wait (the default unless psc_set_wait_limit changed it).
long long wait_limit();

// Baseline coordinates [n_time][n_bl][3] (m) from antenna positions (device
// [n_ant][3] east, north, up) and hour angles (device [n_time]).
cudaError_t launch_uvw(const double *enu_dev, int n_ant, double lat, double dec, const double *ha_dev, int n_time,
                       double *uvw_dev, cudaStream_t s);

// Launchers (defined in the .cu files).
cudaError_t launch_eval(const EvalArgs &a, bool predict, cudaStream_t s);
// Persistent fused launch over several contexts (device arrays of EvalArgs and
// first-brick prefixes [n_ctx + 1]; *queue must be zero at launch).  stacked:
// every context reads a residual-w stack (else none does).
cudaError_t launch_eval_batch(const EvalArgs *args_dev, const long long *prefix_dev, int n_ctx,
                              unsigned long long *queue, int threads, size_t dyn, int grid, bool stacked,
                              cudaStream_t s);
cudaError_t eval_batch_occupancy(int threads, size_t dyn, bool stacked, int *blocks_per_sm);
cudaError_t launch_reduce(const RedArgs &r, cudaStream_t s);
cudaError_t launch_reduce_batch(const RedArgs *ra_dev, const int *bl_prefix_dev, int n_ctx, int total_bl,
                                cudaStream_t s);
// A° tables of every channel (ap_table_dev: the caller's table on the device
// for PSC_AP_TABLE, else unused).
cudaError_t launch_tables(const psc_aperture &ap, const double *ap_table_dev, const double *freq_dev, int nc,
                          double du, int ov, int support, const int *tab_off_dev, const int *tab_len_dev,
                          float2 *tabs, cudaStream_t s);
// Reach of the A° table in grid cells: D_lambda / du (disk, caller table), (S/2) sqrt(2) (Gaussian).
inline double aperture_reach(int kind, double dl, double du, int support) {
    return kind == PSC_AP_GAUSS ? 0.5 * support * 1.4142135623730951 : dl / du;
}
// Argument check of an aperture description (message in *why).
bool aperture_ok(const psc_aperture *ap, const char **why);
cudaError_t launch_lm_update(const LMArgs &a, cudaStream_t s);
// Batched forms: one block per context (device arrays of LMArgs).
cudaError_t launch_lm_update_batch(const LMArgs *la_dev, int n_ctx, size_t dyn, cudaStream_t s);
cudaError_t launch_lm_restart_batch(const LMArgs *la_dev, const LMState *const *st0_dev,
                                    const double *const *lm0_dev, int n_ctx, cudaStream_t s);
size_t lm_smem_bytes(int n_ant);
// Sets the LM kernel's shared-memory limit (once per device, before launches).
cudaError_t lm_prepare(int n_ant);
cudaError_t launch_lm_restart(const LMArgs &a, const LMState *st0, const double *lm0, cudaStream_t s);
cudaError_t set_eval_smem(size_t dyn);
// Dynamic shared memory available to one fused-kernel block on the current device.
cudaError_t eval_smem_allowed(size_t *allowed);
// Exact disk kernel (exact.cu): the fused evaluation with it (one launch per
// context, one visibility per thread), its dynamic shared memory, and the
// per-channel lens-moment combinations ([sum of table lengths][10] floats)
// it reads, computed once per context.
cudaError_t launch_exact(const EvalArgs &a, bool predict, cudaStream_t s);
size_t exact_dyn_smem(int c_group, int tab_stride);
cudaError_t launch_exact_moments(double diam_m, const double *freq_dev, int nc, double du, int ov,
                                 const int *tab_off_dev, const int *tab_len_dev, float *kmom, cudaStream_t s);
// Dynamic shared memory of one fused-kernel block (c_group zero-padded tables).
size_t eval_dyn_smem(int c_group, int tab_stride);
// Largest distance (metres, u-v plane) between the baselines of consecutive
// time steps: *out_bits receives its FP32 bit pattern (atomic max; zero it first).
cudaError_t launch_step_max(const double *uvw, int nt, int n_bl, unsigned *out_bits, cudaStream_t s);
// Records msg as the context-free last error (psc_last_error(NULL)); returns st.
psc_status set_global_error(psc_status st, const char *msg);
cudaError_t launch_features(const StencilArgs &a, double *blsum, int n_ant, float *feat, cudaStream_t s);
// Dynamic shared memory of one stencil block.
size_t stencil_dyn_smem(int c_group, int max_tab_len, int stage);
// The stencil pass, per-baseline sums and features of n pairs in three launches
// (device tables of StencilArgs, first-brick prefixes [n + 1] and FeatPair).
cudaError_t launch_features_batch(const StencilArgs *args_dev, const long long *prefix_dev, const FeatPair *pairs_dev,
                                  int n, long long total_blocks, int threads, size_t dyn, int max_bl, int max_ant,
                                  float sigma, cudaStream_t s);
// Workspace (bytes) of launch_model_grid; the model grid goes to grid_out
// and *err_dev points (inside ws) at a flag set if a tensor-core wait ran out.
size_t model_grid_ws_bytes(int n_img, int n_grid);
// Model grid of n_comp point components (host [n_comp][stride] = l, m, S, and
// with stride 4 also n - 1, which gives flux k the phase 2 pi wp (n_k - 1)) on
// the tensor cores, in the workspace of model_grid_comp_ws_bytes(n_comp, n_grid,
// stride); *err_dev is set if a tensor-core wait ran out.
size_t model_grid_comp_ws_bytes(int n_comp, int n_grid, int stride);
cudaError_t launch_model_grid_comp(int n_comp, const double *comp_host, int stride, double wp, int n_grid, double du,
                                   void *ws, float2 *grid_out, int **err_dev, cudaStream_t s);
// Least-squares plane w = a u + b v of n_rows baselines (device uvw [n_rows][3]):
// the sums uu, uv, vv, uw, vw in FP64 go to sums_dev[5] (zeroed by the launcher).
cudaError_t launch_plane_sums(const double *uvw, long long n_rows, double *sums_dev, cudaStream_t s);
// Per-block (min, max) of w - a u - b v over n_rows baselines into
// out_dev[2 * blocks]; returns the block count used (at most 1024) in *blocks.
cudaError_t launch_wrange(const double *uvw, long long n_rows, double a, double b, double *out_dev, int *blocks,
                          cudaStream_t s);
cudaError_t launch_model_grid(int n_img, int n_grid, const float *image, void *ws, float2 *grid_out, int **err_dev,
                              cudaStream_t s);
// FP32 split (u_hi, u_lo, v_hi, v_lo) of n uvw triples (FP64 metres).
cudaError_t launch_split_uv(const double *uvw, size_t n, float4 *out, cudaStream_t s);
// bfloat16 copy (nearest even, re in the low half) of n complex64 values.
cudaError_t launch_grid_to_bf16(const float2 *grid, size_t n, unsigned *out, cudaStream_t s);

}  // namespace psc

// C ABI of the Pointing SelfCal library (declared in include/psc.h): argument
// checks, context workspace, and the launch sequences of Algorithm 1's
// pre-computes and iteration loop.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "psc_internal.cuh"

using namespace psc;

struct psc_ctx {
    cudaStream_t stream = nullptr;
    int n_ant = 0, n_bl = 0, nt = 0, nc = 0;
    psc_grid_desc gd{};
    psc_aperture ap{};
    double du = 0.0;
    const double *uvw = nullptr;
    const float2 *grid = nullptr;
    unsigned *d_grid_bf16 = nullptr;   // bfloat16 copy of the grid (PSC_GRID_BF16), else null
    float4 *d_uvs = nullptr;           // FP32 split of uvw read by the fused kernel
    // workspace (device)
    ChanConst *d_chan = nullptr;
    float2 *d_tabs = nullptr;
    int2 *d_pairs = nullptr;
    double *d_partials = nullptr;
    size_t partials_cap = 0;     // in bricks
    double *d_blsum = nullptr;
    double *d_ev = nullptr;      // evaluation at d_lm_trial
    double *d_cur = nullptr;     // accepted evaluation
    double *d_lm_trial = nullptr;
    double *d_lm_cur = nullptr;
    double *d_mat = nullptr;
    float *d_mat32 = nullptr;
    double *d_rhs = nullptr;
    LMState *d_state = nullptr;
    LMState *d_state0 = nullptr; // state written by psc_lm_begin (for psc_lm_restart)
    double *d_lm0 = nullptr;     // start offsets written by psc_lm_begin
    bool begun = false;
    int *d_done = nullptr;       // points at d_state->done
    int max_tab_len = 0;
    int t_tile = 32, c_group = 4;
    int kv = 1;                  // visibilities per thread at consecutive times
    int flat = 0;                // > 0: bricks of `flat` consecutive (channel, time-group) items
    int no_stage = 0;            // PSC_STAGE_NEVER: taps read the grid from global memory
    int trk_kv = 0;              // > 0: reduce-mode evaluations run the track kernel, trk_kv visibilities per lane
    float2 *d_tabcs = nullptr;   // track kernel: per-channel (intercept, slope) tables [nc][trk_stride]
    int trk_stride = 0;
    void *d_tmap = nullptr;      // track kernel: tensor maps over the grid (3 x 128 bytes)
    int *d_err = nullptr;        // set by a kernel whose bounded wait ran out
    int kernel_model = PSC_KERNEL_GAUSS;
    int brick_order = PSC_ORDER_BASELINE;
    int *d_bl_order = nullptr;   // baselines in Morton order of their mid-interval (u, v)
    float *d_kmom = nullptr;     // exact disk kernel: lens-moment combinations (psc_set_kernel_model)
    double *d_aptab = nullptr;   // PSC_AP_TABLE: the caller's table, copied
    // residual-w stack (psc_set_wstack): borrowed planes [wp_n][ng][ng], plane
    // w_p = wp_w0 + p wp_dw (wavelengths), residual w of the plane w = wp_a u + wp_b v
    const float2 *wp_grid = nullptr;
    int wp_n = 0;
    double wp_w0 = 0.0, wp_dw = 0.0, wp_a = 0.0, wp_b = 0.0;
    std::vector<double> h_freq;  // channel frequencies (Hz)
    std::vector<int> h_tab_off, h_tab_len;   // radial table layout per channel
    double step_cells = 0.0;     // largest move of a baseline between time steps (cells, top channel)
    bool multi_ok = false;       // kv > 1 allowed: every channel's aperture fits inside the S x S window
    LMState h_state{};
    std::vector<double> h_ev;
    std::string err;
    // stencil features (psc_features)
    double *d_spart = nullptr;
    size_t spart_cap = 0;
    double *d_sblsum = nullptr;
    float *d_feat = nullptr;     // [n_ant][52] (psc_learned_init)
    // fused-kernel timing (psc_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

namespace {

thread_local std::string g_err;
// polls of one bounded mbarrier wait in the library's kernels (psc_set_wait_limit)
constexpr long long kDefaultWaitPolls = 1LL << 24;
long long g_wait_polls = kDefaultWaitPolls;

psc_status fail(psc_ctx *ctx, psc_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_err = msg;
    return st;
}

}  // namespace

long long psc::wait_limit() { return g_wait_polls; }

bool psc::aperture_ok(const psc_aperture *ap, const char **why) {
    if (!ap) { *why = "aperture is NULL"; return false; }
    if (ap->kind != PSC_AP_DISK && ap->kind != PSC_AP_GAUSS && ap->kind != PSC_AP_TABLE) { *why = "unknown aperture kind"; return false; }
    if (!(ap->diam_m > 0.0) || !(ap->alpha_per_dlambda > 0.0) || !std::isfinite(ap->diam_m) ||
        !std::isfinite(ap->alpha_per_dlambda)) {
        *why = "diam_m and alpha_per_dlambda must be finite and > 0";
        return false;
    }
    if (ap->kind == PSC_AP_TABLE) {
        if (!ap->table || ap->table_len < 2 || ap->table_len > 65536) {
            *why = "PSC_AP_TABLE needs a table of 2 .. 65536 samples";
            return false;
        }
        for (int k = 0; k < ap->table_len; ++k)
            if (!std::isfinite(ap->table[k])) { *why = "the aperture table must be finite"; return false; }
    }
    return true;
}

psc_status psc::set_global_error(psc_status st, const char *msg) {
    g_err = msg;
    return st;
}

namespace {

psc_status cuda_fail(psc_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? PSC_ERR_OOM : PSC_ERR_CUDA, m);
}

#define PSC_CUDA(ctx, call)                                       \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

void free_ctx(psc_ctx *c) {
    if (!c) return;
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    cudaFree(c->d_grid_bf16);
    cudaFree(c->d_kmom);
    cudaFree(c->d_tabcs);
    cudaFree(c->d_tmap);
    cudaFree(c->d_aptab);
    cudaFree(c->d_err);
    cudaFree(c->d_bl_order);
    cudaFree(c->d_uvs);
    cudaFree(c->d_spart);
    cudaFree(c->d_sblsum);
    cudaFree(c->d_feat);
    cudaFree(c->d_chan); cudaFree(c->d_tabs); cudaFree(c->d_pairs); cudaFree(c->d_partials);
    cudaFree(c->d_blsum); cudaFree(c->d_ev); cudaFree(c->d_cur); cudaFree(c->d_lm_trial);
    cudaFree(c->d_lm_cur); cudaFree(c->d_mat); cudaFree(c->d_mat32); cudaFree(c->d_rhs); cudaFree(c->d_state);
    cudaFree(c->d_state0); cudaFree(c->d_lm0);
    delete c;
}

int n_tt(const psc_ctx *c) { return (c->nt + c->t_tile * c->kv - 1) / (c->t_tile * c->kv); }

// Largest visibility separation within one thread's kv time steps (cells).
double kv_spread(const psc_ctx *c, int kv) { return (kv - 1) * c->step_cells; }

// kv > 1 needs every tap of the thread's union of rows to be either inside a
// visibility's own S x S window or outside its aperture (then its table entry
// is zero); the union stays within spread + 1 cells of each visibility.
bool kv_allowed(const psc_ctx *c, int kv) {
    if (kv == 1) return true;
    if (kv != 2) return false;
    return c->multi_ok && kv_spread(c, kv) <= 4.0;
}

// Staged table entries per channel: the table plus zero entries for every
// radius a tap of the thread can reach (rho_max + spread + 1 cells).
int tab_stride(const psc_ctx *c, int kv) {
    if (kv == 1) return c->max_tab_len + 2;
    return c->max_tab_len + (int)std::ceil(c->gd.oversample * (kv_spread(c, kv) + 1.0)) + 2;
}
int n_cg(const psc_ctx *c) { return (c->nc + c->c_group - 1) / c->c_group; }
// Track kernel: time chunks of 32 lanes x trk_kv steps per baseline, and the
// staged tile capacity of one buffer (cells).
int trk_chunks(const psc_ctx *c) { return (c->nt + 32 * c->trk_kv - 1) / (32 * c->trk_kv); }
constexpr int kTrkCap = 512;
// Zero table entries the track kernel's tap pattern can reach past a
// channel's table with kv visibilities per lane: its taps lie within
// rho_max + 2 spread + sqrt(2) (+ a margin) cells of each visibility.
int trk_pad(const psc_ctx *c, int kv) {
    return (int)std::ceil(c->gd.oversample * (2.0 * kv_spread(c, kv) + 1.5)) + 2;
}
// Flat bricks: groups of kv consecutive time steps per channel, the bricks
// per baseline, and the most channels one brick's items can span.
int n_tp(const psc_ctx *c) { return (c->nt + c->kv - 1) / c->kv; }
long long bricks_per_bl(const psc_ctx *c) {
    if (c->trk_kv > 0) return trk_chunks(c);
    if (c->flat > 0) return ((long long)c->nc * n_tp(c) + c->flat - 1) / c->flat;
    return (long long)n_cg(c) * n_tt(c);
}
int ch_span(const psc_ctx *c) {
    return c->flat > 0 ? std::min(c->nc, (c->flat + n_tp(c) - 2) / n_tp(c) + 1) : c->c_group;
}
// Block width of the fused kernel for this context's bricks.
int eval_threads(const psc_ctx *c) {
    if (c->trk_kv > 0) return kTrkThreads;
    return ((c->flat > 0 ? c->flat : c->t_tile * c->c_group) + 31) / 32 * 32;
}

psc_status ensure_partials(psc_ctx *c) {
    const size_t need = (size_t)c->n_bl * bricks_per_bl(c);
    if (need <= c->partials_cap) return PSC_OK;
    cudaFree(c->d_partials);
    c->d_partials = nullptr;
    c->partials_cap = 0;
    PSC_CUDA(c, dalloc(&c->d_partials, need * kRed));
    c->partials_cap = need;
    return PSC_OK;
}

EvalArgs eval_args(const psc_ctx *c, const double *lm_dev) {
    EvalArgs a{};
    a.uvw = c->uvw;
    a.uvs = c->d_uvs;
    a.grid = c->grid;
    a.grid_bf16 = c->d_grid_bf16;
    a.chan = c->d_chan;
    a.tabs = c->d_tabs;
    a.pairs = c->d_pairs;
    a.lm = lm_dev;
    a.w_scale = 1.f;
    a.partials = c->d_partials;
    a.n_bl = c->n_bl;
    a.nt = c->nt;
    a.nc = c->nc;
    a.ng = c->gd.n_grid;
    a.support = c->gd.support;
    a.ov = c->gd.oversample;
    a.du = (float)c->du;
    a.t_tile = c->t_tile;
    a.c_group = c->c_group;
    a.kv = c->kv;
    a.no_stage = c->no_stage;
    a.n_tt = n_tt(c);
    a.n_cg = n_cg(c);
    a.decorrelation = c->ap.decorrelation;
    a.max_tab_len = c->max_tab_len;
    a.tab_stride = tab_stride(c, c->kv);
    a.n_bricks = (long long)c->n_bl * bricks_per_bl(c);
    a.flat = c->flat;
    a.n_tp = n_tp(c);
    a.bpb = (int)bricks_per_bl(c);
    a.ch_span = ch_span(c);
    a.exact = c->kernel_model == PSC_KERNEL_EXACT_DISK;
    a.bl_order = c->brick_order == PSC_ORDER_UV ? c->d_bl_order : nullptr;
    a.kmom = c->d_kmom;
    a.err = c->d_err;
    a.wait_limit = wait_limit();
    if (c->trk_kv > 0) {
        a.trk_kv = c->trk_kv;
        a.trk_chunks = trk_chunks(c);
        a.trk_cap = kTrkCap;
        a.trk_stride = c->trk_stride;
        a.trk_pad = trk_pad(c, c->trk_kv);
        // the longest table a channel copies with this tiling's pad (the stride
        // is sized for two visibilities per lane)
        a.trk_tabc = (std::min(c->trk_stride, (c->max_tab_len + a.trk_pad + 1) & ~1) + 15) / 16 * 16;
        a.trk_spread = (float)c->step_cells;
        a.tabs_cs = c->d_tabcs;
        a.tmap = c->d_tmap;
    }
    if (c->wp_n > 0) {
        a.grid = c->wp_grid;
        a.grid_bf16 = nullptr;
        a.wp_n = c->wp_n;
        a.wp_a = c->wp_a;
        a.wp_b = c->wp_b;
        a.wp_scale = c->du / c->wp_dw;             // uv_scale du = nu / c
        a.wp_q0 = c->wp_w0 / c->wp_dw;
    }
    return a;
}

RedArgs red_args(const psc_ctx *c, double *ev_out, const int *skip) {
    RedArgs r{};
    r.partials = c->d_partials;
    r.blsum = c->d_blsum;
    r.ev = ev_out;
    r.skip = skip;
    r.n_bl = c->n_bl;
    r.bpb = (int)bricks_per_bl(c);
    r.n_ant = c->n_ant;
    return r;
}

LMArgs lm_args(const psc_ctx *c) {
    LMArgs a{};
    a.st = c->d_state;
    a.lm_cur = c->d_lm_cur;
    a.lm_trial = c->d_lm_trial;
    a.ev = c->d_ev;
    a.cur = c->d_cur;
    a.mat = c->d_mat;
    a.mat32 = c->d_mat32;
    a.rhs = c->d_rhs;
    a.pairs = c->d_pairs;
    a.n_ant = c->n_ant;
    a.n_bl = c->n_bl;
    a.err = c->d_err;
    return a;
}

bool check_grid_desc(const psc_grid_desc *gd, std::string *why) {
    if (!gd) { *why = "grid descriptor is NULL"; return false; }
    if (gd->n_img < 2 || gd->n_img > 8192 || gd->n_img % 2) { *why = "n_img must be even in [2, 8192]"; return false; }
    if (gd->n_grid < gd->n_img || gd->n_grid > 16384 || gd->n_grid % 2) { *why = "n_grid must be even in [n_img, 16384]"; return false; }
    if (!(gd->cell_rad > 0.0) || !std::isfinite(gd->cell_rad)) { *why = "cell_rad must be > 0"; return false; }
    if (gd->support < 2 || gd->support > 64 || gd->support % 2) { *why = "support must be even in [2, 64]"; return false; }
    if (gd->oversample < 1 || gd->oversample > 64) { *why = "oversample must be in [1, 64]"; return false; }
    return true;
}

psc_status eval_reduce(psc_ctx *c, const double *lm_dev, const void *vis_obs, const float *w, double w_scale,
                       double *ev_out, const int *skip) {
    psc_status st = ensure_partials(c);
    if (st != PSC_OK) return st;
    EvalArgs a = eval_args(c, lm_dev);
    a.vis_obs = (const float2 *)vis_obs;
    a.w = w;
    a.w_scale = (float)w_scale;
    a.skip = skip;
    if (c->prof) {
        while (c->ev_pool.size() < c->ev_used + 2) {
            cudaEvent_t e;
            PSC_CUDA(c, cudaEventCreate(&e));
            c->ev_pool.push_back(e);
        }
        PSC_CUDA(c, cudaEventRecord(c->ev_pool[c->ev_used], c->stream));
    }
    PSC_CUDA(c, a.trk_kv > 0 ? launch_track(a, c->stream) : launch_eval(a, false, c->stream));
    if (c->prof) {
        PSC_CUDA(c, cudaEventRecord(c->ev_pool[c->ev_used + 1], c->stream));
        c->ev_used += 2;
    }
    PSC_CUDA(c, launch_reduce(red_args(c, ev_out, skip), c->stream));
    return PSC_OK;
}

// Stencil-feature arguments of one context and its data: every kept time
// step of up to 32 in one tile, and as many channels (at most 16) as fill 128
// threads (few kept steps would otherwise leave most lanes of a 32-step tile
// idle).
StencilArgs stencil_args(const psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale, double sigma,
                         int time_stride) {
    const int nts = (ctx->nt + time_stride - 1) / time_stride;
    const int t_tile = std::min(32, nts);
    const int c_group = std::min(std::min(16, ctx->nc), std::max(1, 128 / t_tile));
    StencilArgs a{};
    a.uvw = ctx->uvw;
    a.grid = ctx->grid;
    a.chan = ctx->d_chan;
    a.tabs = ctx->d_tabs;
    a.vis_obs = (const float2 *)vis_obs;
    a.w = w;
    a.w_scale = (float)w_scale;
    a.n_bl = ctx->n_bl;
    a.nt = ctx->nt;
    a.nc = ctx->nc;
    a.ng = ctx->gd.n_grid;
    a.support = ctx->gd.support;
    a.ov = ctx->gd.oversample;
    a.du = (float)ctx->du;
    a.t_tile = t_tile;
    a.c_group = c_group;
    a.n_tt = (nts + t_tile - 1) / t_tile;
    a.n_cg = (ctx->nc + c_group - 1) / c_group;
    a.time_stride = time_stride;
    a.decorrelation = ctx->ap.decorrelation;
    a.max_tab_len = ctx->max_tab_len;
    // a 64 x 64 staged tile pays only for bricks of many visibilities; small
    // bricks read the grid directly and keep shared memory (and occupancy) free
    a.stage = t_tile * c_group >= 64;
    a.n_bricks = (long long)ctx->n_bl * a.n_cg * a.n_tt;
    a.sigma = (float)sigma;
    // bricks of exactly one warp with a single channel group and time tile (a
    // brick is then a baseline): four per block, sharing the block's tables
    a.wpb = (t_tile * c_group == 32 && a.n_cg == 1 && a.n_tt == 1 && !a.stage) ? 4 : 1;   // at most 4: one box per warp
    return a;
}

// Track kernel set-up of a context: the per-channel (intercept, slope)
// tables and the grid's tensor maps, once.
psc_status trk_prepare(psc_ctx *c) {
    if (c->d_tmap) return PSC_OK;
    const int stride = (c->max_tab_len + trk_pad(c, kv_allowed(c, 2) ? 2 : 1) + 1) & ~1;
    cudaError_t e = dalloc(&c->d_tabcs, (size_t)c->nc * stride);
    if (e == cudaSuccess) e = launch_track_tables(c->d_chan, c->d_tabs, c->nc, stride, c->d_tabcs, c->stream);
    void *maps = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&maps, 3 * 128);
    if (e == cudaSuccess) e = make_grid_maps(c->grid, c->gd.n_grid, maps, c->stream);
    if (e != cudaSuccess) {
        cudaFree(maps);
        cudaFree(c->d_tabcs);
        c->d_tabcs = nullptr;
        return cuda_fail(c, e, "track kernel set-up");
    }
    c->trk_stride = stride;
    c->d_tmap = maps;
    return PSC_OK;
}

// Why the track kernel cannot serve this context with kv visibilities per
// lane (empty: it can).
std::string trk_refusal(const psc_ctx *c, int kv) {
    if (kv != 1 && kv != 2) return "vis_per_lane must be 1 or 2";
    if (c->kernel_model != PSC_KERNEL_GAUSS) return "the track kernel uses the Gaussian kernel model";
    if (c->wp_n > 0) return "the track kernel does not read a residual-w stack";
    if (c->d_grid_bf16) return "the track kernel reads the FP32 grid";
    if ((uintptr_t)c->grid % 16) return "the track kernel needs a 16-byte aligned grid";
    if (!c->multi_ok) return "the track kernel needs every channel's aperture inside the S x S window";
    if (!kv_allowed(c, kv)) return "vis_per_lane 2 needs consecutive time steps within 4 cells";
    return "";
}

// The evaluation's bounded waits ran out (a kernel set *d_err): clears the flag.
psc_status check_err_flag(psc_ctx *c) {
    int h = 0;
    PSC_CUDA(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PSC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h) {
        PSC_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        return fail(c, PSC_ERR_TIMEOUT, "a bounded wait of the fused evaluation ran out; its results were discarded");
    }
    return PSC_OK;
}

}  // namespace

extern "C" {

psc_status psc_set_wait_limit(long long polls) {
    g_wait_polls = polls < 0 ? kDefaultWaitPolls : polls;
    return PSC_OK;
}

long long psc_get_wait_limit(void) { return g_wait_polls; }

void psc_solve_opts_default(psc_solve_opts *o) {
    if (!o) return;
    o->max_iter = 50;
    o->mode = PSC_LM_FULL;
    o->lam0 = 1e-3;
    o->lam_max = 1e10;
    o->lam_min = 1e-12;
    o->step_tol_rad = 1e-4 * M_PI / (180.0 * 3600.0);
    o->chi2_rtol = 1e-10;
    o->block_gain = 0.5;
}

const char *psc_last_error(const psc_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

psc_status psc_uvw(int n_ant, const double *ant_enu_m, double lat_rad, double dec_rad, int n_time, const double *ha_rad,
                   void *uvw_out, void *stream) {
    if (n_ant < 2 || n_ant > 512) return fail(nullptr, PSC_ERR_ARG, "n_ant must be in [2, 512]");
    if (n_time < 1) return fail(nullptr, PSC_ERR_ARG, "n_time must be >= 1");
    if (!ant_enu_m || !ha_rad || !uvw_out) return fail(nullptr, PSC_ERR_ARG, "ant_enu_m, ha_rad and uvw_out must be non-NULL");
    if (!std::isfinite(lat_rad) || !std::isfinite(dec_rad) || std::fabs(lat_rad) > M_PI / 2 || std::fabs(dec_rad) > M_PI / 2)
        return fail(nullptr, PSC_ERR_ARG, "latitude and declination must be in [-pi/2, pi/2]");
    for (int k = 0; k < 3 * n_ant; ++k)
        if (!std::isfinite(ant_enu_m[k])) return fail(nullptr, PSC_ERR_ARG, "antenna positions must be finite");
    for (int t = 0; t < n_time; ++t)
        if (!std::isfinite(ha_rad[t])) return fail(nullptr, PSC_ERR_ARG, "hour angles must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    double *d_enu = nullptr, *d_ha = nullptr;
    cudaError_t e = dalloc(&d_enu, 3 * (size_t)n_ant);
    if (e == cudaSuccess) e = dalloc(&d_ha, n_time);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_enu, ant_enu_m, sizeof(double) * 3 * n_ant, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ha, ha_rad, sizeof(double) * n_time, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_uvw(d_enu, n_ant, lat_rad, dec_rad, d_ha, n_time, (double *)uvw_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_enu);
    cudaFree(d_ha);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_uvw");
    return PSC_OK;
}

psc_status psc_model_grid(const psc_grid_desc *gd, const float *image_dev, void *grid_out, void *stream) {
    std::string why;
    if (!check_grid_desc(gd, &why)) return fail(nullptr, PSC_ERR_ARG, why);
    if (!image_dev || !grid_out) return fail(nullptr, PSC_ERR_ARG, "image and grid pointers must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = nullptr;
    int *err_dev = nullptr;
    int herr = 0;
    cudaError_t e = cudaMalloc(&ws, model_grid_ws_bytes(gd->n_img, gd->n_grid));
    if (e == cudaSuccess) e = launch_model_grid(gd->n_img, gd->n_grid, image_dev, ws, (float2 *)grid_out, &err_dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err_dev, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_model_grid");
    if (herr) return fail(nullptr, PSC_ERR_TIMEOUT, "psc_model_grid: a tensor-core wait timed out");
    return PSC_OK;
}

psc_status psc_model_grid_components(int n_comp, const double *comp_lmS, int n_grid, double cell_rad,
                                     void *grid_out, void *stream) {
    if (n_comp < 0 || n_comp > (1 << 24)) return fail(nullptr, PSC_ERR_ARG, "n_comp must be in [0, 2^24]");
    if (n_comp > 0 && !comp_lmS) return fail(nullptr, PSC_ERR_ARG, "comp_lmS is NULL");
    if (!grid_out) return fail(nullptr, PSC_ERR_ARG, "grid_out is NULL");
    if (n_grid < 2 || n_grid > 16384 || n_grid % 2) return fail(nullptr, PSC_ERR_ARG, "n_grid must be even in [2, 16384]");
    if (!(cell_rad > 0.0) || !std::isfinite(cell_rad)) return fail(nullptr, PSC_ERR_ARG, "cell_rad must be > 0");
    for (int k = 0; k < 3 * n_comp; ++k)
        if (!std::isfinite(comp_lmS[k])) return fail(nullptr, PSC_ERR_ARG, "components must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = nullptr;
    int *err_dev = nullptr;
    int herr = 0;
    const double du = 1.0 / (n_grid * cell_rad);
    cudaError_t e = cudaMalloc(&ws, model_grid_comp_ws_bytes(n_comp, n_grid, 3));
    if (e == cudaSuccess)
        e = launch_model_grid_comp(n_comp, comp_lmS, 3, 0.0, n_grid, du, ws, (float2 *)grid_out, &err_dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err_dev, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_model_grid_components");
    if (herr) return fail(nullptr, PSC_ERR_TIMEOUT, "psc_model_grid_components: a tensor-core wait timed out");
    return PSC_OK;
}

psc_status psc_snapshot_plane(const double *uvw_dev, long long n_rows, double *a, double *b, void *stream) {
    if (!uvw_dev || !a || !b) return fail(nullptr, PSC_ERR_ARG, "uvw, a and b must be non-NULL");
    if (n_rows < 2) return fail(nullptr, PSC_ERR_ARG, "n_rows must be >= 2");
    cudaStream_t s = (cudaStream_t)stream;
    double *d_sums = nullptr;
    double h[5] = {};
    cudaError_t e = cudaMalloc(&d_sums, 5 * sizeof(double));
    if (e == cudaSuccess) e = launch_plane_sums(uvw_dev, n_rows, d_sums, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_sums);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_snapshot_plane");
    // normal equations [uu uv; uv vv] (a, b) = (uw, vw)
    const double det = h[0] * h[2] - h[1] * h[1];
    if (!(det > 1e-12 * h[0] * h[2])) return fail(nullptr, PSC_ERR_NUMERIC, "psc_snapshot_plane: the baselines span no plane (collinear u, v)");
    *a = (h[3] * h[2] - h[4] * h[1]) / det;
    *b = (h[4] * h[0] - h[3] * h[1]) / det;
    return PSC_OK;
}

psc_status psc_snapshot_components(int n_comp, const double *comp_in, double a, double b, const psc_aperture *ap,
                                   double freq_hz, double *comp_out) {
    if (n_comp < 0 || (n_comp > 0 && (!comp_in || !comp_out))) return fail(nullptr, PSC_ERR_ARG, "component arrays must be non-NULL");
    if (!ap || (ap->kind != PSC_AP_DISK && ap->kind != PSC_AP_GAUSS))
        return fail(nullptr, PSC_ERR_ARG, "the source move needs a disk or Gaussian aperture (its beam in closed form)");
    if (!(ap->diam_m > 0.0) || !(freq_hz > 0.0) || !std::isfinite(a) || !std::isfinite(b))
        return fail(nullptr, PSC_ERR_ARG, "diam_m, freq_hz must be > 0 and a, b finite");
    const double dl = ap->diam_m * freq_hz / kC;
    const double alpha = ap->alpha_per_dlambda * dl;
    auto pb = [&](double rho) {                       // pointing-free power pattern
        if (ap->kind == PSC_AP_GAUSS) return std::exp(-2.0 * alpha * alpha * rho * rho);
        const double x = M_PI * dl * rho;
        const double e = x > 1e-12 ? 2.0 * std::cyl_bessel_j(1.0, x) / x : 1.0;
        return e * e;
    };
    for (int k = 0; k < n_comp; ++k) {
        const double l = comp_in[3 * k], m = comp_in[3 * k + 1], S = comp_in[3 * k + 2];
        const double r2 = l * l + m * m;
        if (!(r2 < 1.0)) return fail(nullptr, PSC_ERR_ARG, "a component lies outside the unit disk");
        const double nm1 = -r2 / (1.0 + std::sqrt(1.0 - r2));     // n - 1 without cancellation
        const double l1 = l + a * nm1, m1 = m + b * nm1;
        const double p1 = pb(std::hypot(l1, m1));
        if (!(p1 > 1e-300)) return fail(nullptr, PSC_ERR_NUMERIC, "a moved component sits on a null of the beam");
        comp_out[3 * k] = l1;
        comp_out[3 * k + 1] = m1;
        comp_out[3 * k + 2] = S * pb(std::sqrt(r2)) / p1;
    }
    return PSC_OK;
}

psc_status psc_wstack_components(int n_comp, const double *comp_in, double a, double b, const psc_aperture *ap,
                                 double freq_hz, double *comp_out) {
    if (n_comp < 0 || (n_comp > 0 && (!comp_in || !comp_out))) return fail(nullptr, PSC_ERR_ARG, "component arrays must be non-NULL");
    const uintptr_t in0 = (uintptr_t)comp_in, out0 = (uintptr_t)comp_out;
    if (n_comp > 0 && out0 < in0 + 3 * sizeof(double) * (size_t)n_comp &&
        in0 < out0 + 4 * sizeof(double) * (size_t)n_comp)
        return fail(nullptr, PSC_ERR_ARG, "comp_out must not overlap comp_in");
    std::vector<double> snap(3 * (size_t)n_comp);
    psc_status st = psc_snapshot_components(n_comp, comp_in, a, b, ap, freq_hz, snap.data());
    if (st != PSC_OK) return st;
    for (int k = 0; k < n_comp; ++k) {
        const double l = comp_in[3 * k], m = comp_in[3 * k + 1];
        const double r2 = l * l + m * m;
        comp_out[4 * k] = snap[3 * k];
        comp_out[4 * k + 1] = snap[3 * k + 1];
        comp_out[4 * k + 2] = snap[3 * k + 2];
        comp_out[4 * k + 3] = -r2 / (1.0 + std::sqrt(1.0 - r2));   // n - 1 of the true direction
    }
    return PSC_OK;
}

psc_status psc_wstack_range(const double *uvw_dev, long long n_rows, double a, double b, double *wmin_m, double *wmax_m,
                            void *stream) {
    if (!uvw_dev || !wmin_m || !wmax_m) return fail(nullptr, PSC_ERR_ARG, "uvw, wmin and wmax must be non-NULL");
    if (n_rows < 1) return fail(nullptr, PSC_ERR_ARG, "n_rows must be >= 1");
    if (!std::isfinite(a) || !std::isfinite(b)) return fail(nullptr, PSC_ERR_ARG, "a and b must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    double *d_out = nullptr;
    int blocks = 0;
    std::vector<double> h;
    cudaError_t e = cudaMalloc(&d_out, 2 * 1024 * sizeof(double));
    if (e == cudaSuccess) e = launch_wrange(uvw_dev, n_rows, a, b, d_out, &blocks, s);
    if (e == cudaSuccess) {
        h.resize(2 * (size_t)blocks);
        e = cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_wstack_range");
    double lo = h[0], hi = h[1];
    for (int k = 1; k < blocks; ++k) {
        lo = std::min(lo, h[2 * k]);
        hi = std::max(hi, h[2 * k + 1]);
    }
    if (!std::isfinite(lo) || !std::isfinite(hi)) return fail(nullptr, PSC_ERR_NUMERIC, "psc_wstack_range: non-finite uvw");
    *wmin_m = lo;
    *wmax_m = hi;
    return PSC_OK;
}

psc_status psc_model_grid_wstack(int n_comp, const double *comp_lmSn, int n_grid, double cell_rad, int n_planes,
                                 double w0, double dw, void *grids_out, void *stream) {
    if (n_comp < 0 || n_comp > (1 << 24)) return fail(nullptr, PSC_ERR_ARG, "n_comp must be in [0, 2^24]");
    if (n_comp > 0 && !comp_lmSn) return fail(nullptr, PSC_ERR_ARG, "comp_lmSn is NULL");
    if (!grids_out) return fail(nullptr, PSC_ERR_ARG, "grids_out is NULL");
    if (n_grid < 2 || n_grid > 16384 || n_grid % 2) return fail(nullptr, PSC_ERR_ARG, "n_grid must be even in [2, 16384]");
    if (!(cell_rad > 0.0) || !std::isfinite(cell_rad)) return fail(nullptr, PSC_ERR_ARG, "cell_rad must be > 0");
    if (n_planes < 2 || n_planes > 65536) return fail(nullptr, PSC_ERR_ARG, "n_planes must be in [2, 65536]");
    if (!std::isfinite(w0) || !(dw > 0.0) || !std::isfinite(dw)) return fail(nullptr, PSC_ERR_ARG, "w0 must be finite and dw > 0");
    for (int k = 0; k < 4 * n_comp; ++k)
        if (!std::isfinite(comp_lmSn[k])) return fail(nullptr, PSC_ERR_ARG, "components must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = nullptr;
    int *err_dev = nullptr;
    int herr = 0;
    const double du = 1.0 / (n_grid * cell_rad);
    const size_t plane = (size_t)n_grid * n_grid;
    cudaError_t e = cudaMalloc(&ws, model_grid_comp_ws_bytes(n_comp, n_grid, 4));
    for (int p = 0; p < n_planes && e == cudaSuccess; ++p) {
        e = launch_model_grid_comp(n_comp, comp_lmSn, 4, w0 + p * dw, n_grid, du, ws, (float2 *)grids_out + p * plane,
                                   &err_dev, s);
        // the workspace (and its error flag) is reused by the next plane
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemcpy(&herr, err_dev, sizeof(int), cudaMemcpyDeviceToHost);
        if (herr) break;
    }
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_model_grid_wstack");
    if (herr) return fail(nullptr, PSC_ERR_TIMEOUT, "psc_model_grid_wstack: a tensor-core wait timed out");
    return PSC_OK;
}

psc_status psc_create(psc_ctx **out, const psc_obs *obs, const psc_aperture *ap, const psc_grid_desc *gd,
                      const void *grid_dev, void *stream) {
    if (!out) return fail(nullptr, PSC_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!obs || !ap) return fail(nullptr, PSC_ERR_ARG, "obs and aperture must be non-NULL");
    if (!check_grid_desc(gd, &why)) return fail(nullptr, PSC_ERR_ARG, why);
    if (obs->n_ant < 2 || obs->n_ant > 512) return fail(nullptr, PSC_ERR_ARG, "n_ant must be in [2, 512]");
    if (obs->n_time < 1) return fail(nullptr, PSC_ERR_ARG, "n_time must be >= 1");
    if (obs->n_chan < 1 || obs->n_chan > 4096) return fail(nullptr, PSC_ERR_ARG, "n_chan must be in [1, 4096]");
    if (!obs->uvw_dev || !obs->freq_hz || !grid_dev) return fail(nullptr, PSC_ERR_ARG, "uvw, freq and grid must be non-NULL");
    const char *ap_why = nullptr;
    if (!aperture_ok(ap, &ap_why)) return fail(nullptr, PSC_ERR_ARG, ap_why);
    for (int c = 0; c < obs->n_chan; ++c)
        if (!(obs->freq_hz[c] > 0.0) || !std::isfinite(obs->freq_hz[c])) return fail(nullptr, PSC_ERR_ARG, "frequencies must be > 0");

    psc_ctx *c = new psc_ctx();
    c->stream = (cudaStream_t)stream;
    c->n_ant = obs->n_ant;
    c->n_bl = obs->n_ant * (obs->n_ant - 1) / 2;
    c->nt = obs->n_time;
    c->nc = obs->n_chan;
    c->gd = *gd;
    c->ap = *ap;
    c->ap.table = nullptr;                            // the copy on the device replaces the caller's array
    c->du = 1.0 / (gd->n_grid * gd->cell_rad);
    c->uvw = obs->uvw_dev;
    c->grid = (const float2 *)grid_dev;

    // per-channel constants and table layout (host, FP64)
    std::vector<ChanConst> ch(c->nc);
    std::vector<int> off(c->nc), len(c->nc);
    int total = 0;
    const int ov = gd->oversample;
    for (int k = 0; k < c->nc; ++k) {
        const double dl = ap->diam_m * obs->freq_hz[k] / kC;
        const double alpha = ap->alpha_per_dlambda * dl;
        const double rho_max = aperture_reach(ap->kind, dl, c->du, gd->support);
        const int L = (int)std::floor(ov * rho_max) + 2;
        if (L > (1 << 20)) { free_ctx(c); return fail(nullptr, PSC_ERR_ARG, "aperture table too long: aperture much wider than the grid cell"); }
        ch[k].uv_scale = obs->freq_hz[k] / (kC * c->du);
        ch[k].sc_hi = (float)ch[k].uv_scale;
        ch[k].sc_lo = (float)(ch[k].uv_scale - (double)ch[k].sc_hi);
        ch[k].alpha2 = (float)(alpha * alpha);
        ch[k].rho_max = (float)((double)(L - 1) / ov);
        ch[k].tab_off = total;
        ch[k].tab_len = L;
        off[k] = total;
        len[k] = L;
        total += L;
        if (L > c->max_tab_len) c->max_tab_len = L;
    }
    c->h_freq.assign(obs->freq_hz, obs->freq_hz + c->nc);
    c->h_tab_off = off;
    c->h_tab_len = len;
    std::vector<int2> pairs;
    pairs.reserve(c->n_bl);
    for (int i = 0; i < c->n_ant; ++i)
        for (int j = i + 1; j < c->n_ant; ++j) pairs.push_back(make_int2(i, j));

    double *d_freq = nullptr;
    int *d_off = nullptr, *d_len = nullptr;
    unsigned *d_step = nullptr;
    unsigned h_step = 0;
    const size_t evn = ev_len(c->n_ant, c->n_bl);
    const int n2 = 2 * c->n_ant;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&c->d_chan, c->nc);
    if (e == cudaSuccess) e = dalloc(&c->d_tabs, total);
    if (e == cudaSuccess) e = dalloc(&c->d_pairs, c->n_bl);
    if (e == cudaSuccess) e = dalloc(&c->d_blsum, (size_t)c->n_bl * kRed);
    if (e == cudaSuccess) e = dalloc(&c->d_ev, evn);
    if (e == cudaSuccess) e = dalloc(&c->d_cur, evn);
    if (e == cudaSuccess) e = dalloc(&c->d_lm_trial, n2);
    if (e == cudaSuccess) e = dalloc(&c->d_lm_cur, n2);
    if (e == cudaSuccess) e = dalloc(&c->d_mat, (size_t)n2 * n2);
    if (e == cudaSuccess) e = dalloc(&c->d_mat32, (size_t)n2 * n2);
    if (e == cudaSuccess) e = dalloc(&c->d_rhs, n2);
    if (e == cudaSuccess) e = dalloc(&c->d_state, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_state0, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_lm0, n2);
    if (e == cudaSuccess) e = dalloc(&c->d_err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = dalloc(&d_freq, c->nc);
    if (e == cudaSuccess) e = dalloc(&d_off, c->nc);
    if (e == cudaSuccess) e = dalloc(&d_len, c->nc);
    if (e == cudaSuccess) e = dalloc(&d_step, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_uvs, (size_t)c->nt * c->n_bl);
    if (e == cudaSuccess) e = launch_split_uv(c->uvw, (size_t)c->nt * c->n_bl, c->d_uvs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_step, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = launch_step_max(c->uvw, c->nt, c->n_bl, d_step, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_step, d_step, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_chan, ch.data(), sizeof(ChanConst) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_pairs, pairs.data(), sizeof(int2) * c->n_bl, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_freq, obs->freq_hz, sizeof(double) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, len.data(), sizeof(int) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && ap->kind == PSC_AP_TABLE) {
        e = dalloc(&c->d_aptab, ap->table_len);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_aptab, ap->table, sizeof(double) * ap->table_len, cudaMemcpyHostToDevice, c->stream);
    }
    if (e == cudaSuccess)
        e = launch_tables(*ap, c->d_aptab, d_freq, c->nc, c->du, ov, gd->support, d_off, d_len, c->d_tabs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_state, 0, sizeof(LMState), c->stream);
    // baselines in Morton (Z) order of their (u, v) at the middle time step, for
    // PSC_ORDER_UV: bricks launched together then read nearby grid cells
    std::vector<double> mid((size_t)c->n_bl * 3);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mid.data(), c->uvw + (size_t)(c->nt / 2) * c->n_bl * 3, sizeof(double) * mid.size(),
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = dalloc(&c->d_bl_order, c->n_bl);
    if (e == cudaSuccess) {
        double span = 0.0;
        for (int b = 0; b < c->n_bl; ++b) span = std::max(span, std::max(std::fabs(mid[3 * b]), std::fabs(mid[3 * b + 1])));
        std::vector<std::pair<uint32_t, int>> key(c->n_bl);
        for (int b = 0; b < c->n_bl; ++b) {
            auto q = [&](double x) { return (uint32_t)std::min(1023.0, std::max(0.0, (x / (span > 0 ? span : 1.0) * 0.5 + 0.5) * 1024.0)); };
            const uint32_t qu = q(mid[3 * b]), qv = q(mid[3 * b + 1]);
            uint32_t z = 0;
            for (int bit = 0; bit < 10; ++bit) z |= (((qu >> bit) & 1u) << (2 * bit)) | (((qv >> bit) & 1u) << (2 * bit + 1));
            key[b] = {z, b};
        }
        std::sort(key.begin(), key.end());
        std::vector<int> order(c->n_bl);
        for (int b = 0; b < c->n_bl; ++b) order[b] = key[b].second;
        e = cudaMemcpyAsync(c->d_bl_order, order.data(), sizeof(int) * c->n_bl, cudaMemcpyHostToDevice, c->stream);
        // default: locality order when the grid is larger than L2 (128 MB)
        if ((size_t)gd->n_grid * gd->n_grid * sizeof(float2) > ((size_t)128 << 20)) c->brick_order = PSC_ORDER_UV;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_freq);
    cudaFree(d_off);
    cudaFree(d_len);
    cudaFree(d_step);
    if (e != cudaSuccess) {
        psc_status st = cuda_fail(nullptr, e, "psc_create");
        free_ctx(c);
        return st;
    }
    c->d_done = &c->d_state->done;
    c->h_ev.resize(evn);
    {
        float step_m = 0.f;
        std::memcpy(&step_m, &h_step, sizeof(float));
        double sc_max = 0.0, rho_top = 0.0;
        for (int k = 0; k < c->nc; ++k) {
            sc_max = std::max(sc_max, ch[k].uv_scale);
            rho_top = std::max(rho_top, (double)(len[k] - 1) / ov);
        }
        c->step_cells = (double)step_m * sc_max;
        c->multi_ok = std::isfinite(c->step_cells) && rho_top <= 0.5 * gd->support - 1.0;
    }
    // room for the tables of the widest channel group, and the LM layouts
    int stride_max = tab_stride(c, 1);
    if (kv_allowed(c, 2)) stride_max = std::max(stride_max, tab_stride(c, 2));
    e = set_eval_smem(eval_dyn_smem(8, stride_max));
    if (e == cudaSuccess) e = lm_prepare(c->n_ant);
    if (e != cudaSuccess) { psc_status st = cuda_fail(nullptr, e, "psc_create: shared memory"); free_ctx(c); return st; }
    *out = c;
    return PSC_OK;
}

void psc_destroy(psc_ctx *ctx) { free_ctx(ctx); }

psc_status psc_set_tiling(psc_ctx *ctx, int t_tile, int c_group, int vis_per_thread) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    const int tt = t_tile ? t_tile : ctx->t_tile;
    const int cg = c_group ? c_group : ctx->c_group;
    const int kv = vis_per_thread ? vis_per_thread : ctx->kv;
    if (!(kv == 1 || kv == 2)) return fail(ctx, PSC_ERR_ARG, "vis_per_thread must be 1 or 2");
    if (kv != 1 && ctx->kernel_model == PSC_KERNEL_EXACT_DISK)
        return fail(ctx, PSC_ERR_ARG, "the exact disk kernel takes one visibility per thread");
    if (!kv_allowed(ctx, kv))
        return fail(ctx, PSC_ERR_ARG, "vis_per_thread 2 needs the aperture inside the S x S window and "
                                      "consecutive time steps within 4 cells");
    if (tt < 1 || tt > kMaxThreads) return fail(ctx, PSC_ERR_ARG, "t_tile must be in [1, 256]");
    if (cg < 1 || cg > 8) return fail(ctx, PSC_ERR_ARG, "c_group must be in [1, 8]");
    if (tt * cg > kMaxThreads) return fail(ctx, PSC_ERR_ARG, "t_tile * c_group must be <= 256");
    ctx->t_tile = tt;
    ctx->c_group = cg;
    ctx->kv = kv;
    ctx->flat = 0;
    ctx->trk_kv = 0;
    return PSC_OK;
}

psc_status psc_set_flat_tiling(psc_ctx *ctx, int items, int vis_per_thread) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (ctx->kernel_model != PSC_KERNEL_GAUSS && vis_per_thread != 1)
        return fail(ctx, PSC_ERR_ARG, "the exact disk kernel takes one visibility per thread");
    if (items < 32 || items > kMaxThreads || items % 32) return fail(ctx, PSC_ERR_ARG, "items must be 32, 64, ..., 256");
    if (!(vis_per_thread == 1 || vis_per_thread == 2)) return fail(ctx, PSC_ERR_ARG, "vis_per_thread must be 1 or 2");
    if (!kv_allowed(ctx, vis_per_thread))
        return fail(ctx, PSC_ERR_ARG, "vis_per_thread 2 needs the aperture inside the S x S window and "
                                      "consecutive time steps within 4 cells");
    const int old_kv = ctx->kv, old_flat = ctx->flat;
    ctx->kv = vis_per_thread;
    ctx->flat = items;
    if (ch_span(ctx) > 8) {
        ctx->kv = old_kv;
        ctx->flat = old_flat;
        return fail(ctx, PSC_ERR_ARG, "a brick would span more than 8 channels (too few time steps per channel)");
    }
    ctx->trk_kv = 0;
    return PSC_OK;
}

psc_status psc_set_track_tiling(psc_ctx *ctx, int vis_per_lane) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (vis_per_lane == 0) {
        ctx->trk_kv = 0;
        return PSC_OK;
    }
    const std::string why = trk_refusal(ctx, vis_per_lane);
    if (!why.empty()) return fail(ctx, PSC_ERR_ARG, why);
    psc_status st = trk_prepare(ctx);
    if (st != PSC_OK) return st;
    ctx->trk_kv = vis_per_lane;
    return PSC_OK;
}

psc_status psc_set_kernel_model(psc_ctx *ctx, int model) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (model == PSC_KERNEL_GAUSS) {
        ctx->kernel_model = model;
        return PSC_OK;
    }
    if (model != PSC_KERNEL_EXACT_DISK) return fail(ctx, PSC_ERR_ARG, "model must be PSC_KERNEL_GAUSS or PSC_KERNEL_EXACT_DISK");
    if (ctx->wp_n > 0) return fail(ctx, PSC_ERR_ARG, "the exact kernel does not read a residual-w stack");
    if (ctx->ap.kind != PSC_AP_DISK) return fail(ctx, PSC_ERR_ARG, "the exact kernel needs a uniform-disk aperture");
    int dev = 0, optin = 0;
    PSC_CUDA(ctx, cudaGetDevice(&dev));
    PSC_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (exact_dyn_smem(1, ctx->max_tab_len + 2) + (size_t)kTile * kTile * sizeof(float2) + 4096 > (size_t)optin)
        return fail(ctx, PSC_ERR_ARG, "aperture table too long for the exact kernel's shared memory");
    if (!ctx->d_kmom) {
        const int nc = ctx->nc;
        const size_t total = (size_t)ctx->h_tab_off[nc - 1] + ctx->h_tab_len[nc - 1];
        double *d_freq = nullptr;
        int *d_off = nullptr, *d_len = nullptr;
        cudaError_t e = dalloc(&ctx->d_kmom, total * 10);
        if (e == cudaSuccess) e = dalloc(&d_freq, nc);
        if (e == cudaSuccess) e = dalloc(&d_off, nc);
        if (e == cudaSuccess) e = dalloc(&d_len, nc);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_freq, ctx->h_freq.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, ctx->h_tab_off.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, ctx->h_tab_len.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = launch_exact_moments(ctx->ap.diam_m, d_freq, nc, ctx->du, ctx->gd.oversample, d_off, d_len, ctx->d_kmom,
                                     ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(d_freq);
        cudaFree(d_off);
        cudaFree(d_len);
        if (e != cudaSuccess) {
            cudaFree(ctx->d_kmom);
            ctx->d_kmom = nullptr;
            return cuda_fail(ctx, e, "psc_set_kernel_model");
        }
    }
    ctx->kernel_model = model;
    ctx->kv = 1;
    ctx->flat = 0;
    ctx->trk_kv = 0;
    return PSC_OK;
}

psc_status psc_set_brick_order(psc_ctx *ctx, int order) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (order != PSC_ORDER_BASELINE && order != PSC_ORDER_UV) return fail(ctx, PSC_ERR_ARG, "order must be PSC_ORDER_BASELINE or PSC_ORDER_UV");
    ctx->brick_order = order;
    return PSC_OK;
}

psc_status psc_set_staging(psc_ctx *ctx, int mode) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (mode != PSC_STAGE_AUTO && mode != PSC_STAGE_NEVER) return fail(ctx, PSC_ERR_ARG, "mode must be PSC_STAGE_AUTO or PSC_STAGE_NEVER");
    ctx->no_stage = mode == PSC_STAGE_NEVER;
    return PSC_OK;
}

psc_status psc_set_grid_precision(psc_ctx *ctx, int precision) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (precision == PSC_GRID_F32) {
        PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));     // no launch may still read the copy
        cudaFree(ctx->d_grid_bf16);
        ctx->d_grid_bf16 = nullptr;
        return PSC_OK;
    }
    if (precision != PSC_GRID_BF16) return fail(ctx, PSC_ERR_ARG, "precision must be PSC_GRID_F32 or PSC_GRID_BF16");
    if (ctx->wp_n > 0) return fail(ctx, PSC_ERR_ARG, "a residual-w stack is read in FP32 only");
    const size_t n = (size_t)ctx->gd.n_grid * ctx->gd.n_grid;
    ctx->trk_kv = 0;                                  // the track kernel reads the FP32 grid
    if (!ctx->d_grid_bf16) PSC_CUDA(ctx, dalloc(&ctx->d_grid_bf16, n));
    PSC_CUDA(ctx, launch_grid_to_bf16(ctx->grid, n, ctx->d_grid_bf16, ctx->stream));
    PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PSC_OK;
}

psc_status psc_set_wstack(psc_ctx *ctx, const void *grids, int n_planes, double w0, double dw, double a, double b) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (n_planes == 0) {
        ctx->wp_n = 0;
        ctx->wp_grid = nullptr;
        return PSC_OK;
    }
    if (n_planes < 2 || n_planes > 65536) return fail(ctx, PSC_ERR_ARG, "n_planes must be 0 or in [2, 65536]");
    if (!grids) return fail(ctx, PSC_ERR_ARG, "grids is NULL");
    if (!std::isfinite(w0) || !(dw > 0.0) || !std::isfinite(dw) || !std::isfinite(a) || !std::isfinite(b))
        return fail(ctx, PSC_ERR_ARG, "w0, a, b must be finite and dw > 0");
    if (ctx->kernel_model != PSC_KERNEL_GAUSS) return fail(ctx, PSC_ERR_ARG, "a residual-w stack needs the Gaussian kernel model");
    if (ctx->d_grid_bf16) return fail(ctx, PSC_ERR_ARG, "a residual-w stack is read in FP32 only (grid precision is BF16)");
    // coverage: the residual w of every row, at the lowest and highest channel
    double lo_m = 0.0, hi_m = 0.0;
    psc_status st = psc_wstack_range(ctx->uvw, (long long)ctx->nt * ctx->n_bl, a, b, &lo_m, &hi_m, ctx->stream);
    if (st != PSC_OK) return fail(ctx, st, psc_last_error(nullptr));
    const auto fr = std::minmax_element(ctx->h_freq.begin(), ctx->h_freq.end());
    const double s_lo = *fr.first / kC, s_hi = *fr.second / kC;
    const double w_lo = std::min(lo_m * s_lo, lo_m * s_hi), w_hi = std::max(hi_m * s_lo, hi_m * s_hi);
    if (w_lo < w0 || w_hi > w0 + (n_planes - 1) * dw) {
        char msg[200];
        std::snprintf(msg, sizeof msg, "the stack covers w in [%.6g, %.6g] wavelengths, the context needs [%.6g, %.6g]",
                      w0, w0 + (n_planes - 1) * dw, w_lo, w_hi);
        return fail(ctx, PSC_ERR_ARG, msg);
    }
    ctx->wp_grid = (const float2 *)grids;
    ctx->wp_n = n_planes;
    ctx->trk_kv = 0;                                  // stacks run the brick kernel
    ctx->wp_w0 = w0;
    ctx->wp_dw = dw;
    ctx->wp_a = a;
    ctx->wp_b = b;
    return PSC_OK;
}

psc_status psc_predict(psc_ctx *ctx, const double *lm, void *vis_out, void *dvis_out) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm || !vis_out) return fail(ctx, PSC_ERR_ARG, "lm and vis_out must be non-NULL");
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_trial, lm, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyHostToDevice, ctx->stream));
    const int trk = ctx->trk_kv;                  // predictions always run the brick kernel
    ctx->trk_kv = 0;
    EvalArgs a = eval_args(ctx, ctx->d_lm_trial);
    ctx->trk_kv = trk;
    a.vis_out = (float2 *)vis_out;
    a.dvis_out = (float2 *)dvis_out;
    PSC_CUDA(ctx, launch_eval(a, true, ctx->stream));
    PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PSC_OK;
}

psc_status psc_predict_dev(psc_ctx *ctx, const double *lm_dev, void *vis_out, void *dvis_out) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm_dev || !vis_out) return fail(ctx, PSC_ERR_ARG, "lm_dev and vis_out must be non-NULL");
    const int trk = ctx->trk_kv;                  // predictions always run the brick kernel
    ctx->trk_kv = 0;
    EvalArgs a = eval_args(ctx, lm_dev);
    ctx->trk_kv = trk;
    a.vis_out = (float2 *)vis_out;
    a.dvis_out = (float2 *)dvis_out;
    PSC_CUDA(ctx, launch_eval(a, true, ctx->stream));
    return PSC_OK;
}

psc_status psc_residual_grad(psc_ctx *ctx, const double *lm, const void *vis_obs, const float *w, double w_scale,
                             double *chi2, double *grad, double *normal, double *cross) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm || !vis_obs || !chi2 || !grad || !normal) return fail(ctx, PSC_ERR_ARG, "lm, vis_obs, chi2, grad and normal must be non-NULL");
    if (!(w_scale > 0.0) || !std::isfinite(w_scale)) return fail(ctx, PSC_ERR_ARG, "w_scale must be > 0");
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_trial, lm, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyHostToDevice, ctx->stream));
    psc_status st = eval_reduce(ctx, ctx->d_lm_trial, vis_obs, w, w_scale, ctx->d_ev, nullptr);
    if (st != PSC_OK) return st;
    const size_t evn = ev_len(ctx->n_ant, ctx->n_bl);
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ev.data(), ctx->d_ev, sizeof(double) * evn, cudaMemcpyDeviceToHost, ctx->stream));
    PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    st = check_err_flag(ctx);
    if (st != PSC_OK) return st;
    const int n = ctx->n_ant;
    *chi2 = ctx->h_ev[0];
    std::memcpy(grad, ctx->h_ev.data() + 1, sizeof(double) * 2 * n);
    std::memcpy(normal, ctx->h_ev.data() + 1 + 2 * n, sizeof(double) * 3 * n);
    if (cross) std::memcpy(cross, ctx->h_ev.data() + 1 + 5 * n, sizeof(double) * 4 * ctx->n_bl);
    return PSC_OK;
}

}  // extern "C"

namespace {

psc_status check_opts(psc_ctx *ctx, const psc_solve_opts &o) {
    if (o.max_iter < 0 || (o.mode != PSC_LM_FULL && o.mode != PSC_LM_BLOCK) || !(o.lam0 > 0.0) ||
        !(o.lam_max >= o.lam0) || !(o.lam_min >= 0.0) || !(o.step_tol_rad >= 0.0) || !(o.chi2_rtol >= 0.0) ||
        !(o.block_gain > 0.0 && o.block_gain <= 1.0))
        return fail(ctx, PSC_ERR_ARG, "invalid solver options");
    return PSC_OK;
}

// Uploads the start offsets and the initial solver state of ctx on `s`.
psc_status lm_begin_on(psc_ctx *ctx, const double *lm0, const psc_solve_opts &o, cudaStream_t s) {
    LMState st{};
    st.lam = o.lam0;
    st.chi2 = INFINITY;
    st.max_iter = o.max_iter;
    st.mode = o.mode;
    st.lam_max = o.lam_max;
    st.lam_min = o.lam_min;
    st.step_tol = o.step_tol_rad;
    st.chi2_rtol = o.chi2_rtol;
    st.block_gain = o.block_gain;
    ctx->h_state = st;
    const size_t lmb = sizeof(double) * 2 * ctx->n_ant;
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_state, &ctx->h_state, sizeof(LMState), cudaMemcpyHostToDevice, s));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_trial, lm0, lmb, cudaMemcpyHostToDevice, s));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_cur, lm0, lmb, cudaMemcpyHostToDevice, s));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_state0, &ctx->h_state, sizeof(LMState), cudaMemcpyHostToDevice, s));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm0, lm0, lmb, cudaMemcpyHostToDevice, s));
    ctx->begun = true;
    return PSC_OK;
}

// Copies the accepted offsets and the solver state of ctx to the host
// (after the caller synchronised `s`).
psc_status lm_fetch(psc_ctx *ctx, double *lm_out, psc_solve_report *rep, cudaStream_t s) {
    if (lm_out)
        PSC_CUDA(ctx, cudaMemcpyAsync(lm_out, ctx->d_lm_cur, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyDeviceToHost, s));
    PSC_CUDA(ctx, cudaMemcpyAsync(&ctx->h_state, ctx->d_state, sizeof(LMState), cudaMemcpyDeviceToHost, s));
    int flag = 0;
    PSC_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PSC_CUDA(ctx, cudaStreamSynchronize(s));
    if (flag) {
        PSC_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
        return fail(ctx, PSC_ERR_TIMEOUT, "a bounded wait of the fused evaluation ran out; its results were discarded");
    }
    if (rep) {
        rep->n_iter = ctx->h_state.n_iter;
        rep->n_eval = ctx->h_state.n_eval;
        rep->reason = ctx->h_state.done ? ctx->h_state.reason : PSC_STOP_NONE;
        rep->chi2 = ctx->h_state.chi2;
        rep->lam = ctx->h_state.lam;
    }
    if (ctx->h_state.done && ctx->h_state.reason == PSC_STOP_NUMERIC)
        return fail(ctx, PSC_ERR_NUMERIC, "solver stopped on a non-finite chi^2 or step");
    return PSC_OK;
}

}  // namespace

extern "C" {

psc_status psc_lm_begin(psc_ctx *ctx, const double *lm0, const psc_solve_opts *opts) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm0) return fail(ctx, PSC_ERR_ARG, "lm0 is NULL");
    psc_solve_opts o;
    if (opts) o = *opts;
    else psc_solve_opts_default(&o);
    psc_status st = check_opts(ctx, o);
    if (st != PSC_OK) return st;
    return lm_begin_on(ctx, lm0, o, ctx->stream);
}

psc_status psc_lm_restart(psc_ctx *ctx) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!ctx->begun) return fail(ctx, PSC_ERR_ARG, "psc_lm_restart before psc_lm_begin");
    PSC_CUDA(ctx, launch_lm_restart(lm_args(ctx), ctx->d_state0, ctx->d_lm0, ctx->stream));
    return PSC_OK;
}

psc_status psc_lm_iterate(psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale, int n_iter) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!vis_obs || n_iter < 0) return fail(ctx, PSC_ERR_ARG, "vis_obs must be non-NULL and n_iter >= 0");
    if (!(w_scale > 0.0) || !std::isfinite(w_scale)) return fail(ctx, PSC_ERR_ARG, "w_scale must be > 0");
    const LMArgs la = lm_args(ctx);
    for (int it = 0; it < n_iter; ++it) {
        psc_status st = eval_reduce(ctx, ctx->d_lm_trial, vis_obs, w, w_scale, ctx->d_ev, ctx->d_done);
        if (st != PSC_OK) return st;
        PSC_CUDA(ctx, launch_lm_update(la, ctx->stream));
    }
    return PSC_OK;
}

psc_status psc_lm_end(psc_ctx *ctx, double *lm_out, psc_solve_report *rep) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    return lm_fetch(ctx, lm_out, rep, ctx->stream);
}

psc_status psc_solve_offsets(psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale,
                             const psc_solve_opts *opts, double *lm_inout, psc_solve_report *rep) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm_inout) return fail(ctx, PSC_ERR_ARG, "lm_inout is NULL");
    psc_solve_opts o;
    if (opts) o = *opts;
    else psc_solve_opts_default(&o);
    psc_status st = psc_lm_begin(ctx, lm_inout, &o);
    if (st != PSC_OK) return st;
    // enqueue in chunks and poll the stop flag between chunks
    int done_evals = 0;
    const int total = o.max_iter + 1;
    while (done_evals < total) {
        const int chunk = std::min(4, total - done_evals);
        st = psc_lm_iterate(ctx, vis_obs, w, w_scale, chunk);
        if (st != PSC_OK) return st;
        done_evals += chunk;
        int done = 0;
        PSC_CUDA(ctx, cudaMemcpyAsync(&done, ctx->d_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (done) break;
    }
    return psc_lm_end(ctx, lm_inout, rep);
}

psc_status psc_features(psc_ctx *ctx, const void *vis_obs, const float *w, double w_scale, double sigma_prior_rad,
                        int time_stride, float *feat_dev) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!vis_obs || !feat_dev) return fail(ctx, PSC_ERR_ARG, "vis_obs and feat must be non-NULL");
    if (!(w_scale > 0.0) || !std::isfinite(w_scale)) return fail(ctx, PSC_ERR_ARG, "w_scale must be > 0");
    if (!(sigma_prior_rad > 0.0) || !std::isfinite(sigma_prior_rad)) return fail(ctx, PSC_ERR_ARG, "sigma_prior must be > 0");
    if (time_stride < 1) return fail(ctx, PSC_ERR_ARG, "time_stride must be >= 1");
    StencilArgs a = stencil_args(ctx, vis_obs, w, w_scale, sigma_prior_rad, time_stride);
    const size_t need = (size_t)a.n_bricks * 56;
    if (need > ctx->spart_cap) {
        cudaFree(ctx->d_spart);
        ctx->d_spart = nullptr;
        ctx->spart_cap = 0;
        PSC_CUDA(ctx, dalloc(&ctx->d_spart, need));
        ctx->spart_cap = need;
    }
    if (!ctx->d_sblsum) PSC_CUDA(ctx, dalloc(&ctx->d_sblsum, (size_t)ctx->n_bl * 56));
    a.partials = ctx->d_spart;
    PSC_CUDA(ctx, launch_features(a, ctx->d_sblsum, ctx->n_ant, feat_dev, ctx->stream));
    return PSC_OK;
}

}  // extern "C"

namespace {

size_t al256b(size_t x) { return (x + 255) / 256 * 256; }

// Workspace layout of psc_features_batch: the argument tables, then per pair
// its partials and per-baseline sums.
size_t features_batch_layout(psc_ctx *const *ctxs, int n, int time_stride, std::vector<size_t> *off_part,
                             std::vector<size_t> *off_bl) {
    size_t o = al256b(sizeof(StencilArgs) * n) + al256b(sizeof(long long) * (n + 1)) + al256b(sizeof(FeatPair) * n);
    for (int j = 0; j < n; ++j) {
        const StencilArgs a = stencil_args(ctxs[j], nullptr, nullptr, 1.0, 1.0, time_stride);
        if (off_part) off_part->push_back(o);
        o = al256b(o + sizeof(double) * 56 * (size_t)a.n_bricks);
        if (off_bl) off_bl->push_back(o);
        o = al256b(o + sizeof(double) * 56 * (size_t)ctxs[j]->n_bl);
    }
    return o;
}

}  // namespace

extern "C" {

psc_status psc_features_batch_work(psc_ctx *const *ctxs, int n, int time_stride, size_t *bytes) {
    if (!ctxs || n < 1 || !bytes) return fail(nullptr, PSC_ERR_ARG, "ctxs and bytes must be non-NULL, n >= 1");
    if (time_stride < 1) return fail(nullptr, PSC_ERR_ARG, "time_stride must be >= 1");
    for (int j = 0; j < n; ++j)
        if (!ctxs[j]) return fail(nullptr, PSC_ERR_ARG, "a context is NULL");
    *bytes = features_batch_layout(ctxs, n, time_stride, nullptr, nullptr);
    return PSC_OK;
}

psc_status psc_features_batch(psc_ctx *const *ctxs, int n, const void *const *vis_obs, const float *const *w,
                              const double *w_scale, double sigma_prior_rad, int time_stride, void *work,
                              size_t work_bytes, float *feat_dev, void *stream) {
    if (!ctxs || n < 1 || !vis_obs || !feat_dev || !work) return fail(nullptr, PSC_ERR_ARG, "ctxs, vis_obs, work and feat must be non-NULL, n >= 1");
    if (!(sigma_prior_rad > 0.0) || !std::isfinite(sigma_prior_rad)) return fail(nullptr, PSC_ERR_ARG, "sigma_prior must be > 0");
    if (time_stride < 1) return fail(nullptr, PSC_ERR_ARG, "time_stride must be >= 1");
    for (int j = 0; j < n; ++j) {
        if (!ctxs[j] || !vis_obs[j]) return fail(nullptr, PSC_ERR_ARG, "a context or its vis_obs is NULL");
        const double ws = w_scale ? w_scale[j] : 1.0;
        if (!(ws > 0.0) || !std::isfinite(ws)) return fail(nullptr, PSC_ERR_ARG, "w_scale must be > 0");
    }
    std::vector<size_t> off_part, off_bl;
    const size_t need = features_batch_layout(ctxs, n, time_stride, &off_part, &off_bl);
    if (work_bytes < need) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "psc_features_batch: the workspace holds %zu bytes, %zu needed", work_bytes, need);
        return fail(nullptr, PSC_ERR_ARG, msg);
    }
    unsigned char *base = (unsigned char *)work;
    std::vector<StencilArgs> args(n);
    std::vector<long long> prefix(n + 1, 0);
    std::vector<FeatPair> pairs(n);
    size_t feat_off = 0;
    int threads = 0, max_bl = 0, max_ant = 0;
    size_t dyn = 0;
    for (int j = 0; j < n; ++j) {
        psc_ctx *c = ctxs[j];
        args[j] = stencil_args(c, vis_obs[j], w ? w[j] : nullptr, w_scale ? w_scale[j] : 1.0, sigma_prior_rad, time_stride);
        args[j].partials = (double *)(base + off_part[j]);
        const int th = args[j].wpb > 1 ? 32 * args[j].wpb : (args[j].t_tile * args[j].c_group + 31) / 32 * 32;
        if (j > 0 && (th != threads || args[j].stage != args[0].stage || args[j].wpb != args[0].wpb))
            return fail(nullptr, PSC_ERR_ARG, "psc_features_batch: every pair needs the same brick shape (time steps and channels)");
        threads = th;
        dyn = std::max(dyn, stencil_dyn_smem(args[j].c_group, args[j].max_tab_len, args[j].stage));
        prefix[j + 1] = prefix[j] + (args[j].n_bricks + args[j].wpb - 1) / args[j].wpb;    // blocks
        pairs[j].partials = args[j].partials;
        pairs[j].blsum = (double *)(base + off_bl[j]);
        pairs[j].feat = feat_dev + feat_off;
        pairs[j].n_bl = c->n_bl;
        pairs[j].bpb = args[j].n_cg * args[j].n_tt;
        pairs[j].n_ant = c->n_ant;
        feat_off += (size_t)c->n_ant * 52;
        max_bl = std::max(max_bl, c->n_bl);
        max_ant = std::max(max_ant, c->n_ant);
    }
    cudaStream_t s = (cudaStream_t)stream;
    StencilArgs *d_args = (StencilArgs *)base;
    long long *d_prefix = (long long *)(base + al256b(sizeof(StencilArgs) * n));
    FeatPair *d_pairs = (FeatPair *)(base + al256b(sizeof(StencilArgs) * n) + al256b(sizeof(long long) * (n + 1)));
    cudaError_t e = cudaMemcpyAsync(d_args, args.data(), sizeof(StencilArgs) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_prefix, prefix.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(FeatPair) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_features_batch(d_args, d_prefix, d_pairs, n, prefix[n], threads, dyn, max_bl, max_ant,
                                  (float)sigma_prior_rad, s);
    // the argument tables live in pageable host memory: they must be copied before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_features_batch");
    return PSC_OK;
}

psc_status psc_learned_init(psc_ctx *ctx, psc_mlp *m, const void *vis_obs, const float *w, double w_scale,
                            double sigma_prior_rad, int time_stride, double *lm_out) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!m || !lm_out) return fail(ctx, PSC_ERR_ARG, "mlp and lm_out must be non-NULL");
    if (!ctx->d_feat) PSC_CUDA(ctx, dalloc(&ctx->d_feat, (size_t)ctx->n_ant * 52));
    psc_status st = psc_features(ctx, vis_obs, w, w_scale, sigma_prior_rad, time_stride, ctx->d_feat);
    if (st != PSC_OK) return st;
    st = psc_mlp_infer_offsets(m, ctx->d_feat, ctx->n_ant, sigma_prior_rad, lm_out);
    if (st != PSC_OK) return fail(ctx, st, psc_last_error(nullptr));
    return PSC_OK;
}

psc_status psc_profile(psc_ctx *ctx, int enable) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    ctx->prof = enable != 0;
    return PSC_OK;
}

psc_status psc_profile_read(psc_ctx *ctx, double *total_ms, int *n_launches) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!total_ms || !n_launches) return fail(ctx, PSC_ERR_ARG, "outputs must be non-NULL");
    PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double tot = 0.0;
    for (size_t k = 0; k + 1 < ctx->ev_used; k += 2) {
        float ms = 0.f;
        PSC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[k], ctx->ev_pool[k + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *n_launches = (int)(ctx->ev_used / 2);
    ctx->ev_used = 0;
    return PSC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of contexts: one persistent fused launch per LM iteration.

struct psc_batch {
    cudaStream_t stream = nullptr;
    std::vector<psc_ctx *> ctxs;
    std::vector<const void *> vis;
    std::vector<const float *> w;
    std::vector<double> w_scale;
    // device tables (rebuilt by build_tables)
    EvalArgs *d_eval = nullptr;
    long long *d_prefix = nullptr;
    RedArgs *d_red = nullptr;
    int *d_bl_prefix = nullptr;
    LMArgs *d_lm = nullptr;
    const LMState **d_st0 = nullptr;
    const double **d_lm0 = nullptr;
    unsigned long long *d_queue = nullptr;
    int *d_active = nullptr;
    // psc_batch_end: every context's offsets, solver state and wait flag
    // gathered on the device ([lm 2n_ant...][state...][flag...]) and copied
    // to pinned host memory in one transfer
    unsigned char *d_gather = nullptr, *h_gather = nullptr;
    size_t gather_bytes = 0;
    std::vector<size_t> lm_off;
    int total_bl = 0;
    int grid = 0;
    int threads = 128;           // fused-kernel block size: the widest context's shape
    bool stacked = false;        // every context reads a residual-w stack (else none does)
    int track = 0;               // > 0: the persistent launch runs the track kernel, this many visibilities per lane
    int trk_tabc = 0;            // track kernel: table capacity of a warp buffer (entries)
    size_t eval_dyn = 0, lm_dyn = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // fused-kernel timing (psc_batch_profile): direct launches with event pairs
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::string err;
};

namespace {

psc_status bfail(psc_batch *b, psc_status st, const std::string &msg) {
    if (b) b->err = msg;
    return fail(nullptr, st, msg);
}

#define PSC_BCUDA(b, call)                                                        \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess)                                                    \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? PSC_ERR_OOM : PSC_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

void drop_graph(psc_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

void free_batch(psc_batch *b) {
    if (!b) return;
    drop_graph(b);
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    cudaFree(b->d_eval); cudaFree(b->d_prefix); cudaFree(b->d_red); cudaFree(b->d_bl_prefix);
    cudaFree(b->d_lm); cudaFree(b->d_st0); cudaFree(b->d_lm0); cudaFree(b->d_queue); cudaFree(b->d_active);
    cudaFree(b->d_gather);
    cudaFreeHost(b->h_gather);
    delete b;
}

// (Re)builds the device argument tables from the contexts' current tiling.
psc_status build_tables(psc_batch *b) {
    const int n = (int)b->ctxs.size();
    std::vector<EvalArgs> ev(n);
    std::vector<long long> prefix(n + 1, 0);
    std::vector<RedArgs> red(n);
    std::vector<int> blp(n + 1, 0);
    std::vector<LMArgs> lm(n);
    std::vector<const LMState *> st0(n);
    std::vector<const double *> lm0(n);
    size_t dyn = 0, lmd = 0;
    int threads = 32;
    for (int k = 0; k < n; ++k) {
        psc_ctx *c = b->ctxs[k];
        threads = std::max(threads, eval_threads(c));
        psc_status st = ensure_partials(c);
        if (st != PSC_OK) return bfail(b, st, c->err);
        ev[k] = eval_args(c, c->d_lm_trial);
        ev[k].vis_obs = (const float2 *)b->vis[k];
        ev[k].w = b->w[k];
        ev[k].w_scale = (float)b->w_scale[k];
        ev[k].skip = c->d_done;
        prefix[k + 1] = prefix[k] + ev[k].n_bricks;
        red[k] = red_args(c, c->d_ev, c->d_done);
        blp[k + 1] = blp[k] + c->n_bl;
        lm[k] = lm_args(c);
        st0[k] = c->d_state0;
        lm0[k] = c->d_lm0;
        dyn = std::max(dyn, eval_dyn_smem(ch_span(c), tab_stride(c, c->kv)));
        lmd = std::max(lmd, lm_smem_bytes(c->n_ant));
    }
    b->total_bl = blp[n];
    b->threads = threads;
    b->eval_dyn = dyn;
    b->lm_dyn = lmd;
    // one fused kernel per persistent launch: the track kernel for all
    // contexts (same visibilities per lane) or for none
    int n_trk = 0, kv_trk = 0, tabc = 0;
    for (int k = 0; k < n; ++k) {
        const psc_ctx *c = b->ctxs[k];
        if (c->trk_kv <= 0) continue;
        ++n_trk;
        if (kv_trk && kv_trk != c->trk_kv) kv_trk = -1;
        else if (kv_trk == 0) kv_trk = c->trk_kv;
        tabc = std::max(tabc, ev[k].trk_tabc);
    }
    if (n_trk != 0 && (n_trk != n || kv_trk < 0))
        return bfail(b, PSC_ERR_ARG, "a batch runs one fused kernel: give every context the same track tiling, or none");
    b->track = n_trk ? kv_trk : 0;
    b->trk_tabc = tabc;
    int per_sm = 0, dev = 0, n_sm = 0;
    b->stacked = b->ctxs[0]->wp_n > 0;
    if (b->track) {
        const size_t tdyn = track_dyn_smem(kTrkCap, tabc);
        PSC_BCUDA(b, set_track_smem(tdyn));
        PSC_BCUDA(b, track_occupancy(b->track, tdyn, &per_sm));
    } else {
        PSC_BCUDA(b, set_eval_smem(dyn));
        PSC_BCUDA(b, eval_batch_occupancy(b->threads, dyn, b->stacked, &per_sm));
    }
    PSC_BCUDA(b, cudaGetDevice(&dev));
    PSC_BCUDA(b, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    b->grid = std::max(1, per_sm) * n_sm;
    if (!b->d_eval) {
        PSC_BCUDA(b, dalloc(&b->d_eval, n));
        PSC_BCUDA(b, dalloc(&b->d_prefix, n + 1));
        PSC_BCUDA(b, dalloc(&b->d_red, n));
        PSC_BCUDA(b, dalloc(&b->d_bl_prefix, n + 1));
        PSC_BCUDA(b, dalloc(&b->d_lm, n));
        PSC_BCUDA(b, dalloc(&b->d_st0, n));
        PSC_BCUDA(b, dalloc(&b->d_lm0, n));
        PSC_BCUDA(b, dalloc(&b->d_queue, 1));
        PSC_BCUDA(b, dalloc(&b->d_active, 1));
    }
    cudaStream_t s = b->stream;
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_eval, ev.data(), sizeof(EvalArgs) * n, cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_prefix, prefix.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_red, red.data(), sizeof(RedArgs) * n, cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_bl_prefix, blp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_lm, lm.data(), sizeof(LMArgs) * n, cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_st0, st0.data(), sizeof(void *) * n, cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaMemcpyAsync(b->d_lm0, lm0.data(), sizeof(void *) * n, cudaMemcpyHostToDevice, s));
    PSC_BCUDA(b, cudaStreamSynchronize(s));
    drop_graph(b);
    return PSC_OK;
}

// The batch's persistent fused launch (its work queue already reset).
psc_status launch_fused(psc_batch *b) {
    const int n = (int)b->ctxs.size();
    cudaStream_t s = b->stream;
    if (b->track)
        PSC_BCUDA(b, launch_track_batch(b->d_eval, b->d_prefix, n, b->d_queue, b->track, kTrkCap, b->trk_tabc, b->grid, s));
    else
        PSC_BCUDA(b, launch_eval_batch(b->d_eval, b->d_prefix, n, b->d_queue, b->threads, b->eval_dyn, b->grid,
                                       b->stacked, s));
    return PSC_OK;
}

// One LM iteration of every context: fused persistent launch, reductions, update.
psc_status enqueue_iteration(psc_batch *b) {
    const int n = (int)b->ctxs.size();
    cudaStream_t s = b->stream;
    PSC_BCUDA(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), s));
    if (b->prof) {
        while (b->ev_pool.size() < b->ev_used + 2) {
            cudaEvent_t e;
            PSC_BCUDA(b, cudaEventCreate(&e));
            b->ev_pool.push_back(e);
        }
        PSC_BCUDA(b, cudaEventRecord(b->ev_pool[b->ev_used], s));
    }
    psc_status fst = launch_fused(b);
    if (fst != PSC_OK) return fst;
    if (b->prof) {
        PSC_BCUDA(b, cudaEventRecord(b->ev_pool[b->ev_used + 1], s));
        b->ev_used += 2;
    }
    PSC_BCUDA(b, launch_reduce_batch(b->d_red, b->d_bl_prefix, n, b->total_bl, s));
    PSC_BCUDA(b, launch_lm_update_batch(b->d_lm, n, b->lm_dyn, s));
    return PSC_OK;
}

psc_status ensure_graph(psc_batch *b) {
    if (b->exec) return PSC_OK;
    cudaStream_t s = b->stream;
    if (s == nullptr) return PSC_OK;                 // the legacy stream cannot be captured: launch directly
    PSC_BCUDA(b, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    psc_status st = enqueue_iteration(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != PSC_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return bfail(b, PSC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        drop_graph(b);
        return bfail(b, PSC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return PSC_OK;
}

// psc_batch_end's gather: context k's accepted offsets to lm + lm_off[k],
// its solver state to st[k] and its wait flag to flag[k] (then cleared).
__global__ void batch_gather_kernel(const LMArgs *la, int n, const long long *lm_off, double *lm, LMState *st,
                                    int *flag) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const LMArgs a = la[k];
        for (int i = threadIdx.x; i < 2 * a.n_ant; i += blockDim.x) lm[lm_off[k] + i] = a.lm_cur[i];
        if (threadIdx.x == 0) {
            st[k] = *a.st;
            flag[k] = *a.err;
            *a.err = 0;
        }
    }
}

__global__ void count_active_kernel(const LMArgs *la, int n, int *out) {
    int c = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) c += la[k].st->done ? 0 : 1;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (threadIdx.x == 0) *out = c;
}

// Smallest time tile that covers nt steps in the fewest tiles of at most
// threads / c_group threads per channel.
int fit_t_tile(int nt, int threads, int cg, int kv) {
    const int tt_max = std::max(1, threads / cg);
    const int n_tt = (nt + tt_max * kv - 1) / (tt_max * kv);
    return (nt + n_tt * kv - 1) / (n_tt * kv);
}

// Launch shapes worth timing for a context: for each block size (128 and 256
// threads), vis_per_thread and channel group, the smallest time tile with the
// fewest tiles that fit the block; ranked by the share of the block's lanes
// that hold a visibility (ragged time and channel tails and idle lanes count
// as waste), the best three of each (block size, vis_per_thread).
// A brick shape: {t_tile, c_group, kv, flat} (flat > 0: bricks of `flat`
// consecutive (channel, time-group) items; t_tile and c_group unused).
using Tiling = std::array<int, 4>;

void apply_tiling(psc_ctx *c, const Tiling &t) {
    c->trk_kv = 0;
    if (t[3] > 0) {
        c->flat = t[3];
    } else {
        c->t_tile = t[0];
        c->c_group = t[1];
        c->flat = 0;
    }
    c->kv = t[2];
}

std::vector<Tiling> tiling_candidates(const psc_ctx *c) {
    struct Scored { double util; int threads; Tiling t; };
    std::vector<Scored> all;
    for (int threads : {128, 256}) {
        for (int kv : {1, 2}) {
            if (!kv_allowed(c, kv)) continue;
            for (int cg : {1, 2, 3, 4, 5, 6, 8}) {
                if (cg > c->nc && cg > 1) continue;
                const int tt = fit_t_tile(c->nt, threads, cg, kv);
                const int n_tt = (c->nt + tt * kv - 1) / (tt * kv);
                if ((tt * cg + 31) / 32 * 32 != threads) continue;   // belongs to the smaller block size
                const int n_cg = (c->nc + cg - 1) / cg;
                const double util = (double)c->nt / ((double)n_tt * tt * kv) * (double)c->nc / ((double)n_cg * cg) *
                                    (double)(tt * cg) / threads;
                all.push_back({util, threads, {tt, cg, kv, 0}});
            }
        }
    }
    std::sort(all.begin(), all.end(), [](const Scored &x, const Scored &y) { return x.util > y.util; });
    std::vector<Tiling> out;
    int taken[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (const Scored &x : all) {
        int &n = taken[x.threads == 256][x.t[2]];
        if (n >= 3) continue;
        ++n;
        out.push_back(x.t);
    }
    const Tiling dflt{32, 4, 1, 0};
    if (std::find(out.begin(), out.end(), dflt) == out.end()) out.push_back(dflt);
    // flat bricks: every lane but the last brick's tail holds an item
    for (int items : {64, 128, 192, 256})
        for (int kv : {1, 2}) {
            if (!kv_allowed(c, kv)) continue;
            const int tp = (c->nt + kv - 1) / kv;
            if (std::min(c->nc, (items + tp - 2) / tp + 1) <= 8) out.push_back({0, 0, kv, items});
        }
    return out;
}

}  // namespace

extern "C" {

psc_status psc_batch_create(psc_batch **out, psc_ctx *const *ctxs, int n_ctx, const void *const *vis_obs,
                            const float *const *w, const double *w_scale, void *stream) {
    if (!out) return fail(nullptr, PSC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctxs || n_ctx < 1 || !vis_obs) return fail(nullptr, PSC_ERR_ARG, "ctxs and vis_obs must be non-NULL, n_ctx >= 1");
    psc_batch *b = new psc_batch();
    b->stream = (cudaStream_t)stream;
    for (int k = 0; k < n_ctx; ++k) {
        if (!ctxs[k] || !vis_obs[k]) { free_batch(b); return fail(nullptr, PSC_ERR_ARG, "a context or its vis_obs is NULL"); }
        const double ws = w_scale ? w_scale[k] : 1.0;
        if (!(ws > 0.0) || !std::isfinite(ws)) { free_batch(b); return fail(nullptr, PSC_ERR_ARG, "w_scale must be > 0"); }
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == ctxs[k]) { free_batch(b); return fail(nullptr, PSC_ERR_ARG, "a context appears twice in the batch"); }
        if (ctxs[k]->kernel_model != PSC_KERNEL_GAUSS) {
            free_batch(b);
            return fail(nullptr, PSC_ERR_ARG, "batches take contexts with the Gaussian kernel model only");
        }
        if ((ctxs[k]->wp_n > 0) != (ctxs[0]->wp_n > 0)) {
            free_batch(b);
            return fail(nullptr, PSC_ERR_ARG, "a batch takes either only contexts with a residual-w stack or none");
        }
        b->ctxs.push_back(ctxs[k]);
        b->vis.push_back(vis_obs[k]);
        b->w.push_back(w ? w[k] : nullptr);
        b->w_scale.push_back(ws);
    }
    psc_status st = build_tables(b);
    if (st != PSC_OK) { free_batch(b); return st; }
    st = lm_prepare(0) == cudaSuccess ? PSC_OK : fail(nullptr, PSC_ERR_CUDA, "LM shared memory");
    if (st != PSC_OK) { free_batch(b); return st; }
    *out = b;
    return PSC_OK;
}

void psc_batch_destroy(psc_batch *b) { free_batch(b); }

psc_status psc_batch_autotune(psc_batch *b, int *tiling_out) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    cudaEvent_t e0, e1;
    PSC_BCUDA(b, cudaEventCreate(&e0));
    PSC_BCUDA(b, cudaEventCreate(&e1));
    const int n = (int)b->ctxs.size();
    std::vector<double> zeros;
    std::vector<std::vector<std::pair<float, Tiling>>> timed(n);
    std::vector<int> reused(n, -1);
    auto time_eval = [&](psc_ctx *c, int k, float *ms) -> psc_status {
        psc_status st = ensure_partials(c);
        if (st != PSC_OK) return bfail(b, st, c->err);
        if (c->trk_kv == 0) PSC_BCUDA(b, set_eval_smem(eval_dyn_smem(ch_span(c), tab_stride(c, c->kv))));
        EvalArgs a = eval_args(c, c->d_lm_trial);
        a.vis_obs = (const float2 *)b->vis[k];
        a.w = b->w[k];
        a.w_scale = (float)b->w_scale[k];
        auto launch = [&]() { return a.trk_kv > 0 ? launch_track(a, b->stream) : launch_eval(a, false, b->stream); };
        PSC_BCUDA(b, launch());                                  // warm
        PSC_BCUDA(b, cudaEventRecord(e0, b->stream));
        for (int r = 0; r < 3; ++r) PSC_BCUDA(b, launch());
        PSC_BCUDA(b, cudaEventRecord(e1, b->stream));
        PSC_BCUDA(b, cudaEventSynchronize(e1));
        PSC_BCUDA(b, cudaEventElapsedTime(ms, e0, e1));
        return PSC_OK;
    };
    for (int k = 0; k < n; ++k) {
        psc_ctx *c = b->ctxs[k];
        // contexts of the same array, channels and grid (any length) reuse the
        // first one's choice, refitted to their own number of time steps
        int reuse = -1;
        for (int j = 0; j < k && reuse < 0; ++j) {
            psc_ctx *o = b->ctxs[j];
            if (reused[j] < 0 && o->n_ant == c->n_ant && o->nc == c->nc && o->gd.n_grid == c->gd.n_grid &&
                o->du == c->du && o->max_tab_len == c->max_tab_len && o->multi_ok == c->multi_ok)
                reuse = j;
        }
        reused[k] = reuse;
        if (reuse < 0) {
            zeros.assign(2 * c->n_ant, 0.0);
            PSC_BCUDA(b, cudaMemcpyAsync(c->d_lm_trial, zeros.data(), sizeof(double) * zeros.size(),
                                         cudaMemcpyHostToDevice, b->stream));
            float best = 1e30f;
            Tiling bt{32, 4, 1, 0};
            timed[k].clear();
            c->no_stage = 0;
            for (const Tiling &cd : tiling_candidates(c)) {
                apply_tiling(c, cd);
                float ms = 0.f;
                psc_status st = time_eval(c, k, &ms);
                if (st != PSC_OK) return st;
                timed[k].push_back({ms, cd});
                if (ms < best) { best = ms; bt = cd; }
            }
            apply_tiling(c, bt);
            // and whether staging the grid pays for this shape
            c->no_stage = 1;
            float ms = 0.f;
            psc_status st = time_eval(c, k, &ms);
            if (st != PSC_OK) return st;
            c->no_stage = ms < best ? 1 : 0;
        }
    }
    // one block size serves the whole persistent launch: contexts whose best
    // shape is narrower take their fastest timed shape of the widest size
    int width = 32;
    for (int k = 0; k < n; ++k)
        if (reused[k] < 0) width = std::max(width, eval_threads(b->ctxs[k]));
    for (int k = 0; k < n; ++k) {
        psc_ctx *c = b->ctxs[k];
        c->trk_kv = 0;
        if (reused[k] >= 0) {
            const psc_ctx *o = b->ctxs[reused[k]];
            c->no_stage = o->no_stage;
            c->c_group = o->c_group;
            c->kv = kv_allowed(c, o->kv) ? o->kv : 1;
            c->flat = o->flat;
            if (c->flat > 0 && ch_span(c) > 8) {          // a shorter interval: fall back to the default shape
                c->flat = 0;
                c->c_group = 4;
            }
            if (c->flat == 0)
                c->t_tile = fit_t_tile(c->nt, o->flat > 0 ? o->flat : eval_threads(o), c->c_group, c->kv);
        } else if (eval_threads(c) != width) {
            float best = 1e30f;
            for (const auto &x : timed[k]) {
                const Tiling &t = x.second;
                const int w = ((t[3] > 0 ? t[3] : t[0] * t[1]) + 31) / 32 * 32;
                if (w == width && x.first < best) {
                    best = x.first;
                    apply_tiling(c, t);
                }
            }
        }
        if (tiling_out) {
            tiling_out[4 * k] = c->flat > 0 ? c->flat : c->t_tile;
            tiling_out[4 * k + 1] = c->flat > 0 ? 0 : c->c_group;
            tiling_out[4 * k + 2] = c->kv;
            tiling_out[4 * k + 3] = c->no_stage ? PSC_STAGE_NEVER : PSC_STAGE_AUTO;
        }
    }
    // the fused kernel, chosen on the whole batch: one persistent launch of the
    // brick kernel (the shapes above) and of the track kernel with each
    // visibilities-per-lane that every context allows.  (Single contexts, timed
    // alone, misjudge it: short intervals leave most of the GPU idle.)
    std::vector<int> cands{0};
    for (int kv = 1; kv <= 2; ++kv) {
        bool all = true;
        for (psc_ctx *c : b->ctxs) all = all && trk_refusal(c, kv).empty();
        if (all) cands.push_back(kv);
    }
    int use_trk = 0;
    if (cands.size() > 1) {
        // the timing evaluates every context at zero offsets with its solver
        // running: save each context's trial offsets and state, restore them after
        size_t lm_len = 0;
        for (psc_ctx *c : b->ctxs) lm_len += 2 * (size_t)c->n_ant;
        double *d_lm_save = nullptr;
        LMState *d_st_save = nullptr;
        cudaError_t e = dalloc(&d_lm_save, lm_len);
        if (e == cudaSuccess) e = dalloc(&d_st_save, (size_t)n);
        size_t off = 0;
        for (int k = 0; k < n && e == cudaSuccess; ++k) {
            psc_ctx *c = b->ctxs[k];
            e = cudaMemcpyAsync(d_lm_save + off, c->d_lm_trial, sizeof(double) * 2 * c->n_ant, cudaMemcpyDeviceToDevice, b->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_st_save + k, c->d_state, sizeof(LMState), cudaMemcpyDeviceToDevice, b->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_lm_trial, 0, sizeof(double) * 2 * c->n_ant, b->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_done, 0, sizeof(int), b->stream);
            off += 2 * (size_t)c->n_ant;
        }
        float best = 1e30f;
        psc_status st = PSC_OK;
        for (size_t q = 0; q < cands.size() && e == cudaSuccess && st == PSC_OK; ++q) {
            const int kv = cands[q];
            for (psc_ctx *c : b->ctxs) {
                if (kv > 0) {
                    st = trk_prepare(c);
                    if (st != PSC_OK) break;
                }
                c->trk_kv = kv;
            }
            if (st == PSC_OK) st = build_tables(b);
            if (st != PSC_OK) break;
            float ms = 0.f;
            for (int r = 0; r < 2 && st == PSC_OK; ++r) {             // warm, then timed
                if (r == 1) e = cudaEventRecord(e0, b->stream);
                if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream);
                if (e == cudaSuccess) st = launch_fused(b);
                if (r == 1 && e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            }
            if (e == cudaSuccess && st == PSC_OK) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && st == PSC_OK) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && st == PSC_OK && ms < best) {
                best = ms;
                use_trk = kv;
            }
        }
        off = 0;
        for (int k = 0; k < n && d_lm_save && d_st_save; ++k) {
            psc_ctx *c = b->ctxs[k];
            cudaMemcpyAsync(c->d_lm_trial, d_lm_save + off, sizeof(double) * 2 * c->n_ant, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(c->d_state, d_st_save + k, sizeof(LMState), cudaMemcpyDeviceToDevice, b->stream);
            off += 2 * (size_t)c->n_ant;
        }
        cudaStreamSynchronize(b->stream);
        cudaFree(d_lm_save);
        cudaFree(d_st_save);
        if (st != PSC_OK || e != cudaSuccess) {
            for (psc_ctx *c : b->ctxs) c->trk_kv = 0;       // no context left half-switched
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st != PSC_OK) return st;
            return bfail(b, PSC_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        }
    }
    for (int k = 0; k < n; ++k) {
        psc_ctx *c = b->ctxs[k];
        c->trk_kv = use_trk;
        if (use_trk && tiling_out) {
            tiling_out[4 * k] = -1;
            tiling_out[4 * k + 1] = 0;
            tiling_out[4 * k + 2] = use_trk;
            tiling_out[4 * k + 3] = PSC_STAGE_AUTO;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return build_tables(b);
}

psc_status psc_batch_begin(psc_batch *b, const double *lm0, const psc_solve_opts *opts) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    if (!lm0) return bfail(b, PSC_ERR_ARG, "lm0 is NULL");
    psc_solve_opts o;
    if (opts) o = *opts;
    else psc_solve_opts_default(&o);
    size_t off = 0;
    for (psc_ctx *c : b->ctxs) {
        psc_status st = check_opts(c, o);
        if (st == PSC_OK) st = lm_begin_on(c, lm0 + off, o, b->stream);
        if (st != PSC_OK) return bfail(b, st, c->err);
        off += 2 * (size_t)c->n_ant;
    }
    PSC_BCUDA(b, cudaStreamSynchronize(b->stream));      // the staged host state must not change under the copies
    return PSC_OK;
}

psc_status psc_batch_restart(psc_batch *b) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    for (psc_ctx *c : b->ctxs)
        if (!c->begun) return bfail(b, PSC_ERR_ARG, "psc_batch_restart before psc_batch_begin");
    PSC_BCUDA(b, launch_lm_restart_batch(b->d_lm, b->d_st0, b->d_lm0, (int)b->ctxs.size(), b->stream));
    return PSC_OK;
}

psc_status psc_batch_iterate(psc_batch *b, int n_iter) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    if (n_iter < 0) return bfail(b, PSC_ERR_ARG, "n_iter must be >= 0");
    psc_status st = b->prof ? PSC_OK : ensure_graph(b);
    if (st != PSC_OK) return st;
    for (int it = 0; it < n_iter; ++it) {
        if (b->exec && !b->prof) PSC_BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
        else {
            st = enqueue_iteration(b);
            if (st != PSC_OK) return st;
        }
    }
    return PSC_OK;
}

psc_status psc_batch_end(psc_batch *b, double *lm_out, psc_solve_report *reps) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    const int n = (int)b->ctxs.size();
    if (!b->d_gather) {
        std::vector<long long> off(n);
        size_t tot = 0;
        for (int k = 0; k < n; ++k) {
            off[k] = (long long)tot;
            tot += 2 * (size_t)b->ctxs[k]->n_ant;
        }
        b->lm_off.assign(off.begin(), off.end());
        const size_t o_off = 0, o_lm = (sizeof(long long) * n + 255) / 256 * 256;
        const size_t o_st = (o_lm + sizeof(double) * tot + 255) / 256 * 256;
        const size_t o_fl = (o_st + sizeof(LMState) * n + 255) / 256 * 256;
        b->gather_bytes = o_fl + sizeof(int) * n;
        PSC_BCUDA(b, cudaMalloc(&b->d_gather, b->gather_bytes));
        PSC_BCUDA(b, cudaMallocHost(&b->h_gather, b->gather_bytes));
        PSC_BCUDA(b, cudaMemcpy(b->d_gather + o_off, off.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    }
    const size_t o_lm = (sizeof(long long) * n + 255) / 256 * 256;
    const size_t tot = b->lm_off.back() + 2 * (size_t)b->ctxs[n - 1]->n_ant;
    const size_t o_st = (o_lm + sizeof(double) * tot + 255) / 256 * 256;
    const size_t o_fl = (o_st + sizeof(LMState) * n + 255) / 256 * 256;
    batch_gather_kernel<<<std::min(n, 1024), 64, 0, b->stream>>>(b->d_lm, n, (const long long *)b->d_gather,
                                                                  (double *)(b->d_gather + o_lm),
                                                                  (LMState *)(b->d_gather + o_st),
                                                                  (int *)(b->d_gather + o_fl));
    PSC_BCUDA(b, cudaGetLastError());
    PSC_BCUDA(b, cudaMemcpyAsync(b->h_gather + o_lm, b->d_gather + o_lm, b->gather_bytes - o_lm,
                                 cudaMemcpyDeviceToHost, b->stream));
    PSC_BCUDA(b, cudaStreamSynchronize(b->stream));
    const double *lm = (const double *)(b->h_gather + o_lm);
    const LMState *st = (const LMState *)(b->h_gather + o_st);
    const int *flag = (const int *)(b->h_gather + o_fl);
    if (lm_out) std::memcpy(lm_out, lm, sizeof(double) * tot);
    psc_status worst = PSC_OK;
    for (int k = 0; k < n; ++k) {
        psc_ctx *c = b->ctxs[k];
        c->h_state = st[k];
        if (reps) {
            reps[k].n_iter = st[k].n_iter;
            reps[k].n_eval = st[k].n_eval;
            reps[k].reason = st[k].done ? st[k].reason : PSC_STOP_NONE;
            reps[k].chi2 = st[k].chi2;
            reps[k].lam = st[k].lam;
        }
        psc_status s_k = PSC_OK;
        if (flag[k]) s_k = fail(c, PSC_ERR_TIMEOUT, "a bounded wait of the fused evaluation ran out; its results were discarded");
        else if (st[k].done && st[k].reason == PSC_STOP_NUMERIC)
            s_k = fail(c, PSC_ERR_NUMERIC, "solver stopped on a non-finite chi^2 or step");
        if (s_k != PSC_OK && worst == PSC_OK) { worst = s_k; b->err = c->err; fail(nullptr, s_k, c->err); }
    }
    return worst;
}

psc_status psc_solve_batch(psc_ctx *const *ctxs, int n_ctx, const void *const *vis_obs, const float *const *w,
                           const double *w_scale, const psc_solve_opts *opts, double *lm_inout,
                           psc_solve_report *reps) {
    if (!lm_inout) return fail(nullptr, PSC_ERR_ARG, "lm_inout is NULL");
    if (!ctxs || n_ctx < 1 || !ctxs[0]) return fail(nullptr, PSC_ERR_ARG, "ctxs must be non-NULL, n_ctx >= 1");
    psc_batch *b = nullptr;
    psc_status st = psc_batch_create(&b, ctxs, n_ctx, vis_obs, w, w_scale, ctxs[0]->stream);
    if (st != PSC_OK) return st;
    psc_solve_opts o;
    if (opts) o = *opts;
    else psc_solve_opts_default(&o);
    st = psc_batch_begin(b, lm_inout, &o);
    int active = n_ctx, done_evals = 0;
    const int total = o.max_iter + 1;
    while (st == PSC_OK && active > 0 && done_evals < total) {
        const int chunk = std::min(4, total - done_evals);
        st = psc_batch_iterate(b, chunk);
        done_evals += chunk;
        if (st != PSC_OK) break;
        count_active_kernel<<<1, 32, 0, b->stream>>>(b->d_lm, n_ctx, b->d_active);
        cudaError_t e = cudaMemcpyAsync(&active, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bfail(b, PSC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (st == PSC_OK) st = psc_batch_end(b, lm_inout, reps);
    free_batch(b);
    return st;
}

const char *psc_batch_last_error(const psc_batch *b) { return b ? b->err.c_str() : g_err.c_str(); }

const char *psc_batch_kernel(const psc_batch *b) {
    if (!b) return "";
    if (b->track == 2) return "track_kernel<2>";
    if (b->track == 1) return "track_kernel<1>";
    return b->stacked ? "eval_kernel<false, true>" : "eval_kernel<false, false>";
}

psc_status psc_batch_profile(psc_batch *b, int enable) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    b->prof = enable != 0;
    return PSC_OK;
}

psc_status psc_batch_profile_read(psc_batch *b, double *total_ms, int *n_launches) {
    if (!b) return fail(nullptr, PSC_ERR_ARG, "batch is NULL");
    if (!total_ms || !n_launches) return bfail(b, PSC_ERR_ARG, "outputs must be non-NULL");
    PSC_BCUDA(b, cudaStreamSynchronize(b->stream));
    double tot = 0.0;
    for (size_t k = 0; k + 1 < b->ev_used; k += 2) {
        float ms = 0.f;
        PSC_BCUDA(b, cudaEventElapsedTime(&ms, b->ev_pool[k], b->ev_pool[k + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *n_launches = (int)(b->ev_used / 2);
    b->ev_used = 0;
    return PSC_OK;
}

}  // extern "C"

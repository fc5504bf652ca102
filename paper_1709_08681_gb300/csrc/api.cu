// C ABI of the Pointing SelfCal library (declared in include/psc.h): argument
// checks, context workspace, and the launch sequences of Algorithm 1's
// pre-computes and iteration loop.
#include <cmath>
#include <cstdio>
#include <cstdlib>
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
    LMState h_state{};
    std::vector<double> h_ev;
    std::string err;
    // fused-kernel timing (psc_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

namespace {

thread_local std::string g_err;

psc_status fail(psc_ctx *ctx, psc_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_err = msg;
    return st;
}

}  // namespace

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
    cudaFree(c->d_chan); cudaFree(c->d_tabs); cudaFree(c->d_pairs); cudaFree(c->d_partials);
    cudaFree(c->d_blsum); cudaFree(c->d_ev); cudaFree(c->d_cur); cudaFree(c->d_lm_trial);
    cudaFree(c->d_lm_cur); cudaFree(c->d_mat); cudaFree(c->d_mat32); cudaFree(c->d_rhs); cudaFree(c->d_state);
    cudaFree(c->d_state0); cudaFree(c->d_lm0);
    delete c;
}

int n_tt(const psc_ctx *c) { return (c->nt + c->t_tile - 1) / c->t_tile; }
int n_cg(const psc_ctx *c) { return (c->nc + c->c_group - 1) / c->c_group; }

psc_status ensure_partials(psc_ctx *c) {
    const size_t need = (size_t)c->n_bl * n_cg(c) * n_tt(c);
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
    a.grid = c->grid;
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
    a.n_tt = n_tt(c);
    a.n_cg = n_cg(c);
    a.decorrelation = c->ap.decorrelation;
    a.max_tab_len = c->max_tab_len;
    return a;
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
    PSC_CUDA(c, launch_eval(a, false, c->stream));
    if (c->prof) {
        PSC_CUDA(c, cudaEventRecord(c->ev_pool[c->ev_used + 1], c->stream));
        c->ev_used += 2;
    }
    PSC_CUDA(c, launch_reduce(c->d_partials, c->n_bl, n_cg(c) * n_tt(c), c->d_pairs, c->n_ant, c->d_blsum,
                              ev_out, skip, c->stream));
    return PSC_OK;
}

}  // namespace

extern "C" {

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

psc_status psc_model_grid(const psc_grid_desc *gd, const float *image_dev, void *grid_out, void *stream) {
    std::string why;
    if (!check_grid_desc(gd, &why)) return fail(nullptr, PSC_ERR_ARG, why);
    if (!image_dev || !grid_out) return fail(nullptr, PSC_ERR_ARG, "image and grid pointers must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    float2 *tmp = nullptr, *tw = nullptr;
    cudaError_t e = dalloc(&tmp, (size_t)gd->n_img * gd->n_grid);
    if (e == cudaSuccess) e = dalloc(&tw, (size_t)gd->n_grid);
    if (e == cudaSuccess) e = launch_model_grid(gd->n_img, gd->n_grid, image_dev, tmp, tw, (float2 *)grid_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    cudaFree(tw);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "psc_model_grid");
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
    if (ap->kind != PSC_AP_DISK && ap->kind != PSC_AP_GAUSS) return fail(nullptr, PSC_ERR_ARG, "unknown aperture kind");
    if (!(ap->diam_m > 0.0) || !(ap->alpha_per_dlambda > 0.0)) return fail(nullptr, PSC_ERR_ARG, "diam_m and alpha_per_dlambda must be > 0");
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
        const double rho_max = ap->kind == PSC_AP_DISK ? dl / c->du : 0.5 * gd->support * std::sqrt(2.0);
        const int L = (int)std::floor(ov * rho_max) + 2;
        if (L > (1 << 20)) { free_ctx(c); return fail(nullptr, PSC_ERR_ARG, "aperture table too long: aperture much wider than the grid cell"); }
        ch[k].uv_scale = obs->freq_hz[k] / (kC * c->du);
        ch[k].alpha2 = (float)(alpha * alpha);
        ch[k].rho_max = (float)((double)(L - 1) / ov);
        ch[k].tab_off = total;
        ch[k].tab_len = L;
        off[k] = total;
        len[k] = L;
        total += L;
        if (L > c->max_tab_len) c->max_tab_len = L;
    }
    std::vector<int2> pairs;
    pairs.reserve(c->n_bl);
    for (int i = 0; i < c->n_ant; ++i)
        for (int j = i + 1; j < c->n_ant; ++j) pairs.push_back(make_int2(i, j));

    double *d_freq = nullptr;
    int *d_off = nullptr, *d_len = nullptr;
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
    if (e == cudaSuccess) e = dalloc(&d_freq, c->nc);
    if (e == cudaSuccess) e = dalloc(&d_off, c->nc);
    if (e == cudaSuccess) e = dalloc(&d_len, c->nc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_chan, ch.data(), sizeof(ChanConst) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_pairs, pairs.data(), sizeof(int2) * c->n_bl, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_freq, obs->freq_hz, sizeof(double) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, len.data(), sizeof(int) * c->nc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_tables(*ap, d_freq, c->nc, c->du, ov, gd->support, d_off, d_len, c->d_tabs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_state, 0, sizeof(LMState), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_freq);
    cudaFree(d_off);
    cudaFree(d_len);
    if (e != cudaSuccess) {
        psc_status st = cuda_fail(nullptr, e, "psc_create");
        free_ctx(c);
        return st;
    }
    c->d_done = &c->d_state->done;
    c->h_ev.resize(evn);
    // room for the tables of the widest channel group, and the LM layouts
    e = set_eval_smem(eval_dyn_smem(8, c->max_tab_len));
    if (e == cudaSuccess) e = lm_prepare(c->n_ant);
    if (e != cudaSuccess) { psc_status st = cuda_fail(nullptr, e, "psc_create: shared memory"); free_ctx(c); return st; }
    *out = c;
    return PSC_OK;
}

void psc_destroy(psc_ctx *ctx) { free_ctx(ctx); }

psc_status psc_set_tiling(psc_ctx *ctx, int t_tile, int c_group) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    const int tt = t_tile ? t_tile : ctx->t_tile;
    const int cg = c_group ? c_group : ctx->c_group;
    if (!(tt == 8 || tt == 16 || tt == 32)) return fail(ctx, PSC_ERR_ARG, "t_tile must be 8, 16 or 32");
    if (!(cg == 1 || cg == 2 || cg == 4 || cg == 8)) return fail(ctx, PSC_ERR_ARG, "c_group must be 1, 2, 4 or 8");
    if (tt * cg < 32 || tt * cg > kMaxThreads) return fail(ctx, PSC_ERR_ARG, "t_tile * c_group must be in [32, 256]");
    ctx->t_tile = tt;
    ctx->c_group = cg;
    return PSC_OK;
}

psc_status psc_predict(psc_ctx *ctx, const double *lm, void *vis_out, void *dvis_out) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm || !vis_out) return fail(ctx, PSC_ERR_ARG, "lm and vis_out must be non-NULL");
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_trial, lm, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyHostToDevice, ctx->stream));
    EvalArgs a = eval_args(ctx, ctx->d_lm_trial);
    a.vis_out = (float2 *)vis_out;
    a.dvis_out = (float2 *)dvis_out;
    PSC_CUDA(ctx, launch_eval(a, true, ctx->stream));
    PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
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
    const int n = ctx->n_ant;
    *chi2 = ctx->h_ev[0];
    std::memcpy(grad, ctx->h_ev.data() + 1, sizeof(double) * 2 * n);
    std::memcpy(normal, ctx->h_ev.data() + 1 + 2 * n, sizeof(double) * 3 * n);
    if (cross) std::memcpy(cross, ctx->h_ev.data() + 1 + 5 * n, sizeof(double) * 4 * ctx->n_bl);
    return PSC_OK;
}

psc_status psc_lm_begin(psc_ctx *ctx, const double *lm0, const psc_solve_opts *opts) {
    if (!ctx) return fail(nullptr, PSC_ERR_ARG, "ctx is NULL");
    if (!lm0) return fail(ctx, PSC_ERR_ARG, "lm0 is NULL");
    psc_solve_opts o;
    if (opts) o = *opts;
    else psc_solve_opts_default(&o);
    if (o.max_iter < 0 || (o.mode != PSC_LM_FULL && o.mode != PSC_LM_BLOCK) || !(o.lam0 > 0.0) ||
        !(o.lam_max >= o.lam0) || !(o.lam_min >= 0.0) || !(o.step_tol_rad >= 0.0) || !(o.chi2_rtol >= 0.0) ||
        !(o.block_gain > 0.0 && o.block_gain <= 1.0))
        return fail(ctx, PSC_ERR_ARG, "invalid solver options");
    LMState s{};
    s.lam = o.lam0;
    s.chi2 = INFINITY;
    s.max_iter = o.max_iter;
    s.mode = o.mode;
    s.lam_max = o.lam_max;
    s.lam_min = o.lam_min;
    s.step_tol = o.step_tol_rad;
    s.chi2_rtol = o.chi2_rtol;
    s.block_gain = o.block_gain;
    ctx->h_state = s;
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_state, &ctx->h_state, sizeof(LMState), cudaMemcpyHostToDevice, ctx->stream));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_trial, lm0, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyHostToDevice, ctx->stream));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm_cur, lm0, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyHostToDevice, ctx->stream));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_state0, &ctx->h_state, sizeof(LMState), cudaMemcpyHostToDevice, ctx->stream));
    PSC_CUDA(ctx, cudaMemcpyAsync(ctx->d_lm0, lm0, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyHostToDevice, ctx->stream));
    ctx->begun = true;
    return PSC_OK;
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
    if (lm_out)
        PSC_CUDA(ctx, cudaMemcpyAsync(lm_out, ctx->d_lm_cur, sizeof(double) * 2 * ctx->n_ant, cudaMemcpyDeviceToHost, ctx->stream));
    PSC_CUDA(ctx, cudaMemcpyAsync(&ctx->h_state, ctx->d_state, sizeof(LMState), cudaMemcpyDeviceToHost, ctx->stream));
    PSC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
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

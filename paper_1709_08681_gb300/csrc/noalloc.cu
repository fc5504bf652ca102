// psc_residual_grad_noalloc: the fused evaluation of psc_residual_grad for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc.  Their device memory may belong to
// another allocator, such as a framework's caching pool or an arena sized once
// at start-up.  Or they run in a real-time loop where cudaMalloc and cudaFree,
// which can synchronise the whole device, are not acceptable.  This entry
// point needs no psc_ctx and allocates nothing.  All of its working memory
// lives in one file-scope device array of kScratchBytes (16 MiB), which every
// GPU that loads the library holds until the process exits: channel
// constants, A° tables (and a caller's aperture table), antenna pairs, the
// FP32 split of the baseline coordinates, per-brick partial sums,
// per-baseline sums and the packed result.  The caller still passes every input and output.
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device; that call also raises the fused kernel's
// shared-memory limit on the device.  Every call shares the array: each call
// rewrites every scratch word that it reads, so no clearing is needed, and
// calls that overlap on the GPU (two streams, or two host threads) race on it.
// The kernels, their inputs and their launch shape are the ones
// psc_residual_grad uses with its default tiling, so the results are the same
// bit for bit.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices] = {};
size_t g_smem_allowed[kMaxDevices] = {};      // fused kernel's dynamic shared memory on each device

// Channel constants, table layout and antenna pairs, computed on the device
// from the channel frequencies (one block).
__global__ void noalloc_setup_kernel(const double *freq, int nc, double du, int kind, double diam_m,
                                     double alpha_per_dl, int ov, int support, ChanConst *chan, int *tab_off,
                                     int *tab_len, int n_ant, int2 *pairs) {
    if (threadIdx.x == 0) {
        int total = 0;
        for (int c = 0; c < nc; ++c) {
            const double dl = diam_m * freq[c] / kC;
            const double alpha = alpha_per_dl * dl;
            const double rho_max = kind == PSC_AP_GAUSS ? 0.5 * support * sqrt(2.0) : dl / du;
            const int L = (int)floor(ov * rho_max) + 2;
            ChanConst ch;
            ch.uv_scale = freq[c] / (kC * du);
            ch.sc_hi = (float)ch.uv_scale;
            ch.sc_lo = (float)(ch.uv_scale - (double)ch.sc_hi);
            ch.alpha2 = (float)(alpha * alpha);
            ch.rho_max = (float)((double)(L - 1) / ov);
            ch.tab_off = total;
            ch.tab_len = L;
            chan[c] = ch;
            tab_off[c] = total;
            tab_len[c] = L;
            total += L;
        }
    }
    for (int i = threadIdx.x; i < n_ant; i += blockDim.x) {
        const int base = i * (2 * n_ant - i - 1) / 2;
        for (int j = i + 1; j < n_ant; ++j) pairs[base + j - i - 1] = make_int2(i, j);
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

psc_status fail_arg(const char *msg) { return set_global_error(PSC_ERR_ARG, msg); }

psc_status fail_cuda(cudaError_t e, const char *what) {
    static thread_local char buf[256];
    snprintf(buf, sizeof buf, "psc_residual_grad_noalloc: %s: %s", what, cudaGetErrorString(e));
    return set_global_error(e == cudaErrorMemoryAllocation ? PSC_ERR_OOM : PSC_ERR_CUDA, buf);
}

}  // namespace
}  // namespace psc

using namespace psc;

extern "C" psc_status psc_residual_grad_noalloc(const psc_obs *obs, const psc_aperture *ap, const psc_grid_desc *gd,
                                                const void *grid_dev, const double *lm, const void *vis_obs,
                                                const float *w, double w_scale, double *chi2, double *grad,
                                                double *normal, double *cross, void *stream) {
    if (!obs || !ap || !gd) return fail_arg("psc_residual_grad_noalloc: obs, aperture and grid descriptor must be non-NULL");
    if (!grid_dev || !lm || !vis_obs || !chi2 || !grad || !normal || !obs->uvw_dev || !obs->freq_hz)
        return fail_arg("psc_residual_grad_noalloc: grid, uvw, freq, lm, vis_obs, chi2, grad and normal must be non-NULL");
    if (gd->n_img < 2 || gd->n_img > 8192 || gd->n_img % 2 || gd->n_grid < gd->n_img || gd->n_grid > 16384 ||
        gd->n_grid % 2 || !(gd->cell_rad > 0.0) || gd->support < 2 || gd->support > 64 || gd->support % 2 ||
        gd->oversample < 1 || gd->oversample > 64)
        return fail_arg("psc_residual_grad_noalloc: invalid grid descriptor");
    if (obs->n_ant < 2 || obs->n_ant > 512 || obs->n_time < 1 || obs->n_chan < 1 || obs->n_chan > 4096)
        return fail_arg("psc_residual_grad_noalloc: n_ant, n_time or n_chan out of range");
    const char *ap_why = nullptr;
    if (!aperture_ok(ap, &ap_why)) return fail_arg("psc_residual_grad_noalloc: invalid aperture");
    if (!(w_scale > 0.0) || !std::isfinite(w_scale)) return fail_arg("psc_residual_grad_noalloc: w_scale must be > 0");

    const int n_ant = obs->n_ant, nc = obs->n_chan, nt = obs->n_time;
    const int n_bl = n_ant * (n_ant - 1) / 2;
    const double du = 1.0 / (gd->n_grid * gd->cell_rad);
    const int ov = gd->oversample;
    int total_tab = 0, max_tab = 0;
    for (int c = 0; c < nc; ++c) {
        const double f = obs->freq_hz[c];
        if (!(f > 0.0) || !std::isfinite(f)) return fail_arg("psc_residual_grad_noalloc: frequencies must be > 0");
        const double dl = ap->diam_m * f / kC;
        const double rho_max = aperture_reach(ap->kind, dl, du, gd->support);
        const double Ld = std::floor(ov * rho_max) + 2;
        if (Ld > (1 << 20)) return fail_arg("psc_residual_grad_noalloc: aperture table too long");
        const int L = (int)Ld;
        total_tab += L;
        if (L > max_tab) max_tab = L;
    }
    const int t_tile = 32, c_group = 4;
    const int n_tt = (nt + t_tile - 1) / t_tile, n_cg = (nc + c_group - 1) / c_group;
    const size_t n_bricks = (size_t)n_bl * n_cg * n_tt;
    const size_t evn = ev_len(n_ant, n_bl);

    // scratch layout (256-byte aligned sections)
    size_t off = 0;
    const size_t o_freq = off;  off = align256(off + sizeof(double) * nc);
    const size_t o_chan = off;  off = align256(off + sizeof(ChanConst) * nc);
    const size_t o_toff = off;  off = align256(off + sizeof(int) * nc);
    const size_t o_tlen = off;  off = align256(off + sizeof(int) * nc);
    const size_t o_tabs = off;  off = align256(off + sizeof(float2) * (size_t)total_tab);
    const size_t o_aptb = off;  off = align256(off + (ap->kind == PSC_AP_TABLE ? sizeof(double) * ap->table_len : 0));
    const size_t o_pair = off;  off = align256(off + sizeof(int2) * (size_t)n_bl);
    const size_t o_uvs = off;   off = align256(off + sizeof(float4) * (size_t)nt * n_bl);
    const size_t o_part = off;  off = align256(off + sizeof(double) * kRed * n_bricks);
    const size_t o_blsm = off;  off = align256(off + sizeof(double) * kRed * (size_t)n_bl);
    const size_t o_ev = off;    off = align256(off + sizeof(double) * evn);
    const size_t o_lm = off;    off = align256(off + sizeof(double) * 2 * (size_t)n_ant);
    if (off > kScratchBytes) {
        static thread_local char buf[200];
        snprintf(buf, sizeof buf,
                 "psc_residual_grad_noalloc: this problem needs %zu bytes of scratch; the allocation-free entry "
                 "point holds at most %zu (use psc_residual_grad)", off, kScratchBytes);
        return set_global_error(PSC_ERR_ARG, buf);
    }

    // once per device, with that device current: the array's device address,
    // and the fused kernel's shared-memory limit raised to what the device allows
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail_arg("psc_residual_grad_noalloc: device ordinal beyond 63");
    unsigned char *base = nullptr;
    size_t smem_allowed = 0;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress");
            size_t allowed = 0;
            e = eval_smem_allowed(&allowed);
            if (e != cudaSuccess) return fail_cuda(e, "shared-memory limit");
            e = set_eval_smem(0);
            if (e != cudaSuccess) return fail_cuda(e, "shared-memory limit");
            g_smem_allowed[dev] = allowed;
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
        smem_allowed = g_smem_allowed[dev];
    }
    // the tables of one channel group must fit the block's shared memory; checked
    // before any work is queued
    if (eval_dyn_smem(c_group, max_tab + 2) > smem_allowed)
        return fail_arg("psc_residual_grad_noalloc: the aperture tables of 4 channels exceed the fused kernel's "
                        "shared memory (aperture much wider than the grid cell)");

    cudaStream_t s = (cudaStream_t)stream;
    double *d_freq = (double *)(base + o_freq);
    ChanConst *d_chan = (ChanConst *)(base + o_chan);
    int *d_toff = (int *)(base + o_toff), *d_tlen = (int *)(base + o_tlen);
    float2 *d_tabs = (float2 *)(base + o_tabs);
    int2 *d_pairs = (int2 *)(base + o_pair);
    float4 *d_uvs = (float4 *)(base + o_uvs);
    double *d_part = (double *)(base + o_part), *d_blsum = (double *)(base + o_blsm);
    double *d_ev = (double *)(base + o_ev), *d_lm = (double *)(base + o_lm);

#define NA_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call); \
    } while (0)

    NA_CUDA(cudaMemcpyAsync(d_freq, obs->freq_hz, sizeof(double) * nc, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_lm, lm, sizeof(double) * 2 * n_ant, cudaMemcpyHostToDevice, s));
    noalloc_setup_kernel<<<1, 256, 0, s>>>(d_freq, nc, du, ap->kind, ap->diam_m, ap->alpha_per_dlambda, ov,
                                           gd->support, d_chan, d_toff, d_tlen, n_ant, d_pairs);
    NA_CUDA(cudaGetLastError());
    double *d_aptb = (double *)(base + o_aptb);
    if (ap->kind == PSC_AP_TABLE)
        NA_CUDA(cudaMemcpyAsync(d_aptb, ap->table, sizeof(double) * ap->table_len, cudaMemcpyHostToDevice, s));
    NA_CUDA(launch_tables(*ap, d_aptb, d_freq, nc, du, ov, gd->support, d_toff, d_tlen, d_tabs, s));
    NA_CUDA(launch_split_uv(obs->uvw_dev, (size_t)nt * n_bl, d_uvs, s));

    EvalArgs a{};
    a.uvw = obs->uvw_dev;
    a.uvs = d_uvs;
    a.grid = (const float2 *)grid_dev;
    a.chan = d_chan;
    a.tabs = d_tabs;
    a.pairs = d_pairs;
    a.lm = d_lm;
    a.vis_obs = (const float2 *)vis_obs;
    a.w = w;
    a.w_scale = (float)w_scale;
    a.partials = d_part;
    a.n_bl = n_bl;
    a.nt = nt;
    a.nc = nc;
    a.ng = gd->n_grid;
    a.support = gd->support;
    a.ov = ov;
    a.du = (float)du;
    a.t_tile = t_tile;
    a.c_group = c_group;
    a.n_tt = n_tt;
    a.n_cg = n_cg;
    a.kv = 1;
    a.no_stage = 0;
    a.decorrelation = ap->decorrelation;
    a.max_tab_len = max_tab;
    a.tab_stride = max_tab + 2;              // the table and two zero entries
    a.n_bricks = (long long)n_bricks;
    RedArgs r{};
    r.partials = d_part;
    r.blsum = d_blsum;
    r.ev = d_ev;
    r.skip = nullptr;
    r.n_bl = n_bl;
    r.bpb = n_cg * n_tt;
    r.n_ant = n_ant;
    NA_CUDA(launch_eval(a, false, s));
    NA_CUDA(launch_reduce(r, s));
    NA_CUDA(cudaMemcpyAsync(chi2, d_ev, sizeof(double), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaMemcpyAsync(grad, d_ev + 1, sizeof(double) * 2 * n_ant, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaMemcpyAsync(normal, d_ev + 1 + 2 * n_ant, sizeof(double) * 3 * n_ant, cudaMemcpyDeviceToHost, s));
    if (cross)
        NA_CUDA(cudaMemcpyAsync(cross, d_ev + 1 + 5 * n_ant, sizeof(double) * 4 * n_bl, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
#undef NA_CUDA
    return PSC_OK;
}

// Input features of the learned initial estimate (not part of the paper; an
// addition to the method): per antenna i, the block Newton step at zero
// offsets and a 5 x 5 trial-offset stencil, all from one pass over the time
// steps t with t % stride == 0.  For trial offset
// delta_s = sigma (a, b), a, b in -2..2, on antenna i alone:
//   A_i(s) = sum w Re(conj(V_obs) V_s) / sum w |V_s|^2
//   C_i(s) = (chi2_i(delta_s) - chi2_i(0)) / sum w |V_0|^2,
// sums over the baselines of i and over time steps t with t % stride == 0.
// V_s is the model of Eq. AIJPOINTING with l_i + l_j = delta and
// |l_i - l_j| = |delta|, which is the same whichever end of a baseline carries
// delta, so one stencil evaluation per baseline serves both antennas.
//
// Stencil kernel: bricks as in the fused evaluation, but the staged grid tile
// is not rotated.  All 25 ramps exp(i pi du sigma (dx a + dy b)) are built
// from per-tap and per-row phasors z_x, z_y and their squares, so one A° table
// lookup per tap serves the 25 trial offsets: per row R_a = sum A G z_x^a
// (a = -2..2), then V[b][a] += R_a z_y^b.  The centre point also carries the
// derivative sums of Eq. DAIJPOINTING at zero offsets (dV/dl = i pi Tu,
// dV/dm = i pi Tv, the same for both antennas there).  Per visibility it
// returns X_s = w Re(conj(V_obs) D_s V_s), Y_s = w |D_s V_s|^2,
// Z = w |V_obs|^2, and the gradient (g_l, g_m) and Gauss-Newton block
// (H_ll, H_lm, H_mm) terms of Eqs. Chisq / DCHIDD at zero offsets.
#include <climits>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kTabPad = 2;
constexpr int kSRed = 56;                 // X[25], Y[25], Z, g_l, g_m, H_ll, H_lm, H_mm

__device__ __forceinline__ float rsqrt_fast(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 lds_f2(unsigned addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// One brick of the stencil pass (s_tab: dynamic shared memory).
__device__ __forceinline__ void stencil_brick(const StencilArgs &a, int blk, float2 *s_tab) {
    float2 *s_tile = s_tab + a.c_group * (a.max_tab_len + kTabPad);
    __shared__ int s_boxes[4][4];                 // one box per warp: wpb <= 4 (128 threads)
    __shared__ double s_red[4][kSRed];

    // block blk runs brick blk, or (a.wpb > 1) bricks blk wpb + w, one per warp w,
    // which share the block's channel group and so its tables
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool wb = a.wpb > 1;
    const long long brick_ll = wb ? (long long)blk * a.wpb + (tid >> 5) : blk;
    const bool brick_ok = brick_ll < a.n_bricks;
    const int brick = brick_ok ? (int)brick_ll : 0;
    const int bt = wb ? lane : tid;               // the thread within its brick
    int *s_box = s_boxes[wb ? tid >> 5 : 0];
    const int tt = brick % a.n_tt;
    const int cgi = (brick / a.n_tt) % a.n_cg;
    const int bl = brick / (a.n_tt * a.n_cg);
    const int lt = bt % a.t_tile;
    const int lc = bt / a.t_tile;
    const int t = (tt * a.t_tile + lt) * a.time_stride;
    const int c = cgi * a.c_group + lc;
    const bool valid = brick_ok && lc < a.c_group && t < a.nt && c < a.nc;
    const int tab_stride = a.max_tab_len + kTabPad;

    if (bt == 0) { s_box[0] = INT_MAX; s_box[1] = INT_MIN; s_box[2] = INT_MAX; s_box[3] = INT_MIN; }
    __syncthreads();
    int ix0 = 0, iy0 = 0;
    float fx = 0.f, fy = 0.f;
    if (valid) {
        const double *p = a.uvw + ((size_t)t * a.n_bl + bl) * 3;
        const double sc = a.chan[c].uv_scale;
        const double x = p[0] * sc + 0.5 * a.ng;
        const double y = p[1] * sc + 0.5 * a.ng;
        const double flx = floor(x), fly = floor(y);
        fx = (float)(x - flx);
        fy = (float)(y - fly);
        ix0 = (int)flx - a.support / 2 + 1;
        iy0 = (int)fly - a.support / 2 + 1;
        // staged box: the cells within rho_max of the visibility, inside its window
        const float rm = a.chan[c].rho_max;
        const float hx0 = fx + (float)(a.support / 2 - 1), hy0 = fy + (float)(a.support / 2 - 1);
        const int lox = ix0 + max(0, (int)floorf(hx0 - rm) + 1);
        const int hix = ix0 + min(a.support - 1, (int)ceilf(hx0 + rm) - 1);
        const int loy = iy0 + max(0, (int)floorf(hy0 - rm) + 1);
        const int hiy = iy0 + min(a.support - 1, (int)ceilf(hy0 + rm) - 1);
        if (lox <= hix && loy <= hiy) {
            atomicMin(&s_box[0], lox); atomicMax(&s_box[1], hix);
            atomicMin(&s_box[2], loy); atomicMax(&s_box[3], hiy);
        }
    }
    for (int j = 0; j < a.c_group; ++j) {
        const int cc = cgi * a.c_group + j;
        const int off = cc < a.nc ? a.chan[cc].tab_off : 0;
        const int len = cc < a.nc ? a.chan[cc].tab_len : 0;
        for (int n = tid; n < tab_stride; n += blockDim.x)
            s_tab[j * tab_stride + n] = n < len ? a.tabs[off + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const bool empty = s_box[0] > s_box[1];
    const int bx0 = empty ? 0 : s_box[0], by0 = empty ? 0 : s_box[2];
    const int ex = empty ? 0 : s_box[1] - bx0 + 1, ey = empty ? 0 : s_box[3] - by0 + 1;
    const bool staged = a.stage && ex <= kTile && ey <= kTile;
    if (staged && !empty) {
        const int cshift = blockDim.x >= kTile ? 6 : 5;
        const int cols = 1 << cshift;
        const int rstep = blockDim.x >> cshift;
        for (int xx = tid & (cols - 1); xx < ex; xx += cols) {
            const int gx = bx0 + xx;
            const bool xin = gx >= 0 && gx < a.ng;
            for (int yy = tid >> cshift; yy < ey; yy += rstep) {
                const int gy = by0 + yy;
                float2 g = make_float2(0.f, 0.f);
                if (xin && gy >= 0 && gy < a.ng) g = __ldg(&a.grid[(size_t)gy * a.ng + gx]);
                s_tile[yy * kTile + xx] = g;
            }
        }
    }
    __syncthreads();

    float vr[25], vi[25];
#pragma unroll
    for (int s = 0; s < 25; ++s) { vr[s] = 0.f; vi[s] = 0.f; }
    float sur = 0.f, sui = 0.f, svr = 0.f, svi = 0.f;    // centre-point derivative sums
    const float hx = fx + (float)(a.support / 2 - 1);
    const float hy = fy + (float)(a.support / 2 - 1);
    const float ph = a.du * a.sigma;                     // phase per cell per unit of a (units of pi)
    if (valid) {
        const ChanConst ch = a.chan[c];
        const float2 *tab = s_tab + lc * tab_stride;
        const unsigned tab_adj = (unsigned)__cvta_generic_to_shared(tab) - (0x4B000000u << 3);
        const float ov = (float)a.ov;
        const float rmax = ch.rho_max;
        const float rmax2 = rmax * rmax;
        const int b_lo = max(0, (int)floorf(hy - rmax) + 1);
        const int b_hi = min(a.support - 1, (int)ceilf(hy + rmax) - 1);
        float stp_s, stp_c;
        sincospif(-ph, &stp_s, &stp_c);                  // z_x step per tap
        for (int b = b_lo; b <= b_hi; ++b) {
            const float dy = hy - (float)b;
            const float rem = rmax2 - dy * dy;
            if (!(rem > 0.f)) continue;
            const float r = fminf(rem * rsqrt_fast(rem), rmax);     // keeps the span inside the staged box
            const int a_lo = max(0, (int)floorf(hx - r) + 1);
            const int a_hi = min(a.support - 1, (int)ceilf(hx + r) - 1);
            const float dyo = dy * ov;
            const float dyo2 = fmaf(dyo, dyo, 1e-20f);
            float dxo = (hx - (float)a_lo) * ov;
            float zr, zi;
            sincospif(ph * (hx - (float)a_lo), &zi, &zr);
            float Rr[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Ri[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float qr = 0.f, qi = 0.f;
            for (int aa = a_lo; aa <= a_hi; ++aa) {
                float2 g;
                if (staged) {
                    g = s_tile[(iy0 - by0 + b) * kTile + (ix0 - bx0 + aa)];
                } else {
                    const int gx = ix0 + aa, gy = iy0 + b;
                    g = make_float2(0.f, 0.f);
                    if (gx >= 0 && gx < a.ng && gy >= 0 && gy < a.ng) g = __ldg(&a.grid[(size_t)gy * a.ng + gx]);
                }
                const float s2 = fmaf(dxo, dxo, dyo2);
                const float tv = s2 * rsqrt_fast(s2);
                const float tf = __fadd_rz(tv, 8388608.0f);
                const float2 e = lds_f2(tab_adj + ((unsigned)__float_as_int(tf) << 3));
                const float A = fmaf(tv - (tf - 8388608.0f), e.y, e.x);
                const float pr = A * g.x, pim = A * g.y;
                const float Ad = A * dxo;
                qr = fmaf(Ad, g.x, qr);
                qi = fmaf(Ad, g.y, qi);
                const float z2r = zr * zr - zi * zi, z2i = 2.f * zr * zi;
                Rr[2] += pr; Ri[2] += pim;
                // p z and p conj(z), p z^2 and p conj(z^2)
                const float a1 = pr * zr, a2 = pim * zi, a3 = pr * zi, a4 = pim * zr;
                Rr[3] += a1 - a2; Ri[3] += a3 + a4;
                Rr[1] += a1 + a2; Ri[1] += a4 - a3;
                const float c1 = pr * z2r, c2 = pim * z2i, c3 = pr * z2i, c4 = pim * z2r;
                Rr[4] += c1 - c2; Ri[4] += c3 + c4;
                Rr[0] += c1 + c2; Ri[0] += c4 - c3;
                const float nzr = zr * stp_c - zi * stp_s;
                zi = zr * stp_s + zi * stp_c;
                zr = nzr;
                dxo -= ov;
            }
            sur += qr;
            sui += qi;
            svr = fmaf(dy, Rr[2], svr);
            svi = fmaf(dy, Ri[2], svi);
            float yr, yi;
            sincospif(ph * dy, &yi, &yr);
            const float y2r = yr * yr - yi * yi, y2i = 2.f * yr * yi;
            // z_y^b for b = -2..2: conj(z^2), conj(z), 1, z, z^2
            const float pbr[5] = {y2r, yr, 1.f, yr, y2r};
            const float pbi[5] = {-y2i, -yi, 0.f, yi, y2i};
#pragma unroll
            for (int bb = 0; bb < 5; ++bb) {
#pragma unroll
                for (int aa = 0; aa < 5; ++aa) {
                    const int sidx = bb * 5 + aa;
                    vr[sidx] += Rr[aa] * pbr[bb] - Ri[aa] * pbi[bb];
                    vi[sidx] += Rr[aa] * pbi[bb] + Ri[aa] * pbr[bb];
                }
            }
        }
    }

    float acc[kSRed];
#pragma unroll
    for (int k = 0; k < kSRed; ++k) acc[k] = 0.f;
    if (valid) {
        const size_t k = ((size_t)t * a.n_bl + bl) * a.nc + c;
        const float2 vo = a.vis_obs[k];
        const float w = a.w_scale * (a.w != nullptr ? a.w[k] : 1.f);
        const float al2s2 = a.chan[c].alpha2 * a.sigma * a.sigma;
#pragma unroll
        for (int bb = 0; bb < 5; ++bb) {
#pragma unroll
            for (int aa = 0; aa < 5; ++aa) {
                const int sidx = bb * 5 + aa;
                const float ia = (float)(aa - 2), ib = (float)(bb - 2);
                const float D = a.decorrelation ? expf(-0.5f * al2s2 * (ia * ia + ib * ib)) : 1.f;
                const float xr = D * vr[sidx], xi = D * vi[sidx];
                acc[sidx] = w * (vo.x * xr + vo.y * xi);
                acc[25 + sidx] = w * (xr * xr + xi * xi);
            }
        }
        acc[50] = w * (vo.x * vo.x + vo.y * vo.y);
        // zero offsets: V_0 = centre sum, dV/dl = i pi du Su, dV/dm = i pi du Sv
        const float pi_du = 3.14159265358979f * a.du;
        const float inv_ov = 1.0f / (float)a.ov;
        const float2 dl = make_float2(-pi_du * sui * inv_ov, pi_du * sur * inv_ov);
        const float2 dm = make_float2(-pi_du * svi, pi_du * svr);
        const float2 R = make_float2(vo.x - vr[12], vo.y - vi[12]);
        const float w2 = 2.f * w;
        acc[51] = -w2 * (R.x * dl.x + R.y * dl.y);
        acc[52] = -w2 * (R.x * dm.x + R.y * dm.y);
        acc[53] = w2 * (dl.x * dl.x + dl.y * dl.y);
        acc[54] = w2 * (dl.x * dm.x + dl.y * dm.y);
        acc[55] = w2 * (dm.x * dm.x + dm.y * dm.y);
    }
#pragma unroll
    for (int k = 0; k < kSRed; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[k] = v;
    }
    if (wb) {
        // the warp is the brick: its sums are the record
        if (brick_ok) {
#pragma unroll
            for (int k = 0; k < kSRed; ++k)
                if (lane == (k & 31)) a.partials[(size_t)k * a.n_bricks + brick] = (double)acc[k];
        }
        return;
    }
    const int warp = tid >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kSRed; ++k) s_red[warp][k] = (double)acc[k];
    }
    __syncthreads();
    // kSRed sums may outnumber the threads of a small block
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = tid; k < kSRed; k += blockDim.x) {
        double sum = 0.0;
        for (int wi = 0; wi < nw; ++wi) sum += s_red[wi][k];
        a.partials[(size_t)k * a.n_bricks + brick] = sum;
    }
}

__global__ void __launch_bounds__(128) stencil_kernel(const StencilArgs a) {
    extern __shared__ float2 s_tab[];                 // tables, then the staged tile when a.stage
    stencil_brick(a, blockIdx.x, s_tab);
}

// Many (context, data) pairs in one launch: block b runs block b - prefix[p]
// of pair p (prefix counts blocks), the last pair with prefix[p] <= b.  Every
// pair has the same block shape (t_tile, c_group, bricks per block) and staging.
__global__ void __launch_bounds__(128) stencil_batch_kernel(const StencilArgs *__restrict__ args,
                                                            const long long *__restrict__ prefix, int n) {
    extern __shared__ float2 s_tab[];
    __shared__ StencilArgs s_a;
    __shared__ int s_brick;
    if (threadIdx.x == 0) {
        const long long b = blockIdx.x;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
        }
        s_a = args[lo];
        s_brick = (int)(b - prefix[lo]);
    }
    __syncthreads();
    stencil_brick(s_a, s_brick, s_tab);
}

// Per-baseline sums of the stencil partials: one thread per (sum, baseline),
// bricks added in order (deterministic).
__device__ __forceinline__ void stencil_bl(const double *__restrict__ partials, int n_bl, int bpb,
                                           double *__restrict__ blsum, long long id) {
    if (id >= (long long)n_bl * kSRed) return;
    const int k = (int)(id / n_bl), bl = (int)(id % n_bl);
    const size_t nb = (size_t)n_bl * bpb;
    const double *p = partials + (size_t)k * nb + (size_t)bl * bpb;
    double sum = 0.0;
    for (int b = 0; b < bpb; ++b) sum += p[b];
    blsum[(size_t)bl * kSRed + k] = sum;
}

__global__ void stencil_bl_kernel(const double *__restrict__ partials, int n_bl, int bpb, double *__restrict__ blsum) {
    stencil_bl(partials, n_bl, bpb, blsum, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Batched: blockIdx.y is the pair.
__global__ void stencil_bl_batch_kernel(const FeatPair *__restrict__ pairs) {
    const FeatPair p = pairs[blockIdx.y];
    stencil_bl(p.partials, p.n_bl, p.bpb, p.blsum, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Features of one antenna per block: thread k < kSRed sums value k over the
// antenna's baselines (partners in increasing order), then the block Newton
// step and the 25 stencil ratios and chi^2 changes.
__device__ __forceinline__ void antenna_features(const double *__restrict__ blsum, int n_ant, float sigma,
                                                 float *__restrict__ feat, int an) {
    __shared__ double v[kSRed];
    const int k = threadIdx.x;
    if (k < kSRed) {
        double sum = 0.0;
        for (int o = 0; o < n_ant; ++o) {
            if (o == an) continue;
            const int i = min(an, o), j = max(an, o);
            const int bl = i * (2 * n_ant - i - 1) / 2 + (j - i - 1);
            sum += blsum[(size_t)bl * kSRed + k];
        }
        v[k] = sum;
    }
    __syncthreads();
    float *f = feat + (size_t)an * 52;
    const double *X = v, *Y = v + 25;
    const double Z = v[50], g0 = v[51], g1 = v[52], H0 = v[53], H1 = v[54], H2 = v[55];
    if (k == 0) {
        const double det = H0 * H2 - H1 * H1;
        float s0 = 0.f, s1 = 0.f;
        if (det > 0.0 && H0 > 0.0) {
            s0 = (float)(-(H2 * g0 - H1 * g1) / det / sigma);
            s1 = (float)(-(-H1 * g0 + H0 * g1) / det / sigma);
        }
        f[0] = s0;
        f[1] = s1;
    }
    if (k < 25) {
        const double chi0 = Z - 2.0 * X[12] + Y[12];
        f[2 + k] = Y[k] > 0.0 ? (float)(X[k] / Y[k]) : 0.f;
        f[27 + k] = Y[12] > 0.0 ? (float)((Z - 2.0 * X[k] + Y[k] - chi0) / Y[12]) : 0.f;
    }
}

__global__ void features_kernel(const double *__restrict__ blsum, int n_ant, float sigma, float *__restrict__ feat) {
    antenna_features(blsum, n_ant, sigma, feat, blockIdx.x);
}

// Batched: blockIdx.y is the pair, blockIdx.x the antenna (blocks past the
// pair's antennas return).
__global__ void features_batch_kernel(const FeatPair *__restrict__ pairs, float sigma) {
    const FeatPair p = pairs[blockIdx.y];
    if ((int)blockIdx.x >= p.n_ant) return;
    antenna_features(p.blsum, p.n_ant, sigma, p.feat, blockIdx.x);
}

}  // namespace

size_t stencil_dyn_smem(int c_group, int max_tab_len, int stage) {
    return sizeof(float2) * ((size_t)c_group * (max_tab_len + kTabPad) + (stage ? (size_t)kTile * kTile : 0));
}

cudaError_t launch_features_batch(const StencilArgs *args_dev, const long long *prefix_dev, const FeatPair *pairs_dev,
                                  int n, long long total_blocks, int threads, size_t dyn, int max_bl, int max_ant,
                                  float sigma, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(stencil_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(dyn > 48 * 1024 ? dyn : 48 * 1024));
    if (e != cudaSuccess) return e;
    if (total_blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    stencil_batch_kernel<<<(unsigned)total_blocks, threads, dyn, s>>>(args_dev, prefix_dev, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n_sum = (long long)max_bl * kSRed;
    stencil_bl_batch_kernel<<<dim3((unsigned)((n_sum + 255) / 256), n), 256, 0, s>>>(pairs_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    features_batch_kernel<<<dim3(max_ant, n), 64, 0, s>>>(pairs_dev, sigma);
    return cudaGetLastError();
}

cudaError_t launch_features(const StencilArgs &a, double *blsum, int n_ant, float *feat, cudaStream_t s) {
    const size_t dyn = stencil_dyn_smem(a.c_group, a.max_tab_len, a.stage);
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(dyn > 48 * 1024 ? dyn : 48 * 1024));
    if (e != cudaSuccess) return e;
    const int threads = a.wpb > 1 ? 32 * a.wpb : (a.t_tile * a.c_group + 31) / 32 * 32;
    stencil_kernel<<<(int)((a.n_bricks + a.wpb - 1) / a.wpb), threads, dyn, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n_sum = (long long)a.n_bl * kSRed;
    stencil_bl_kernel<<<(int)((n_sum + 255) / 256), 256, 0, s>>>(a.partials, a.n_bl, a.n_cg * a.n_tt, blsum);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    features_kernel<<<n_ant, 64, 0, s>>>(blsum, n_ant, a.sigma, feat);
    return cudaGetLastError();
}

}  // namespace psc

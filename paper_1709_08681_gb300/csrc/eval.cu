// Fused evaluation kernel of the Pointing SelfCal hot path (sm_103a):
// degridding with the pointing-modified aperture kernel, the four pointing
// derivatives, the residual against the observed visibilities and the
// per-baseline sums of chi^2, gradient and Gauss-Newton normals.
//
// Paper basis (Bhatnagar & Cornwell 2017): Algorithm 1's inner loop; the
// kernel A_ij of Eq. AIJPOINTING and its derivative of Eq. DAIJPOINTING
// (extended to m, Sec. 3); chi^2 of Eq. Chisq and its gradient, Eq. DCHIDD.
//
// Work decomposition.  One thread block handles one "brick": a baseline
// (i, j), a group of c_group channels and t_tile * kv consecutive time steps.
// Each thread owns kv visibilities of one channel at consecutive times; they
// sit within a fraction of a grid cell of each other (the uv track moves
// slowly), so the thread walks the union of their tap rows and loads each
// grid cell once for all kv of them.  The block stages the grid cells its
// visibilities touch (the bounding box of their aperture disks) in shared
// memory.  The kernel's ramp factorises, exp(i pi (u_k - u_g) L) =
// exp(i pi (u_k - u_o) L) exp(-i pi (u_g - u_o) L) for any origin u_o, so the
// staged cells are pre-multiplied by the second factor (per cell, once per
// block) and each visibility applies the first factor once; the inner loop
// over taps then needs only the real radial A° and five FMAs per tap.  Taps
// outside the aperture's support are not visited, or read zero table entries
// (the tables are zero-padded far enough for every tap a thread visits).  If
// a brick's footprint does not fit the staging tile, the block falls back to
// reading the grid from global memory with the ramp applied per tap (same
// arithmetic, slower).
//
// Inner loop per tap and visibility (rho in units of table samples, t = rho
// ov): s2 = dxo^2 + dyo^2 (dxo = dx ov; dyo^2 carries a 1e-20 floor so s2 > 0),
// t = sqrt(s2) (hardware approximation, ~1 ulp), n = floor(t) by a round-toward-zero add of 2^23 whose bit
// pattern also gives the table address, A° = c_n + t s_n with the staged entry
// (c_n, s_n) = (A°(n) - n s_n, A°(n+1) - A°(n)) (the linear interpolation
// A°(n) + (t - n) s_n rearranged), then P += A° G', Q += (A° dxo) G' (each a
// packed FP32x2 FMA over the real and imaginary parts).
#include <algorithm>
#include <climits>

#include <cuda_bf16.h>

#include "psc_internal.cuh"
#include "tap_math.cuh"

namespace psc {
namespace {

using namespace tap;


// Grid cell (gy, gx) as FP32: from the bfloat16 copy when there is one
// (the widening is exact), else from the complex64 grid.
__device__ __forceinline__ float2 grid_cell(const EvalArgs &a, size_t idx) {
    if (a.grid_bf16 != nullptr) {
        const unsigned u = __ldg(&a.grid_bf16[idx]);
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
    }
    return __ldg(&a.grid[idx]);
}

// Shared memory of one block besides the dynamic tables; the staging tile only
// in instantiations that stage.
template <bool kTiled>
struct BlockSharedT {
    float2 tile[kTiled ? kTile * kTile : 1];
    float2 phx[kTile], phy[kTile];
    float red[kMaxThreads / 32][kRed];
    float red_c[kMaxThreads / 32][5];      // rounding errors of the compensated warp sums
    float bl[4];
    int box[4];
    int taps;          // taps of the brick's visibilities (pi rho_max^2 each, rounded up)
};

// One brick: kv visibilities per thread.  acc receives the thread's 15 sums
// (reduce mode); predict mode writes V and the derivative planes.
// kW: the grid is a residual-w stack (EvalArgs::wp_n); every tap reads the two
// planes around its visibility's w and interpolates, unstaged.
template <bool kPredict, int kV, bool kW>
__device__ __forceinline__ void eval_brick(const EvalArgs &a, int brick, float2 *s_tab, BlockSharedT<!kW> &sh,
                                           float (&acc)[kRed]) {
    const int tid = threadIdx.x;
    // brick -> baseline, this thread's channel c and first time step t0, and
    // the block's channels [c_first, c_first + n_ch) (lc = c - c_first)
    int bl, c, t0, c_first, n_ch;
    bool active;
    if (a.flat > 0) {
        bl = brick / a.bpb;
        const int first = (brick - bl * a.bpb) * a.flat;
        const int k = first + tid;
        c = k / a.n_tp;
        t0 = (k - c * a.n_tp) * kV;
        c_first = first / a.n_tp;
        n_ch = min(a.nc - 1, (first + a.flat - 1) / a.n_tp) - c_first + 1;
        active = tid < a.flat && c < a.nc;
    } else {
        const int tt = brick % a.n_tt;
        const int cgi = (brick / a.n_tt) % a.n_cg;
        bl = brick / (a.n_tt * a.n_cg);
        const int lt = tid % a.t_tile;
        const int lcg = tid / a.t_tile;
        t0 = (tt * a.t_tile + lt) * kV;
        c_first = cgi * a.c_group;
        c = c_first + lcg;
        n_ch = a.c_group;
        active = lcg < a.c_group && t0 < a.nt && c < a.nc;
    }
    const int lc = c - c_first;
    const int tab_stride = a.tab_stride;
    const int S = a.support;

    // per-baseline constants, computed once per block in FP64
    if (tid == 0) {
        const int2 ij = a.pairs[bl];
        const double li = a.lm[2 * ij.x], mi = a.lm[2 * ij.x + 1];
        const double lj = a.lm[2 * ij.y], mj = a.lm[2 * ij.y + 1];
        sh.bl[0] = (float)(li + lj);   // ramp: l_i + l_j
        sh.bl[1] = (float)(mi + mj);
        sh.bl[2] = (float)(li - lj);   // decorrelation: l_i - l_j
        sh.bl[3] = (float)(mi - mj);
        sh.box[0] = INT_MAX; sh.box[1] = INT_MIN; sh.box[2] = INT_MAX; sh.box[3] = INT_MIN;
        sh.taps = 0;
    }
    __syncthreads();
    const float L = sh.bl[0], M = sh.bl[1], dL = sh.bl[2], dM = sh.bl[3];

    // Grid position of each visibility: x = u / du + Ng/2 (cells), window
    // origin floor(x) - S/2 + 1, hx = x - origin.  Times past the end of the
    // interval repeat the last one (computed, never stored), so every tap the
    // thread visits stays within its table padding.
    int ix0[kV], iy0[kV];
    float hx[kV], hy[kV];
    float rmax = 0.f;
    size_t woff[kV];                                  // kW: first cell of the lower plane
    float wf[kV];                                     // kW: weight of the upper plane
    if (active) {
        const ChanConst ch = a.chan[c];
        rmax = ch.rho_max;
        int lox = INT_MAX, hix = INT_MIN, loy = INT_MAX, hiy = INT_MIN;
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int t = min(t0 + v, a.nt - 1);
            int nx, ny;
            float fx, fy;
            if (a.uvs != nullptr) {
                const float4 q = a.uvs[(size_t)t * a.n_bl + bl];
                const float half = 0.5f * (float)a.ng;
                grid_pos(q.x, q.y, ch.sc_hi, ch.sc_lo, half, nx, fx);
                grid_pos(q.z, q.w, ch.sc_hi, ch.sc_lo, half, ny, fy);
            } else {
                const double *p = a.uvw + ((size_t)t * a.n_bl + bl) * 3;
                const double x = p[0] * ch.uv_scale + 0.5 * a.ng;
                const double y = p[1] * ch.uv_scale + 0.5 * a.ng;
                const double flx = floor(x), fly = floor(y);
                nx = (int)flx;
                ny = (int)fly;
                fx = (float)(x - flx);
                fy = (float)(y - fly);
            }
            if constexpr (kW) {
                const double *p = a.uvw + ((size_t)t * a.n_bl + bl) * 3;
                double q = (p[2] - a.wp_a * p[0] - a.wp_b * p[1]) * ch.uv_scale * a.wp_scale - a.wp_q0;
                q = fmin(fmax(q, 0.0), (double)(a.wp_n - 1));
                const int pl = min((int)floor(q), a.wp_n - 2);
                woff[v] = (size_t)pl * a.ng * a.ng;
                wf[v] = (float)(q - (double)pl);
            }
            ix0[v] = nx - S / 2 + 1;
            iy0[v] = ny - S / 2 + 1;
            hx[v] = fx + (float)(S / 2 - 1);
            hy[v] = fy + (float)(S / 2 - 1);
            // cells within rho_max of the visibility, inside its window
            lox = min(lox, ix0[v] + max(0, (int)floorf(hx[v] - rmax) + 1));
            hix = max(hix, ix0[v] + min(S - 1, (int)ceilf(hx[v] + rmax) - 1));
            loy = min(loy, iy0[v] + max(0, (int)floorf(hy[v] - rmax) + 1));
            hiy = max(hiy, iy0[v] + min(S - 1, (int)ceilf(hy[v] + rmax) - 1));
        }
        if (lox <= hix && loy <= hiy) {
            atomicMin(&sh.box[0], lox); atomicMax(&sh.box[1], hix);
            atomicMin(&sh.box[2], loy); atomicMax(&sh.box[3], hiy);
            const int nv = min(kV, a.nt - t0);
            atomicAdd(&sh.taps, nv * (int)ceilf(3.14159265f * rmax * rmax));
        }
    }
    // radial tables of this block's channels as (c_n, s_n), zero-padded
    for (int j = 0; j < n_ch; ++j) {
        const int cc = c_first + j;
        const int off = cc < a.nc ? a.chan[cc].tab_off : 0;
        const int len = cc < a.nc ? a.chan[cc].tab_len : 0;
        for (int n = tid; n < tab_stride; n += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (n < len) {
                const float2 e = a.tabs[off + n];
                v = make_float2(fmaf(-(float)n, e.y, e.x), e.y);
            }
            s_tab[j * tab_stride + n] = v;
        }
    }
    __syncthreads();
    const bool empty = sh.box[0] > sh.box[1];         // no visibility of the brick has a tap
    const int bx0 = empty ? 0 : sh.box[0], by0 = empty ? 0 : sh.box[2];
    const int ex = empty ? 0 : sh.box[1] - bx0 + 1, ey = empty ? 0 : sh.box[3] - by0 + 1;
    // Staging pays when the brick's taps reuse its cells: a staged cell costs
    // a global load, two complex products and a store (about four unstaged
    // taps' extra work), so stage only boxes of at most taps / 4 cells that
    // fit the tile.  Uniform over the block.
    const bool staged = !kW && !a.no_stage && ex <= kTile && ey <= kTile && 4 * ex * ey <= sh.taps;

    // per-cell half of the ramp, exp(-i pi du (k_x L + k_y M)) = phx[k_x] phy[k_y],
    // with (k_x, k_y) relative to the tile origin (staged) or to each
    // visibility's window origin (unstaged: k < S)
    if (!empty) {
        const int nx = staged ? ex : S, ny = staged ? ey : S;
        for (int k = tid; k < nx; k += blockDim.x) {
            float s, co;
            sincospif(-(float)k * a.du * L, &s, &co);
            sh.phx[k] = make_float2(co, s);
        }
        for (int k = tid; k < ny; k += blockDim.x) {
            float s, co;
            sincospif(-(float)k * a.du * M, &s, &co);
            sh.phy[k] = make_float2(co, s);
        }
        __syncthreads();
    }
    if (!kW && staged && !empty) {
        // threads -> (column, row group) with shifts: 64 columns per pass for
        // blocks of >= 64 threads, 32 for a 32-thread block (two passes);
        // the row step blockDim >> cshift is >= 1 for every allowed block size
        const int cshift = blockDim.x >= kTile ? 6 : 5;
        const int cols = 1 << cshift;
        const int rstep = blockDim.x >> cshift;
        for (int xx = tid & (cols - 1); xx < ex; xx += cols) {
            const int gx = bx0 + xx;
            const bool xin = gx >= 0 && gx < a.ng;
            const float2 px = sh.phx[xx];
            for (int yy = tid >> cshift; yy < ey; yy += rstep) {
                const int gy = by0 + yy;
                float2 g = make_float2(0.f, 0.f);
                if (xin && gy >= 0 && gy < a.ng) g = grid_cell(a, (size_t)gy * a.ng + gx);
                sh.tile[yy * kTile + xx] = cmul(g, cmul(px, sh.phy[yy]));
            }
        }
        __syncthreads();
    }

    // ---- per-visibility tap sums (relative to each visibility's window) ----
    float2 S0[kV], Su[kV], Sv[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) S0[v] = Su[v] = Sv[v] = make_float2(0.f, 0.f);
    if (active && !empty) {
        const float2 *tab = s_tab + lc * tab_stride;
        const unsigned tab_adj = (unsigned)__cvta_generic_to_shared(tab) - (0x4B000000u << 3);
        const float ov = (float)a.ov;
        const float rmax2 = rmax * rmax;
        if (!kW && staged) {
            int wx[kV], wy[kV];
            int r_lo = INT_MAX, r_hi = INT_MIN;
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                wx[v] = ix0[v] - bx0;
                wy[v] = iy0[v] - by0;
                r_lo = min(r_lo, wy[v] + max(0, (int)floorf(hy[v] - rmax) + 1));
                r_hi = max(r_hi, wy[v] + min(S - 1, (int)ceilf(hy[v] + rmax) - 1));
            }
            for (int cy = r_lo; cy <= r_hi; ++cy) {
                float dy[kV], dyo2[kV];
                int c_lo = INT_MAX, c_hi = INT_MIN;
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    dy[v] = hy[v] - (float)(cy - wy[v]);
                    const float dyo = dy[v] * ov;
                    dyo2[v] = fmaf(dyo, dyo, 1e-20f);
                    const float rem = rmax2 - dy[v] * dy[v];
                    if (rem > 0.f) {
                        // r <= rho_max keeps the span inside the staged box
                        const float r = fminf(rem * rsqrt_fast(rem), rmax);
                        const int a_lo = max(0, (int)floorf(hx[v] - r) + 1);
                        const int a_hi = min(S - 1, (int)ceilf(hx[v] + r) - 1);
                        if (a_lo <= a_hi) {
                            c_lo = min(c_lo, wx[v] + a_lo);
                            c_hi = max(c_hi, wx[v] + a_hi);
                        }
                    }
                }
                if (c_lo > c_hi) continue;
                float dxo[kV], pr[kV], pi[kV], qr[kV], qi[kV];
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    dxo[v] = (hx[v] - (float)(c_lo - wx[v])) * ov;
                    pr[v] = pi[v] = qr[v] = qi[v] = 0.f;
                }
                if constexpr (kV == 2)
                    row_taps2(sh.tile + cy * kTile + c_lo, c_hi - c_lo + 1, make_float2(dxo[0], dxo[1]),
                              make_float2(dyo2[0], dyo2[1]), ov, tab_adj, pr, pi, qr, qi);
                else
                    row_taps<kV>(sh.tile + cy * kTile + c_lo, c_hi - c_lo + 1, dxo, dyo2, ov, tab_adj, pr, pi, qr, qi);
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    S0[v].x += pr[v]; S0[v].y += pi[v];
                    Su[v].x += qr[v]; Su[v].y += qi[v];
                    Sv[v].x = fmaf(dy[v], pr[v], Sv[v].x);
                    Sv[v].y = fmaf(dy[v], pi[v], Sv[v].y);
                }
            }
        } else {
            // unstaged: taps read the grid (L1/L2), the cell half of the ramp
            // comes from phx / phy; rows and columns are clipped to the grid
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const int b_lo = max(max(0, (int)floorf(hy[v] - rmax) + 1), -iy0[v]);
                const int b_hi = min(min(S - 1, (int)ceilf(hy[v] + rmax) - 1), a.ng - 1 - iy0[v]);
                for (int b = b_lo; b <= b_hi; ++b) {
                    const float dy = hy[v] - (float)b;
                    const float rem = rmax2 - dy * dy;
                    if (!(rem > 0.f)) continue;
                    const float r = fminf(rem * rsqrt_fast(rem), rmax);
                    const int a_lo = max(max(0, (int)floorf(hx[v] - r) + 1), -ix0[v]);
                    const int a_hi = min(min(S - 1, (int)ceilf(hx[v] + r) - 1), a.ng - 1 - ix0[v]);
                    const float dyo = dy * ov;
                    const float dyo2 = fmaf(dyo, dyo, 1e-20f);
                    float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
                    const size_t row = (size_t)(iy0[v] + b) * a.ng + ix0[v];
                    float dd = (hx[v] - (float)a_lo) * ov;
                    for (int aa = a_lo; aa <= a_hi; ++aa, dd -= ov) {
                        float2 gc;
                        if constexpr (kW) {
                            const float2 g0 = __ldg(&a.grid[woff[v] + row + aa]);
                            const float2 g1 = __ldg(&a.grid[woff[v] + (size_t)a.ng * a.ng + row + aa]);
                            gc = make_float2(fmaf(wf[v], g1.x - g0.x, g0.x), fmaf(wf[v], g1.y - g0.y, g0.y));
                        } else {
                            gc = grid_cell(a, row + aa);
                        }
                        const float2 g = cmul(gc, sh.phx[aa]);
                        const float s2 = fmaf(dd, dd, dyo2);
                        const float tv = sqrt_fast(s2);
                        const float tf = __fadd_rz(tv, 8388608.0f);
                        const float2 e = lds_f2(tab_adj + ((unsigned)__float_as_int(tf) << 3));
                        const float A = fmaf(tv, e.y, e.x);
                        pr = fmaf(A, g.x, pr);
                        pi = fmaf(A, g.y, pi);
                        const float Ad = A * dd;
                        qr = fmaf(Ad, g.x, qr);
                        qi = fmaf(Ad, g.y, qi);
                    }
                    const float2 py = sh.phy[b];
                    const float2 P = cmul(make_float2(pr, pi), py);
                    const float2 Q = cmul(make_float2(qr, qi), py);
                    S0[v].x += P.x; S0[v].y += P.y;
                    Su[v].x += Q.x; Su[v].y += Q.y;
                    Sv[v].x = fmaf(dy, P.x, Sv[v].x);
                    Sv[v].y = fmaf(dy, P.y, Sv[v].y);
                }
            }
        }
        const float inv_ov = 1.0f / ov;
#pragma unroll
        for (int v = 0; v < kV; ++v) {                       // Q was accumulated with dx * ov
            Su[v].x *= inv_ov; Su[v].y *= inv_ov;
        }
    }

    // ---- epilogue: visibility half of the ramp, decorrelation, derivatives ----
    if (!active) return;
    const float al2 = a.chan[c].alpha2;
    float D = 1.f, el = 0.f, em = 0.f;
    if (a.decorrelation) {
        D = expf(-0.5f * al2 * (dL * dL + dM * dM));
        el = -dL * al2;                      // (l_j - l_i) alpha^2
        em = -dM * al2;
    }
    const float pi_f = 3.14159265358979f;
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const int t = t0 + v;
        if (t >= a.nt) break;
        const int ox = staged ? bx0 : ix0[v];
        const int oy = staged ? by0 : iy0[v];
        const float ph_arg = a.du * (((float)(ix0[v] - ox) + hx[v]) * L + ((float)(iy0[v] - oy) + hy[v]) * M);
        float s, co;
        sincospif(ph_arg, &s, &co);
        const float2 ph = make_float2(co, s);
        const float2 T0 = cmul(ph, S0[v]);
        float2 Tu = cmul(ph, Su[v]), Tv = cmul(ph, Sv[v]);
        Tu.x *= a.du; Tu.y *= a.du;          // tap offsets in wavelengths
        Tv.x *= a.du; Tv.y *= a.du;
        const float2 V = make_float2(D * T0.x, D * T0.y);
        // d/dl_i = D [(l_j - l_i) a^2 T0 + i pi Tu]; d/dl_j flips the first term; m likewise
        const float2 dli = make_float2(D * (el * T0.x - pi_f * Tu.y), D * (el * T0.y + pi_f * Tu.x));
        const float2 dmi = make_float2(D * (em * T0.x - pi_f * Tv.y), D * (em * T0.y + pi_f * Tv.x));
        const float2 dlj = make_float2(D * (-el * T0.x - pi_f * Tu.y), D * (-el * T0.y + pi_f * Tu.x));
        const float2 dmj = make_float2(D * (-em * T0.x - pi_f * Tv.y), D * (-em * T0.y + pi_f * Tv.x));
        const size_t k = ((size_t)t * a.n_bl + bl) * a.nc + c;
        if constexpr (kPredict) {
            a.vis_out[k] = V;
            if (a.dvis_out != nullptr) {
                const size_t plane = (size_t)a.nt * a.n_bl * a.nc;
                a.dvis_out[k] = dli;
                a.dvis_out[plane + k] = dmi;
                a.dvis_out[2 * plane + k] = dlj;
                a.dvis_out[3 * plane + k] = dmj;
            }
        } else {
            const float2 vo = a.vis_obs[k];
            const float w = a.w_scale * (a.w != nullptr ? a.w[k] : 1.f);
            const float2 R = make_float2(vo.x - V.x, vo.y - V.y);
            const float w2 = 2.f * w;
            acc[0] += w * (R.x * R.x + R.y * R.y);
            acc[1] -= w2 * (R.x * dli.x + R.y * dli.y);
            acc[2] -= w2 * (R.x * dmi.x + R.y * dmi.y);
            acc[3] -= w2 * (R.x * dlj.x + R.y * dlj.y);
            acc[4] -= w2 * (R.x * dmj.x + R.y * dmj.y);
            acc[5] += w2 * (dli.x * dli.x + dli.y * dli.y);
            acc[6] += w2 * (dli.x * dmi.x + dli.y * dmi.y);
            acc[7] += w2 * (dmi.x * dmi.x + dmi.y * dmi.y);
            acc[8] += w2 * (dlj.x * dlj.x + dlj.y * dlj.y);
            acc[9] += w2 * (dlj.x * dmj.x + dlj.y * dmj.y);
            acc[10] += w2 * (dmj.x * dmj.x + dmj.y * dmj.y);
            acc[11] += w2 * (dli.x * dlj.x + dli.y * dlj.y);
            acc[12] += w2 * (dli.x * dmj.x + dli.y * dmj.y);
            acc[13] += w2 * (dmi.x * dlj.x + dmi.y * dlj.y);
            acc[14] += w2 * (dmi.x * dmj.x + dmi.y * dmj.y);
        }
    }
}

// One launch covers either one context (queue == nullptr: block b handles
// brick b of a0) or a batch of contexts (persistent: each block pulls global
// brick numbers from an atomic queue until all sum(bricks) are taken; prefix
// holds the first global brick of each context).  Every brick writes its own
// partial record, so the result does not depend on which block ran it.
// The stacked instantiation (kW) asks for 4 blocks of kMaxThreads per SM,
// i.e. at most 64 registers (some spill): its unstaged two-plane taps gain
// more from the warps than they lose (vla27_l64ch as one interval: 5.56 ms
// against 6.36 ms at 99 registers).  A minimum of 0 leaves the co-planar
// instantiations with the plain bound.
template <bool kPredict, bool kW>
__global__ void __launch_bounds__(kMaxThreads, kW ? 4 : 0) eval_kernel(const EvalArgs a0, const EvalArgs *__restrict__ args,
                                                           const long long *__restrict__ prefix, int n_ctx,
                                                           unsigned long long *queue) {
    extern __shared__ float2 s_tab[];                 // c_group * tab_stride
    __shared__ BlockSharedT<!kW> sh;
    __shared__ EvalArgs s_a;
    __shared__ long long s_work, s_first;
    __shared__ int s_done;
    const bool persistent = queue != nullptr;
    long long next = -1;                              // thread 0: prefetched queue entry
    int cur = -1;                                     // thread 0: context whose arguments s_a holds
    for (;;) {
    if (persistent) {
        __syncthreads();                              // the previous brick is done with shared memory
        if (threadIdx.x == 0) {
            const long long gb = next >= 0 ? next : (long long)atomicAdd(queue, 1ull);
            next = (long long)atomicAdd(queue, 1ull);  // consumed next round: its latency overlaps this brick
            const long long end = prefix[n_ctx];
            s_done = gb >= end;
            if (gb < end) {
                // a block's bricks come in increasing order: the context is the
                // current one unless gb has passed its end
                if (cur < 0 || gb < prefix[cur] || gb >= prefix[cur + 1]) {
                    int lo = 0, hi = n_ctx - 1;       // last context with prefix[k] <= gb
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (prefix[mid] <= gb) lo = mid; else hi = mid - 1;
                    }
                    cur = lo;
                    s_a = args[lo];                   // copied once per context change
                    s_first = prefix[lo];
                }
                s_work = gb;
            }
        }
        __syncthreads();
        if (s_done) return;
    } else {
        if (threadIdx.x == 0) s_a = a0;
        __syncthreads();
    }
    const EvalArgs &a = s_a;
    if (!(a.skip != nullptr && *a.skip)) {
    const int tid = threadIdx.x;
    const int qbrick = persistent ? (int)(s_work - s_first) : (int)blockIdx.x;
    // launch order -> brick (baseline groups permuted for locality when bl_order is set)
    const int brick = a.bl_order != nullptr ? a.bl_order[qbrick / a.bpb] * a.bpb + qbrick % a.bpb : qbrick;
    float acc[kRed];
#pragma unroll
    for (int k = 0; k < kRed; ++k) acc[k] = 0.f;
    if (a.kv == 2) eval_brick<kPredict, 2, kW>(a, brick, s_tab, sh, acc);
    else eval_brick<kPredict, 1, kW>(a, brick, s_tab, sh, acc);
    if constexpr (!kPredict) {
        // ---- block reduction: a butterfly within each warp -- compensated
        // (Knuth's TwoSum, the rounding errors summed beside) for chi^2 and the
        // gradient, plain FP32 for the normal blocks -- then FP64 across warps ----
        float comp[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float so = __shfl_xor_sync(0xffffffffu, acc[k], o);
                const float co = __shfl_xor_sync(0xffffffffu, comp[k], o);
                const float t = __fadd_rn(acc[k], so);
                const float bp = __fsub_rn(t, acc[k]);
                const float err = __fadd_rn(__fsub_rn(acc[k], __fsub_rn(t, bp)), __fsub_rn(so, bp));
                acc[k] = t;
                comp[k] = __fadd_rn(__fadd_rn(comp[k], co), err);
            }
#pragma unroll
            for (int k = 5; k < kRed; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        }
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < kRed; ++k) sh.red[warp][k] = acc[k];
#pragma unroll
            for (int k = 0; k < 5; ++k) sh.red_c[warp][k] = comp[k];
        }
        __syncthreads();
        if (tid < kRed) {
            double s = 0.0;
            const int nw = (blockDim.x + 31) >> 5;
            for (int wi = 0; wi < nw; ++wi) {
                s += (double)sh.red[wi][tid];
                if (tid < 5) s += (double)sh.red_c[wi][tid];
            }
            a.partials[(size_t)tid * a.n_bricks + brick] = s;      // [kRed][n_bricks]
        }
    }
    }                                                 // not skipped
    if (!persistent) return;
    }                                                 // brick loop
}

// Second stage (a): per-baseline sums over its bricks, one thread per
// (baseline, sum), the bricks added in order (deterministic).  partials is
// [kRed][n_bricks] with the bricks of baseline bl at [bl * bpb, (bl + 1) * bpb).
// Batched form: the global baseline number runs over the baselines of all
// contexts (bl_prefix).
__global__ void bl_reduce_kernel(const RedArgs r0, const RedArgs *__restrict__ ra,
                                 const int *__restrict__ bl_prefix, int n_ctx) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int gb = (int)(gt / kRed), k = (int)(gt - (long long)gb * kRed);
    RedArgs r = r0;
    int bl = gb;
    if (ra != nullptr) {
        if (gb >= bl_prefix[n_ctx]) return;
        int lo = 0, hi = n_ctx - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bl_prefix[mid] <= gb) lo = mid; else hi = mid - 1;
        }
        r = ra[lo];
        bl = gb - bl_prefix[lo];
    }
    if (bl >= r.n_bl) return;
    if (r.skip != nullptr && *r.skip) return;
    const size_t nb = (size_t)r.n_bl * r.bpb;
    const double *p = r.partials + (size_t)k * nb + (size_t)bl * r.bpb;
    double sum = 0.0;
    for (int b = 0; b < r.bpb; ++b) sum += p[b];
    r.blsum[(size_t)bl * kRed + k] = sum;
}

// Second stage (b): chi^2, per-antenna gradient and diagonal blocks, cross
// blocks; ev = chi2 | g[2n] | H[3n] | X[4 nbl].  One block per context
// (blockIdx.x indexes ra when batched), fixed order.
__global__ void ev_kernel(const RedArgs r0, const RedArgs *__restrict__ ra) {
    const RedArgs r = ra != nullptr ? ra[blockIdx.x] : r0;
    if (r.skip != nullptr && *r.skip) return;
    __shared__ double s_chi[kMaxThreads];
    const int tid = threadIdx.x;
    const int n_ant = r.n_ant, n_bl = r.n_bl;
    double chi = 0.0;
    for (int bl = tid; bl < n_bl; bl += blockDim.x) {
        const double *sb = r.blsum + (size_t)bl * kRed;
        chi += sb[0];
        double *x = r.ev + 1 + 5 * (size_t)n_ant + 4 * (size_t)bl;
        x[0] = sb[11]; x[1] = sb[12]; x[2] = sb[13]; x[3] = sb[14];
    }
    s_chi[tid] = chi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) s_chi[tid] += s_chi[tid + o];
        __syncthreads();
    }
    if (tid == 0) r.ev[0] = s_chi[0];
    for (int an = tid; an < n_ant; an += blockDim.x) {
        double g0 = 0, g1 = 0, h0 = 0, h1 = 0, h2 = 0;
        for (int o = 0; o < n_ant; ++o) {
            if (o == an) continue;
            const int i = min(an, o), j = max(an, o);
            const int bl = i * (2 * n_ant - i - 1) / 2 + (j - i - 1);
            const double *sb = r.blsum + (size_t)bl * kRed;
            if (an == i) {
                g0 += sb[1]; g1 += sb[2]; h0 += sb[5]; h1 += sb[6]; h2 += sb[7];
            } else {
                g0 += sb[3]; g1 += sb[4]; h0 += sb[8]; h1 += sb[9]; h2 += sb[10];
            }
        }
        r.ev[1 + 2 * an] = g0;
        r.ev[2 + 2 * an] = g1;
        double *h = r.ev + 1 + 2 * (size_t)n_ant + 3 * (size_t)an;
        h[0] = h0; h[1] = h1; h[2] = h2;
    }
}

// Largest |uv(t+1) - uv(t)| over consecutive time steps and baselines.
__global__ void step_max_kernel(const double *__restrict__ uvw, int nt, int n_bl, unsigned *out_bits) {
    float m = 0.f;
    const long long n = (long long)(nt - 1) * n_bl;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double *p = uvw + 3 * k;
        const double *q = p + 3 * (size_t)n_bl;
        const double du = q[0] - p[0], dv = q[1] - p[1];
        m = fmaxf(m, (float)sqrt(du * du + dv * dv));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));   // m >= 0: bits order as values
}

__global__ void grid_to_bf16_kernel(const float2 *__restrict__ g, size_t n, unsigned *__restrict__ out) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const __nv_bfloat162 b = __float22bfloat162_rn(g[k]);
        out[k] = *reinterpret_cast<const unsigned *>(&b);
    }
}

__global__ void split_uv_kernel(const double *__restrict__ uvw, size_t n, float4 *__restrict__ out) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double u = uvw[3 * k], v = uvw[3 * k + 1];
        const float uh = (float)u, vh = (float)v;
        out[k] = make_float4(uh, (float)(u - (double)uh), vh, (float)(v - (double)vh));
    }
}

}  // namespace

cudaError_t launch_split_uv(const double *uvw, size_t n, float4 *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    split_uv_kernel<<<blocks, 256, 0, s>>>(uvw, n, out);
    return cudaGetLastError();
}

cudaError_t launch_grid_to_bf16(const float2 *grid, size_t n, unsigned *out, cudaStream_t s) {
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    grid_to_bf16_kernel<<<blocks, 256, 0, s>>>(grid, n, out);
    return cudaGetLastError();
}

cudaError_t launch_step_max(const double *uvw, int nt, int n_bl, unsigned *out_bits, cudaStream_t s) {
    if (nt < 2) return cudaSuccess;
    const long long n = (long long)(nt - 1) * n_bl;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    step_max_kernel<<<blocks, 256, 0, s>>>(uvw, nt, n_bl, out_bits);
    return cudaGetLastError();
}

size_t eval_dyn_smem(int c_group, int tab_stride) {
    return sizeof(float2) * (size_t)c_group * tab_stride;
}

cudaError_t launch_eval(const EvalArgs &a, bool predict, cudaStream_t s) {
    if (a.exact) return launch_exact(a, predict, s);
    const int threads = ((a.flat > 0 ? a.flat : a.t_tile * a.c_group) + 31) / 32 * 32;
    const int blocks = (int)a.n_bricks;
    const size_t dyn = eval_dyn_smem(a.flat > 0 ? a.ch_span : a.c_group, a.tab_stride);
    if (a.wp_n > 0) {
        if (predict) eval_kernel<true, true><<<blocks, threads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr);
        else eval_kernel<false, true><<<blocks, threads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr);
    } else if (predict) {
        eval_kernel<true, false><<<blocks, threads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr);
    } else {
        eval_kernel<false, false><<<blocks, threads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_eval_batch(const EvalArgs *args_dev, const long long *prefix_dev, int n_ctx,
                              unsigned long long *queue, int threads, size_t dyn, int grid, bool stacked,
                              cudaStream_t s) {
    EvalArgs none{};
    if (stacked) eval_kernel<false, true><<<grid, threads, dyn, s>>>(none, args_dev, prefix_dev, n_ctx, queue);
    else eval_kernel<false, false><<<grid, threads, dyn, s>>>(none, args_dev, prefix_dev, n_ctx, queue);
    return cudaGetLastError();
}

cudaError_t eval_batch_occupancy(int threads, size_t dyn, bool stacked, int *blocks_per_sm) {
    if (stacked)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, eval_kernel<false, true>, threads, dyn);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, eval_kernel<false, false>, threads, dyn);
}

// Dynamic shared memory the fused kernel can have on the current device: the
// opt-in limit less its static shared memory.
cudaError_t eval_smem_allowed(size_t *allowed) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, eval_kernel<false, false>);
    if (e != cudaSuccess) return e;
    *allowed = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    return cudaSuccess;
}

// Raises the fused kernel's dynamic shared-memory limit to everything the
// device allows beyond its static shared memory (never lowers it, so contexts
// with different channel groups can share the kernel), after checking that
// `dyn` bytes fit.
cudaError_t set_eval_smem(size_t dyn) {
    size_t allowed = 0;
    cudaError_t e = eval_smem_allowed(&allowed);
    if (e != cudaSuccess) return e;
    if (dyn > allowed) return cudaErrorInvalidValue;
    for (const void *k : {(const void *)eval_kernel<true, false>, (const void *)eval_kernel<false, false>,
                          (const void *)eval_kernel<true, true>, (const void *)eval_kernel<false, true>}) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)allowed);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_reduce(const RedArgs &r, cudaStream_t s) {
    const long long threads = (long long)r.n_bl * kRed;
    bl_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(r, nullptr, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ev_kernel<<<1, kMaxThreads, 0, s>>>(r, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_reduce_batch(const RedArgs *ra_dev, const int *bl_prefix_dev, int n_ctx, int total_bl,
                                cudaStream_t s) {
    const long long threads = (long long)total_bl * kRed;
    RedArgs none{};
    bl_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(none, ra_dev, bl_prefix_dev, n_ctx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ev_kernel<<<n_ctx, kMaxThreads, 0, s>>>(none, ra_dev);
    return cudaGetLastError();
}

}  // namespace psc

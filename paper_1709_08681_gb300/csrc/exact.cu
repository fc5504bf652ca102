// Exact aperture kernel of a pair of uniform disks with different pointing
// offsets, and the fused evaluation (degrid, pointing derivatives, residual,
// per-brick sums) that uses it in place of Eq. AIJPOINTING's Gaussian
// decorrelation factor.
//
// Paper basis (Bhatnagar & Cornwell 2017, Sec. 3): A_ij is the transform of
// the baseline's primary beam E_i E_j, each antenna's pattern shifted by its
// offset; the Gaussian main-lobe model may be replaced by a more accurate
// pattern.  For the uniform disk (aperture radius R = D_lambda / 2):
//
//   A_ij(du) = exp(i pi du.(l_i + l_j)) O(du; dl) / (pi R^2)^2,   dl = l_i - l_j,
//   O(du; dl) = integral over the lens {|w - du/2| <= R, |w + du/2| <= R} of cos(2 pi w.dl).
//
// Series.  On the lens |2 pi w.dl| <= x = pi D_lambda |dl|.  In the frame of
// du (w = w_par e + w_perp e_perp), the Taylor series of the cosine, with the
// lens moments M_pq(rho) = integral of w_par^p w_perp^q (odd p or q vanish
// by symmetry), gives, with A = (dl.e)^2 and s = |dl|^2,
//
//   O = P_0 + P_1 A + P_2 A^2 + P_3 A^3,   P_k = P_k(rho; s),
//
// keeping the terms up to (2 pi w.dl)^6.  The dropped remainder is at most
// x^8 / 8! of the lens area, and that of the derivative below at most
// x^7 / 7! times 2 pi R times the lens area (alternating series): below
// 1e-7 relative for x <= 0.3 (|dl| <= 2 arcmin for a 25 m dish at 1.5 GHz).
// With gamma_n = (-1)^n (2 pi)^2n / (2n)! and the ten per-channel moment
// combinations K0..K9 of moments_kernel,
//
//   P_0 = K0 + g1 s K1 + g2 s^2 K2 + g3 s^3 K3      Q_0 = dP_0/ds
//   P_1 = g1 K4 + g2 s K5 + g3 s^2 K6               Q_1 = dP_1/ds
//   P_2 = g2 K7 + g3 s K8                           Q_2 = dP_2/ds
//   P_3 = g3 K9.
//
// Derivative in dl (A depends on dl through dl.e, s through |dl|):
//   dO/d(dl) = 2 (dO/dA) ((dl.du) / |du|^2) du + 2 (dO/ds) dl.
// So dA_ij/dl_i = i pi du A_ij + ramp dO/d(dl) / (pi R^2)^2 and
// dA_ij/dl_j = i pi du A_ij - ramp dO/d(dl) / (pi R^2)^2 (m likewise).
//
// Tables and interpolation follow the radial kernel's rule: sample n is at
// rho = n du / ov, a tap at t = rho ov takes the linear interpolation of
// samples floor(t) and floor(t) + 1 (zero when floor(t) + 1 >= len) -- here
// of each P_k and Q_k, i.e. of O at fixed direction.  Each brick builds its
// channels' interpolation entries (intercept, slope) for its own s from the
// moment combinations, then the tap loop evaluates the cubic in A.
//
// Work decomposition as in the Gaussian-model kernel (eval.cu), with one
// visibility per thread: a brick is a baseline, c_group channels and t_tile
// time steps; the block stages the grid cells of its visibilities' aperture
// disks in shared memory when they fit, pre-multiplied by the cell half of
// the phase ramp, else reads the grid per tap.  It reads the FP32 grid (the
// BF16 copy of psc_set_grid_precision is not used) and the FP64 uvw.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kNodes = 32;            // Gauss-Legendre nodes of the moment quadrature
constexpr int kExTile = 48;           // staged box of this kernel: at most kExTile x kExTile cells (18 KB)
// An interpolation entry is three float4 (P0, P1 | P2, P3 | Q0, Q1 as intercepts
// then slopes) and one float2 (Q2); each of the four parts lives in its own
// array, so that entries of neighbouring radii are 16 (8) bytes apart and the
// lanes' lookups spread over the shared-memory banks.
struct TabView {
    const float4 *e0, *e1, *e2;
    const float2 *e3;
};
__constant__ double c_gl[2 * kNodes]; // nodes on [-1, 1], then weights

// gamma_n = (-1)^n (2 pi)^(2n) / (2n)!
constexpr float kG1 = -19.7392088021787f;   // -(2 pi)^2 / 2
constexpr float kG2 = 64.9393940226683f;    //  (2 pi)^4 / 24
constexpr float kG3 = -85.4568172426067f;   // -(2 pi)^6 / 720

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_fast(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Lens moments of channel c at sample n (rho = n du / ov wavelengths) by
// Gauss-Legendre quadrature in theta, with w_par + rho / 2 = R cos(theta),
// half-height R sin(theta), theta in [0, acos(rho / 2R)]:
//   M_pq = 4 / (q + 1) int (R cos(theta) - rho/2)^p (R sin(theta))^(q+1) R sin(theta) dtheta,
// then the combinations K0..K9 (of the file header) normalised like the
// radial table, times du^2 / (pi R^2)^2, rounded to FP32.
__global__ void moments_kernel(double diam_m, const double *__restrict__ freq, int nc, double du, int ov,
                               const int *__restrict__ off, const int *__restrict__ len, float *__restrict__ kmom) {
    const int c = blockIdx.y;
    if (c >= nc) return;
    const double R = 0.5 * diam_m * freq[c] / kC;
    const double area = M_PI * R * R;
    const double norm = du * du / (area * area);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < len[c]; n += gridDim.x * blockDim.x) {
        const double rho = (double)n * du / ov;
        double m[4][4] = {};                  // m[p/2][q/2]
        if (rho < 2.0 * R) {
            const double th0 = acos(rho / (2.0 * R));
            for (int i = 0; i < kNodes; ++i) {
                const double th = 0.5 * th0 * (c_gl[i] + 1.0);
                const double wt = 0.5 * th0 * c_gl[kNodes + i];
                const double wp = R * cos(th) - 0.5 * rho;
                const double h = R * sin(th);
                const double wp2 = wp * wp, h2 = h * h;
                double pp = 1.0;                  // wp^p
                for (int p = 0; p < 4; ++p) {
                    double hq = h;                // h^(q+1)
                    for (int q = 0; p + q < 4; ++q) {
                        m[p][q] += wt * pp * hq * h * 4.0 / (2 * q + 1);   // jacobian R sin(theta) = h
                        hq *= h2;
                    }
                    pp *= wp2;
                }
            }
        }
        // m[a][b] = M_(2a)(2b)
        const double K[10] = {
            m[0][0], m[0][1], m[0][2], m[0][3],
            m[1][0] - m[0][1],
            6.0 * m[1][1] - 2.0 * m[0][2],
            15.0 * m[1][2] - 3.0 * m[0][3],
            m[2][0] - 6.0 * m[1][1] + m[0][2],
            15.0 * m[2][1] - 30.0 * m[1][2] + 3.0 * m[0][3],
            m[3][0] - 15.0 * m[2][1] + 15.0 * m[1][2] - m[0][3]};
        float *o = kmom + (size_t)(off[c] + n) * 10;
        for (int k = 0; k < 10; ++k) o[k] = (float)(K[k] * norm);
    }
}

// P_0..P_3, Q_0..Q_2 of one sample from its moment combinations and s.
__device__ __forceinline__ void series_values(const float *K, float s, float (&v)[7]) {
    v[0] = fmaf(s, fmaf(s, fmaf(s, kG3 * K[3], kG2 * K[2]), kG1 * K[1]), K[0]);
    v[1] = fmaf(s, fmaf(s, kG3 * K[6], kG2 * K[5]), kG1 * K[4]);
    v[2] = fmaf(s, kG3 * K[8], kG2 * K[7]);
    v[3] = kG3 * K[9];
    v[4] = fmaf(s, fmaf(s, 3.f * kG3 * K[3], 2.f * kG2 * K[2]), kG1 * K[1]);
    v[5] = fmaf(s, 2.f * kG3 * K[6], kG2 * K[5]);
    v[6] = kG3 * K[8];
}

struct ExactShared {
    float2 tile[kExTile * kExTile];
    float2 phx[kTile], phy[kTile];
    float red[kMaxThreads / 32][kRed];
    float bl[6];       // L, M, dl_x, dl_y, s = |dl|^2
    int box[4];
    int taps;
};

// Per-tap sums of one row of taps (n cells from `row`, the first at table
// coordinate dxo, the row at dyo2 = dyo^2, q = dl.(dxo, dyo)).  Entry parts
// (intercepts, then slopes): e0 = (P0, P1 | P0, P1), e1 = (P2, P3 | ..),
// e2 = (Q0, Q1 | ..), e3 = (Q2 | Q2).
struct RowSums {
    float2 P, Q, X, Y, Z;   // sum O g, O dxo g, Os g, W g, W dxo g
};

template <bool kGlobal>
__device__ __forceinline__ void exact_row(const float2 *__restrict__ row, const float2 *__restrict__ phx, int a0,
                                          int n, float dxo, float dyo2, float q, float ov, float dlx_ov,
                                          const TabView tab, RowSums &r) {
    for (int k = 0; k < n; ++k) {
        float2 g = row[k];
        if constexpr (kGlobal) g = cmul(g, phx[a0 + k]);
        const float s2 = fmaf(dxo, dxo, dyo2);
        const float t = sqrt_fast(s2);
        const int idx = (int)t;
        const float4 e0 = tab.e0[idx], e1 = tab.e1[idx], e2 = tab.e2[idx];
        const float2 e3 = tab.e3[idx];
        const float P0 = fmaf(t, e0.z, e0.x), P1 = fmaf(t, e0.w, e0.y);
        const float P2 = fmaf(t, e1.z, e1.x), P3 = fmaf(t, e1.w, e1.y);
        const float Q0 = fmaf(t, e2.z, e2.x), Q1 = fmaf(t, e2.w, e2.y);
        const float Q2 = fmaf(t, e3.y, e3.x);
        const float rr = q * rcp_fast(s2);             // (dl.du) / |du|^2 (table units)
        const float A = q * rr;                        // (dl.e)^2
        const float O = fmaf(A, fmaf(A, fmaf(A, P3, P2), P1), P0);
        const float Oa = fmaf(A, fmaf(3.f * A, P3, P2 + P2), P1);
        const float Os = fmaf(A, fmaf(A, Q2, Q1), Q0);
        const float W = Oa * rr;
        const float Od = O * dxo, Wd = W * dxo;
        r.P.x = fmaf(O, g.x, r.P.x);   r.P.y = fmaf(O, g.y, r.P.y);
        r.Q.x = fmaf(Od, g.x, r.Q.x);  r.Q.y = fmaf(Od, g.y, r.Q.y);
        r.X.x = fmaf(Os, g.x, r.X.x);  r.X.y = fmaf(Os, g.y, r.X.y);
        r.Y.x = fmaf(W, g.x, r.Y.x);   r.Y.y = fmaf(W, g.y, r.Y.y);
        r.Z.x = fmaf(Wd, g.x, r.Z.x);  r.Z.y = fmaf(Wd, g.y, r.Z.y);
        dxo -= ov;
        q -= dlx_ov;
    }
}

// One brick per block.  Reduce mode writes the brick's 15 sums to
// partials[k * n_bricks + brick]; predict mode writes V and dV.
template <bool kPredict>
__global__ void __launch_bounds__(kMaxThreads) exact_kernel(const EvalArgs a) {
    extern __shared__ float4 s_tab[];                 // three float4 arrays, then a float2 array, of c_group * tab_stride
    __shared__ ExactShared sh;
    const int tid = threadIdx.x;
    const int brick = blockIdx.x;
    // brick -> baseline, this thread's channel c and time step t, and the
    // block's channels [c_first, c_first + n_ch) (flat or rectangular bricks
    // as in eval.cu, one visibility per thread)
    int bl, c, t, c_first, n_ch;
    bool active;
    if (a.flat > 0) {
        bl = brick / a.bpb;
        const int first = (brick - bl * a.bpb) * a.flat;
        const int k = first + tid;
        c = k / a.n_tp;
        t = k - c * a.n_tp;
        c_first = first / a.n_tp;
        n_ch = min(a.nc - 1, (first + a.flat - 1) / a.n_tp) - c_first + 1;
        active = tid < a.flat && c < a.nc;
    } else {
        const int tt = brick % a.n_tt;
        const int cgi = (brick / a.n_tt) % a.n_cg;
        bl = brick / (a.n_tt * a.n_cg);
        const int lcg = tid / a.t_tile;
        t = tt * a.t_tile + tid % a.t_tile;
        c_first = cgi * a.c_group;
        c = c_first + lcg;
        n_ch = a.c_group;
        active = lcg < a.c_group && t < a.nt && c < a.nc;
    }
    const int lc = c - c_first;
    // channel slots of the tables in shared memory (as launch_exact sizes them)
    const size_t cs = (size_t)(a.flat > 0 ? a.ch_span : a.c_group) * a.tab_stride;
    const int tab_stride = a.tab_stride;
    const int S = a.support;
    if (a.skip != nullptr && *a.skip) return;

    if (tid == 0) {
        const int2 ij = a.pairs[bl];
        const double li = a.lm[2 * ij.x], mi = a.lm[2 * ij.x + 1];
        const double lj = a.lm[2 * ij.y], mj = a.lm[2 * ij.y + 1];
        const double dlx = li - lj, dly = mi - mj;
        sh.bl[0] = (float)(li + lj);
        sh.bl[1] = (float)(mi + mj);
        sh.bl[2] = (float)dlx;
        sh.bl[3] = (float)dly;
        sh.bl[4] = (float)(dlx * dlx + dly * dly);
        sh.box[0] = INT_MAX; sh.box[1] = INT_MIN; sh.box[2] = INT_MAX; sh.box[3] = INT_MIN;
        sh.taps = 0;
    }
    __syncthreads();
    const float L = sh.bl[0], M = sh.bl[1], dlx = sh.bl[2], dly = sh.bl[3], s = sh.bl[4];

    // grid position (FP64), window origin and in-window offset as in eval.cu
    int ix0 = 0, iy0 = 0;
    float hx = 0.f, hy = 0.f, rmax = 0.f;
    if (active) {
        const ChanConst ch = a.chan[c];
        rmax = ch.rho_max;
        const double *p = a.uvw + ((size_t)t * a.n_bl + bl) * 3;
        const double x = p[0] * ch.uv_scale + 0.5 * a.ng;
        const double y = p[1] * ch.uv_scale + 0.5 * a.ng;
        const double flx = floor(x), fly = floor(y);
        ix0 = (int)flx - S / 2 + 1;
        iy0 = (int)fly - S / 2 + 1;
        hx = (float)(x - flx) + (float)(S / 2 - 1);
        hy = (float)(y - fly) + (float)(S / 2 - 1);
        const int lox = ix0 + max(0, (int)floorf(hx - rmax) + 1);
        const int hix = ix0 + min(S - 1, (int)ceilf(hx + rmax) - 1);
        const int loy = iy0 + max(0, (int)floorf(hy - rmax) + 1);
        const int hiy = iy0 + min(S - 1, (int)ceilf(hy + rmax) - 1);
        if (lox <= hix && loy <= hiy) {
            atomicMin(&sh.box[0], lox); atomicMax(&sh.box[1], hix);
            atomicMin(&sh.box[2], loy); atomicMax(&sh.box[3], hiy);
            atomicAdd(&sh.taps, (int)ceilf(3.14159265f * rmax * rmax));
        }
    }
    // interpolation entries of this block's channels for this baseline's s
    for (int j = 0; j < n_ch; ++j) {
        const int cc = c_first + j;
        const int off = cc < a.nc ? a.chan[cc].tab_off : 0;
        const int len = cc < a.nc ? a.chan[cc].tab_len : 0;
        for (int n = tid; n < tab_stride; n += blockDim.x) {
            float c0[7] = {}, sl[7] = {};
            if (n + 1 < len) {
                float v0[7], v1[7];
                series_values(a.kmom + (size_t)(off + n) * 10, s, v0);
                series_values(a.kmom + (size_t)(off + n + 1) * 10, s, v1);
                for (int k = 0; k < 7; ++k) {
                    sl[k] = v1[k] - v0[k];
                    c0[k] = fmaf(-(float)n, sl[k], v0[k]);
                }
            }
            const size_t at = (size_t)j * tab_stride + n;
            s_tab[at] = make_float4(c0[0], c0[1], sl[0], sl[1]);
            s_tab[cs + at] = make_float4(c0[2], c0[3], sl[2], sl[3]);
            s_tab[2 * cs + at] = make_float4(c0[4], c0[5], sl[4], sl[5]);
            reinterpret_cast<float2 *>(s_tab + 3 * cs)[at] = make_float2(c0[6], sl[6]);
        }
    }
    __syncthreads();
    const bool empty = sh.box[0] > sh.box[1];
    const int bx0 = empty ? 0 : sh.box[0], by0 = empty ? 0 : sh.box[2];
    const int ex = empty ? 0 : sh.box[1] - bx0 + 1, ey = empty ? 0 : sh.box[3] - by0 + 1;
    const bool staged = !a.no_stage && ex <= kExTile && ey <= kExTile && 4 * ex * ey <= sh.taps;
    if (!empty) {
        const int nx = staged ? ex : S, ny = staged ? ey : S;
        for (int k = tid; k < nx; k += blockDim.x) {
            float sn, cs;
            sincospif(-(float)k * a.du * L, &sn, &cs);
            sh.phx[k] = make_float2(cs, sn);
        }
        for (int k = tid; k < ny; k += blockDim.x) {
            float sn, cs;
            sincospif(-(float)k * a.du * M, &sn, &cs);
            sh.phy[k] = make_float2(cs, sn);
        }
        __syncthreads();
    }
    if (staged && !empty) {
        for (int k = tid; k < ex * ey; k += blockDim.x) {
            const int yy = k / ex, xx = k - yy * ex;
            const int gx = bx0 + xx, gy = by0 + yy;
            float2 g = make_float2(0.f, 0.f);
            if (gx >= 0 && gx < a.ng && gy >= 0 && gy < a.ng) g = __ldg(&a.grid[(size_t)gy * a.ng + gx]);
            sh.tile[yy * kExTile + xx] = cmul(g, cmul(sh.phx[xx], sh.phy[yy]));
        }
        __syncthreads();
    }

    // ---- tap sums, relative to the visibility's window ----
    float2 S0 = make_float2(0.f, 0.f), Su = S0, Sv = S0, SX = S0, SZx = S0, SZy = S0;
    if (active && !empty) {
        const size_t at = (size_t)lc * tab_stride;
        const TabView tab{s_tab + at, s_tab + cs + at, s_tab + 2 * cs + at,
                          reinterpret_cast<const float2 *>(s_tab + 3 * cs) + at};
        const float ov = (float)a.ov;
        const float rmax2 = rmax * rmax;
        const float dlx_ov = dlx * ov;
        const int b_lo = max(max(0, (int)floorf(hy - rmax) + 1), staged ? 0 : -iy0);
        const int b_hi = min(min(S - 1, (int)ceilf(hy + rmax) - 1), staged ? S - 1 : a.ng - 1 - iy0);
        for (int b = b_lo; b <= b_hi; ++b) {
            const float dy = hy - (float)b;
            const float rem = rmax2 - dy * dy;
            if (!(rem > 0.f)) continue;
            const float r = fminf(rem * rsqrt_fast(rem), rmax);
            int a_lo = max(0, (int)floorf(hx - r) + 1);
            int a_hi = min(S - 1, (int)ceilf(hx + r) - 1);
            if (!staged) {
                a_lo = max(a_lo, -ix0);
                a_hi = min(a_hi, a.ng - 1 - ix0);
            }
            if (a_lo > a_hi) continue;
            const float dyo = dy * ov;
            const float dyo2 = fmaf(dyo, dyo, 1e-20f);
            const float dxo = (hx - (float)a_lo) * ov;
            const float q = fmaf(dlx, dxo, dly * dyo);
            RowSums rs{};
            if (staged) {
                const float2 *row = sh.tile + (iy0 - by0 + b) * kExTile + (ix0 - bx0 + a_lo);
                exact_row<false>(row, nullptr, 0, a_hi - a_lo + 1, dxo, dyo2, q, ov, dlx_ov, tab, rs);
            } else {
                const float2 *row = a.grid + (size_t)(iy0 + b) * a.ng + ix0 + a_lo;
                exact_row<true>(row, sh.phx, a_lo, a_hi - a_lo + 1, dxo, dyo2, q, ov, dlx_ov, tab, rs);
                const float2 py = sh.phy[b];
                rs.P = cmul(rs.P, py); rs.Q = cmul(rs.Q, py); rs.X = cmul(rs.X, py);
                rs.Y = cmul(rs.Y, py); rs.Z = cmul(rs.Z, py);
            }
            S0.x += rs.P.x; S0.y += rs.P.y;
            Su.x += rs.Q.x; Su.y += rs.Q.y;
            Sv.x = fmaf(dy, rs.P.x, Sv.x); Sv.y = fmaf(dy, rs.P.y, Sv.y);
            SX.x += rs.X.x; SX.y += rs.X.y;
            SZx.x += rs.Z.x; SZx.y += rs.Z.y;
            SZy.x = fmaf(dyo, rs.Y.x, SZy.x); SZy.y = fmaf(dyo, rs.Y.y, SZy.y);
        }
        const float inv_ov = 1.0f / ov;
        Su.x *= inv_ov; Su.y *= inv_ov;
    }

    // ---- epilogue ----
    float acc[kRed];
#pragma unroll
    for (int k = 0; k < kRed; ++k) acc[k] = 0.f;
    if (active) {
        const int ox = staged ? bx0 : ix0, oy = staged ? by0 : iy0;
        const float ph_arg = a.du * (((float)(ix0 - ox) + hx) * L + ((float)(iy0 - oy) + hy) * M);
        float sn, cs;
        sincospif(ph_arg, &sn, &cs);
        const float2 ph = make_float2(cs, sn);
        const float pi_f = 3.14159265358979f;
        const float2 V = cmul(ph, S0);
        float2 Tu = cmul(ph, Su), Tv = cmul(ph, Sv);
        Tu.x *= a.du; Tu.y *= a.du;
        Tv.x *= a.du; Tv.y *= a.du;
        // sum of dO/d(dl) G' = 2 (Z + dl X), per axis
        const float2 GX = cmul(ph, make_float2(2.f * fmaf(dlx, SX.x, SZx.x), 2.f * fmaf(dlx, SX.y, SZx.y)));
        const float2 GY = cmul(ph, make_float2(2.f * fmaf(dly, SX.x, SZy.x), 2.f * fmaf(dly, SX.y, SZy.y)));
        const float2 dli = make_float2(GX.x - pi_f * Tu.y, GX.y + pi_f * Tu.x);
        const float2 dmi = make_float2(GY.x - pi_f * Tv.y, GY.y + pi_f * Tv.x);
        const float2 dlj = make_float2(-GX.x - pi_f * Tu.y, -GX.y + pi_f * Tu.x);
        const float2 dmj = make_float2(-GY.x - pi_f * Tv.y, -GY.y + pi_f * Tv.x);
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
            acc[0] = w * (R.x * R.x + R.y * R.y);
            acc[1] = -w2 * (R.x * dli.x + R.y * dli.y);
            acc[2] = -w2 * (R.x * dmi.x + R.y * dmi.y);
            acc[3] = -w2 * (R.x * dlj.x + R.y * dlj.y);
            acc[4] = -w2 * (R.x * dmj.x + R.y * dmj.y);
            acc[5] = w2 * (dli.x * dli.x + dli.y * dli.y);
            acc[6] = w2 * (dli.x * dmi.x + dli.y * dmi.y);
            acc[7] = w2 * (dmi.x * dmi.x + dmi.y * dmi.y);
            acc[8] = w2 * (dlj.x * dlj.x + dlj.y * dlj.y);
            acc[9] = w2 * (dlj.x * dmj.x + dlj.y * dmj.y);
            acc[10] = w2 * (dmj.x * dmj.x + dmj.y * dmj.y);
            acc[11] = w2 * (dli.x * dlj.x + dli.y * dlj.y);
            acc[12] = w2 * (dli.x * dmj.x + dli.y * dmj.y);
            acc[13] = w2 * (dmi.x * dlj.x + dmi.y * dlj.y);
            acc[14] = w2 * (dmi.x * dmj.x + dmi.y * dmj.y);
        }
    }
    if constexpr (!kPredict) {
        // block reduction: FP32 within a warp, FP64 across warps (as eval.cu)
#pragma unroll
        for (int k = 0; k < kRed; ++k) {
            float v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[k] = v;
        }
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < kRed; ++k) sh.red[warp][k] = acc[k];
        }
        __syncthreads();
        if (tid < kRed) {
            double sum = 0.0;
            const int nw = (blockDim.x + 31) >> 5;
            for (int wi = 0; wi < nw; ++wi) sum += (double)sh.red[wi][tid];
            a.partials[(size_t)tid * a.n_bricks + brick] = sum;
        }
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (host, FP64): Newton's method on
// the Legendre polynomial P_n, evaluated with Bonnet's recurrence, from the
// initial guesses cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dpn = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm = 1.0, pn = z;              // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2 * k - 1) * z * pn - (k - 1) * pm) / k;
                pm = pn;
                pn = pk;
            }
            dpn = n * (z * pn - pm) / (z * z - 1.0);
            const double step = pn / dpn;
            z -= step;
            if (std::fabs(step) <= 1e-15 * std::fabs(z) + 1e-300) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

}  // namespace

cudaError_t launch_exact_moments(double diam_m, const double *freq_dev, int nc, double du, int ov,
                                 const int *tab_off_dev, const int *tab_len_dev, float *kmom, cudaStream_t s) {
    double gl[2 * kNodes];
    gauss_legendre(kNodes, gl, gl + kNodes);
    cudaError_t e = cudaMemcpyToSymbolAsync(c_gl, gl, sizeof(gl), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);             // gl is a host stack array
    if (e != cudaSuccess) return e;
    dim3 grid(4, nc);
    moments_kernel<<<grid, 128, 0, s>>>(diam_m, freq_dev, nc, du, ov, tab_off_dev, tab_len_dev, kmom);
    return cudaGetLastError();
}

size_t exact_dyn_smem(int c_group, int tab_stride) {
    return (3 * sizeof(float4) + sizeof(float2)) * (size_t)c_group * tab_stride;
}

cudaError_t launch_exact(const EvalArgs &a, bool predict, cudaStream_t s) {
    const int threads = ((a.flat > 0 ? a.flat : a.t_tile * a.c_group) + 31) / 32 * 32;
    const int blocks = (int)a.n_bricks;
    const size_t dyn = exact_dyn_smem(a.flat > 0 ? a.ch_span : a.c_group, a.tab_stride);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, predict ? exact_kernel<true> : exact_kernel<false>);
    if (e != cudaSuccess) return e;
    if (dyn + fa.sharedSizeBytes > (size_t)optin) return cudaErrorInvalidValue;
    if (predict) {
        e = cudaFuncSetAttribute(exact_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        exact_kernel<true><<<blocks, threads, dyn, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(exact_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        exact_kernel<false><<<blocks, threads, dyn, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace psc

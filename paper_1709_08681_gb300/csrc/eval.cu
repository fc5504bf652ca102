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
// (i, j), a group of c_group channels and a tile of t_tile time steps, one
// visibility per thread (warps are single-channel, consecutive times).  The
// block stages the grid cells its visibilities touch in shared memory.  The
// kernel's ramp factorises, exp(i pi (u_k - u_g) L) =
// exp(i pi (u_k - u_o) L) exp(-i pi (u_g - u_o) L) for any origin u_o, so the
// staged cells are pre-multiplied by the second factor (per cell, once per
// block) and each visibility applies the first factor once; the inner loop
// over taps then needs only the real radial A° and five FMAs per tap.  Taps
// outside the aperture's support are not visited (their A° is zero by the
// table rule).  If a brick's footprint does not fit the staging tile, the
// block falls back to reading the grid from global memory with the ramp
// applied per tap (same arithmetic, slower).
//
// Inner loop per tap (rho in units of table samples, t = rho * ov):
//   s2 = dxo^2 + dyo^2 (dxo = dx ov, dyo^2 carries a 1e-20 floor so s2 > 0),
//   t = s2 * rsqrt(s2), n = floor(t) by a round-toward-zero add of 2^23 whose
//   bit pattern also gives the table address, A° = value + f * slope, then
//   P += A° G', Q += (A° dxo) G'.  Tables are padded with zero entries so no
//   index clamp is needed (taps are limited to rho < rho_max).
#include <climits>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kTabPad = 2;     // zero entries after each staged table

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

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

// One row of taps: a_n consecutive staged cells starting at `row`, first tap
// at dxo (= dx * ov), table at shared address tab_adj + (0x4B000000 << 3).
// Accumulates P = sum A G' and Q = sum A dxo G'.
__device__ __forceinline__ void row_taps(const float2 *__restrict__ row, int a_n, float dxo, float dyo2, float ov,
                                         unsigned tab_adj, float &pr, float &pi, float &qr, float &qi) {
#pragma unroll 4
    for (int k = 0; k < a_n; ++k) {
        const float s2 = fmaf(dxo, dxo, dyo2);
        const float t = s2 * rsqrt_fast(s2);
        const float tf = __fadd_rz(t, 8388608.0f);             // floor(t) + 2^23
        const float2 e = lds_f2(tab_adj + ((unsigned)__float_as_int(tf) << 3));
        const float f = t - (tf - 8388608.0f);
        const float A = fmaf(f, e.y, e.x);
        const float2 g = row[k];
        pr = fmaf(A, g.x, pr);
        pi = fmaf(A, g.y, pi);
        const float Ad = A * dxo;
        qr = fmaf(Ad, g.x, qr);
        qi = fmaf(Ad, g.y, qi);
        dxo -= ov;
    }
}

// One launch covers either one context (queue == nullptr: block b handles
// brick b of a0) or a batch of contexts (persistent: each block pulls global
// brick numbers from an atomic queue until all sum(bricks) are taken; prefix
// holds the first global brick of each context).  Every brick writes its own
// partial record, so the result does not depend on which block ran it.
template <bool kPredict>
__global__ void __launch_bounds__(kMaxThreads) eval_kernel(const EvalArgs a0, const EvalArgs *__restrict__ args,
                                                           const long long *__restrict__ prefix, int n_ctx,
                                                           unsigned long long *queue) {
    extern __shared__ float2 s_tab[];                 // c_group * (max_tab_len + kTabPad)
    __shared__ float2 s_tile[kTile * kTile];
    __shared__ float2 s_phx[kTile], s_phy[kTile];
    __shared__ int s_box[4];
    __shared__ double s_red[kMaxThreads / 32][kRed];
    __shared__ EvalArgs s_a;
    __shared__ long long s_work, s_first;
    __shared__ int s_ctx;
    const bool persistent = queue != nullptr;
    long long next = -1;                              // thread 0: prefetched queue entry
    for (;;) {
    if (persistent) {
        __syncthreads();                              // the previous brick is done with shared memory
        if (threadIdx.x == 0) {
            const long long gb = next >= 0 ? next : (long long)atomicAdd(queue, 1ull);
            next = (long long)atomicAdd(queue, 1ull);  // consumed next round: its latency overlaps this brick
            int lo = 0, hi = n_ctx - 1;               // last context with prefix[k] <= gb
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prefix[mid] <= gb) lo = mid; else hi = mid - 1;
            }
            s_work = gb;
            s_ctx = lo;
            s_first = prefix[lo];
            if (gb < prefix[n_ctx]) s_a = args[lo];
        }
        __syncthreads();
        if (s_work >= prefix[n_ctx]) return;
    } else {
        if (threadIdx.x == 0) s_a = a0;
        __syncthreads();
    }
    const EvalArgs &a = s_a;
    if (!(a.skip != nullptr && *a.skip)) {
    const int tid = threadIdx.x;
    const int brick = persistent ? (int)(s_work - s_first) : (int)blockIdx.x;
    const int tt = brick % a.n_tt;
    const int cgi = (brick / a.n_tt) % a.n_cg;
    const int bl = brick / (a.n_tt * a.n_cg);
    const int lt = tid % a.t_tile;
    const int lc = tid / a.t_tile;
    const int t = tt * a.t_tile + lt;
    const int c = cgi * a.c_group + lc;
    const bool valid = lc < a.c_group && t < a.nt && c < a.nc;
    const int tab_stride = a.max_tab_len + kTabPad;

    // per-baseline constants, computed once per block in FP64
    __shared__ float s_bl[4];
    if (tid == 0) {
        const int2 ij = a.pairs[bl];
        const double li = a.lm[2 * ij.x], mi = a.lm[2 * ij.x + 1];
        const double lj = a.lm[2 * ij.y], mj = a.lm[2 * ij.y + 1];
        s_bl[0] = (float)(li + lj);   // ramp: l_i + l_j
        s_bl[1] = (float)(mi + mj);
        s_bl[2] = (float)(li - lj);   // decorrelation: l_i - l_j
        s_bl[3] = (float)(mi - mj);
        s_box[0] = INT_MAX; s_box[1] = INT_MIN; s_box[2] = INT_MAX; s_box[3] = INT_MIN;
    }
    __syncthreads();
    const float L = s_bl[0], M = s_bl[1], dL = s_bl[2], dM = s_bl[3];

    // Grid position of this visibility: x = u / du + Ng/2 (cells), window
    // origin floor(x) - S/2 + 1.
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
        atomicMin(&s_box[0], ix0); atomicMax(&s_box[1], ix0);
        atomicMin(&s_box[2], iy0); atomicMax(&s_box[3], iy0);
    }
    // radial tables of this block's channels, zero-padded
    for (int k = tid; k < a.c_group * tab_stride; k += blockDim.x) {
        const int cc = cgi * a.c_group + k / tab_stride;
        const int n = k % tab_stride;
        float2 v = make_float2(0.f, 0.f);
        if (cc < a.nc) {
            const ChanConst ch = a.chan[cc];
            if (n < ch.tab_len) v = a.tabs[ch.tab_off + n];
        }
        s_tab[k] = v;
    }
    __syncthreads();
    const int bx0 = s_box[0], by0 = s_box[2];
    const int ex = s_box[1] - bx0 + a.support, ey = s_box[3] - by0 + a.support;
    const bool staged = ex <= kTile && ey <= kTile;      // uniform over the block

    if (staged) {
        // per-cell half of the ramp, relative to the tile origin
        for (int k = tid; k < ex; k += blockDim.x) {
            float s, co;
            sincospif(-(float)k * a.du * L, &s, &co);
            s_phx[k] = make_float2(co, s);
        }
        for (int k = tid; k < ey; k += blockDim.x) {
            float s, co;
            sincospif(-(float)k * a.du * M, &s, &co);
            s_phy[k] = make_float2(co, s);
        }
        __syncthreads();
        // threads -> (column, row group) with shifts: 64 columns per pass for
        // blocks of >= 64 threads, 32 for a 32-thread block (two passes);
        // the row step blockDim >> cshift is >= 1 for every allowed block size
        const int cshift = blockDim.x >= kTile ? 6 : 5;
        const int cols = 1 << cshift;
        const int rstep = blockDim.x >> cshift;
        for (int xx = tid & (cols - 1); xx < kTile; xx += cols) {
            const int gx = bx0 + xx;
            const bool xin = xx < ex && gx >= 0 && gx < a.ng;
            const float2 px = xin ? s_phx[xx] : make_float2(0.f, 0.f);
            for (int yy = tid >> cshift; yy < ey; yy += rstep) {
                const int gy = by0 + yy;
                float2 g = make_float2(0.f, 0.f);
                if (xin && gy >= 0 && gy < a.ng) g = __ldg(&a.grid[(size_t)gy * a.ng + gx]);
                s_tile[yy * kTile + xx] = cmul(g, cmul(px, s_phy[yy]));
            }
        }
        __syncthreads();
    }

    // ---- per-visibility tap sums (relative to origin (ox, oy)) ----
    const int ox = staged ? bx0 : ix0;
    const int oy = staged ? by0 : iy0;
    float2 S0 = make_float2(0.f, 0.f), Su = S0, Sv = S0;
    const float hx = fx + (float)(a.support / 2 - 1);   // dx of tap 0 (cells)
    const float hy = fy + (float)(a.support / 2 - 1);
    if (valid) {
        const ChanConst ch = a.chan[c];
        const float2 *tab = s_tab + lc * tab_stride;
        const unsigned tab_adj = (unsigned)__cvta_generic_to_shared(tab) - (0x4B000000u << 3);
        const float ov = (float)a.ov;
        const float rmax = ch.rho_max;
        const float rmax2 = rmax * rmax;
        const int b_lo = max(0, (int)floorf(hy - rmax) + 1);
        const int b_hi = min(a.support - 1, (int)ceilf(hy + rmax) - 1);
        float sdx = 0.f, cdx = 0.f;
        if (!staged) sincospif(-a.du * L, &sdx, &cdx);     // per-column ramp step
        for (int b = b_lo; b <= b_hi; ++b) {
            const float dy = hy - (float)b;
            const float rem = rmax2 - dy * dy;
            if (!(rem > 0.f)) continue;
            const float r = rem * rsqrt_fast(rem);
            const int a_lo = max(0, (int)floorf(hx - r) + 1);
            const int a_hi = min(a.support - 1, (int)ceilf(hx + r) - 1);
            const float dyo = dy * ov;
            const float dyo2 = fmaf(dyo, dyo, 1e-20f);
            float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
            const float dxo = (hx - (float)a_lo) * ov;
            if (staged) {
                const float2 *row = s_tile + (iy0 - oy + b) * kTile + (ix0 - ox) + a_lo;
                row_taps(row, a_hi - a_lo + 1, dxo, dyo2, ov, tab_adj, pr, pi, qr, qi);
            } else {
                // ramp exp(-i pi du (a L + b M)) relative to this visibility's window origin
                float sz, cz;
                sincospif(-a.du * ((float)a_lo * L + (float)b * M), &sz, &cz);
                float2 z = make_float2(cz, sz);
                const float2 step = make_float2(cdx, sdx);
                const int gy = iy0 + b;
                float dd = dxo;
                for (int aa = a_lo; aa <= a_hi; ++aa, dd -= ov) {
                    const int gx = ix0 + aa;
                    float2 g = make_float2(0.f, 0.f);
                    if (gx >= 0 && gx < a.ng && gy >= 0 && gy < a.ng) g = __ldg(&a.grid[(size_t)gy * a.ng + gx]);
                    g = cmul(g, z);
                    z = cmul(z, step);
                    const float s2 = fmaf(dd, dd, dyo2);
                    const float tv = s2 * rsqrt_fast(s2);
                    const float tf = __fadd_rz(tv, 8388608.0f);
                    const float2 e = lds_f2(tab_adj + ((unsigned)__float_as_int(tf) << 3));
                    const float A = fmaf(tv - (tf - 8388608.0f), e.y, e.x);
                    pr = fmaf(A, g.x, pr);
                    pi = fmaf(A, g.y, pi);
                    const float Ad = A * dd;
                    qr = fmaf(Ad, g.x, qr);
                    qi = fmaf(Ad, g.y, qi);
                }
            }
            S0.x += pr; S0.y += pi;
            Su.x += qr; Su.y += qi;
            Sv.x = fmaf(dy, pr, Sv.x);
            Sv.y = fmaf(dy, pi, Sv.y);
        }
        const float inv_ov = 1.0f / ov;
        Su.x *= inv_ov; Su.y *= inv_ov;                  // Q was accumulated with dx * ov
    }

    // ---- epilogue: visibility half of the ramp, decorrelation, derivatives ----
    float acc[kRed];
#pragma unroll
    for (int k = 0; k < kRed; ++k) acc[k] = 0.f;
    if (valid) {
        const float ph_arg = a.du * (((float)(ix0 - ox) + hx) * L + ((float)(iy0 - oy) + hy) * M);
        float s, co;
        sincospif(ph_arg, &s, &co);
        const float2 ph = make_float2(co, s);
        const float2 T0 = cmul(ph, S0);
        float2 Tu = cmul(ph, Su), Tv = cmul(ph, Sv);
        Tu.x *= a.du; Tu.y *= a.du;          // tap offsets in wavelengths
        Tv.x *= a.du; Tv.y *= a.du;
        const float al2 = a.chan[c].alpha2;
        float D = 1.f, el = 0.f, em = 0.f;
        if (a.decorrelation) {
            D = expf(-0.5f * al2 * (dL * dL + dM * dM));
            el = -dL * al2;                  // (l_j - l_i) alpha^2
            em = -dM * al2;
        }
        const float pi_f = 3.14159265358979f;
        const float2 V = make_float2(D * T0.x, D * T0.y);
        // d/dl_i = D [(l_j - l_i) a^2 T0 + i pi Tu]; d/dl_j flips the first term; m likewise
        const float2 dli = make_float2(D * (el * T0.x - pi_f * Tu.y), D * (el * T0.y + pi_f * Tu.x));
        const float2 dmi = make_float2(D * (em * T0.x - pi_f * Tv.y), D * (em * T0.y + pi_f * Tv.x));
        const float2 dlj = make_float2(D * (-el * T0.x - pi_f * Tu.y), D * (-el * T0.y + pi_f * Tu.x));
        const float2 dmj = make_float2(D * (-em * T0.x - pi_f * Tv.y), D * (-em * T0.y + pi_f * Tv.x));
        const size_t k = ((size_t)t * a.n_bl + bl) * a.nc + c;
        if (kPredict) {
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
        // ---- block reduction: FP32 within a warp, FP64 across warps ----
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
            for (int k = 0; k < kRed; ++k) s_red[warp][k] = (double)acc[k];
        }
        __syncthreads();
        if (tid < kRed) {
            double s = 0.0;
            const int nw = (blockDim.x + 31) >> 5;
            for (int wi = 0; wi < nw; ++wi) s += s_red[wi][tid];
            a.partials[(size_t)tid * a.n_bricks + brick] = s;      // [kRed][n_bricks]
        }
    }
    }                                                 // not skipped
    if (!persistent) return;
    }                                                 // brick loop
}

// Second stage (a): per-baseline sums over its bricks, one warp per baseline,
// a fixed butterfly order (deterministic).  partials is [kRed][n_bricks] with
// the bricks of baseline bl at [bl * bpb, (bl + 1) * bpb).  Batched form: the
// global warp number runs over the baselines of all contexts (bl_prefix).
__global__ void bl_reduce_kernel(const RedArgs r0, const RedArgs *__restrict__ ra,
                                 const int *__restrict__ bl_prefix, int n_ctx) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    RedArgs r = r0;
    int bl = gw;
    if (ra != nullptr) {
        if (gw >= bl_prefix[n_ctx]) return;
        int lo = 0, hi = n_ctx - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bl_prefix[mid] <= gw) lo = mid; else hi = mid - 1;
        }
        r = ra[lo];
        bl = gw - bl_prefix[lo];
    }
    if (bl >= r.n_bl) return;
    if (r.skip != nullptr && *r.skip) return;
    const size_t nb = (size_t)r.n_bl * r.bpb;
    for (int k = 0; k < kRed; ++k) {
        const double *p = r.partials + (size_t)k * nb + (size_t)bl * r.bpb;
        double sum = 0.0;
        for (int b = lane; b < r.bpb; b += 32) sum += p[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) r.blsum[(size_t)bl * kRed + k] = sum;
    }
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

}  // namespace

size_t eval_dyn_smem(int c_group, int max_tab_len) {
    return sizeof(float2) * (size_t)c_group * (max_tab_len + kTabPad);
}

cudaError_t launch_eval(const EvalArgs &a, bool predict, cudaStream_t s) {
    const int threads = a.t_tile * a.c_group;
    const int blocks = (int)a.n_bricks;
    const size_t dyn = eval_dyn_smem(a.c_group, a.max_tab_len);
    if (predict) {
        eval_kernel<true><<<blocks, threads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr);
    } else {
        eval_kernel<false><<<blocks, threads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_eval_batch(const EvalArgs *args_dev, const long long *prefix_dev, int n_ctx,
                              unsigned long long *queue, int threads, size_t dyn, int grid, cudaStream_t s) {
    EvalArgs none{};
    eval_kernel<false><<<grid, threads, dyn, s>>>(none, args_dev, prefix_dev, n_ctx, queue);
    return cudaGetLastError();
}

cudaError_t eval_batch_occupancy(int threads, size_t dyn, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, eval_kernel<false>, threads, dyn);
}

// Raises the fused kernel's dynamic shared-memory limit to everything the
// device allows beyond its static shared memory (never lowers it, so contexts
// with different channel groups can share the kernel), after checking that
// `dyn` bytes fit.
cudaError_t set_eval_smem(size_t dyn) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, eval_kernel<false>);
    if (e != cudaSuccess) return e;
    const size_t allowed = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (dyn > allowed) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(eval_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)allowed);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(eval_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)allowed);
}

cudaError_t launch_reduce(const RedArgs &r, cudaStream_t s) {
    const int warps_per_block = 8;
    bl_reduce_kernel<<<(r.n_bl + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(
        r, nullptr, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ev_kernel<<<1, kMaxThreads, 0, s>>>(r, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_reduce_batch(const RedArgs *ra_dev, const int *bl_prefix_dev, int n_ctx, int total_bl,
                                cudaStream_t s) {
    const int warps_per_block = 8;
    RedArgs none{};
    bl_reduce_kernel<<<(total_bl + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(
        none, ra_dev, bl_prefix_dev, n_ctx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ev_kernel<<<n_ctx, kMaxThreads, 0, s>>>(none, ra_dev);
    return cudaGetLastError();
}

}  // namespace psc

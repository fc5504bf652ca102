// Levenberg-Marquardt update on the device (Algorithm 1's Terminate() and
// f(), left to the minimiser by the paper, Sec. 2.2).
//
// One thread block per context.  After each fused evaluation at the trial
// offsets it (1) accepts the trial if chi^2 went down (lam /= 10, floored at
// lam_min) or rejects it (lam *= 10), (2) applies the stop rules, and (3) solves
// the damped system (H + lam diag(H)) delta = -g for the next trial, either
// over all 2 n_ant parameters (the full Gauss-Newton matrix: per-antenna 2x2
// diagonal blocks and one 2x2 cross block per baseline) or per antenna from
// the diagonal block alone with the step scaled by the loop gain block_gain.
// Parameters whose diagonal is not positive (antennas with no data) are held
// fixed.
//
// Precision.  The damped matrix and right-hand side are assembled in FP64.
// GB300 runs FP64 at a small fraction of its FP32 rate, so the full system is
// factored in FP32 (Cholesky) and the solution is refined in FP64: the
// residual b - A x is formed in FP64 and the correction solved with the FP32
// factor, until max|r| <= 1e-12 max|b| (at most 6 rounds).  That gives the
// FP64 solution for any matrix whose condition number is well below 1e7.  If
// the FP32 factorisation meets a non-positive pivot or the refinement does
// not converge, the system is factored in FP64 instead.
//
// Small systems live in shared memory and are factored column by column.
// Large ones (2 n_ant above 90, e.g. 394 x 394 for 197 antennas) live in
// global memory, where a column-by-column update would wait on one L2 round
// trip per element: they are factored in panels of 32 columns (diagonal block
// in shared memory, rows below solved from registers, trailing update in
// 64 x 64 tiles staged in shared memory), solved in blocks of 32 rows, and the
// FP64 residual is formed one warp per row with coalesced loads.
#include <math.h>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kLmThreads = 256;
constexpr int kSmallN2 = 90;            // 2 n_ant up to this: matrices in shared memory
constexpr int kRefineMax = 6;
constexpr double kRefineTol = 1e-12;
constexpr int kPan = 32;                // panel width of the blocked factorisation
constexpr int kTile = 64;               // trailing-update tile, 4 x 4 elements per thread
constexpr int kLd = kPan + 1;           // padded row of the shared tiles
constexpr int kWsFloats = 2 * kTile * kLd;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ double block_max(double v, double *s) {
    const int tid = threadIdx.x;
    s[tid] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) s[tid] = fmax(s[tid], s[tid + o]);
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

// FP32 Cholesky A = L L^T in place (row-major, lower triangle), all threads
// of the block.  Returns nonzero (uniformly) if a pivot is not positive.
__device__ int chol32(float *A, int n) {
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;            // 16 x 16 thread grid
    int bad = 0;
    for (int k = 0; k < n; ++k) {
        const float d = A[(size_t)k * n + k];
        const bool nonpos = !(d > 0.f);
        bad |= nonpos;
        const float inv = nonpos ? 1.f : rsqrtf(d);
        for (int i = k + 1 + tid; i < n; i += blockDim.x) A[(size_t)i * n + k] *= inv;
        __syncthreads();
        for (int i = k + 1 + ty; i < n; i += 16) {
            const float lik = A[(size_t)i * n + k];
            for (int j = k + 1 + tx; j <= i; j += 16) A[(size_t)i * n + j] -= lik * A[(size_t)j * n + k];
        }
        __syncthreads();
        if (tid == 0) A[(size_t)k * n + k] = nonpos ? 1.f : d * inv;
    }
    __syncthreads();
    return bad;
}

// Solves L L^T y = y in place with the FP32 factor, warp 0 only.
__device__ void solve32_warp(const float *L, int n, float *y) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < n; ++k) {
        const float yk = y[k] / L[(size_t)k * n + k];
        __syncwarp();
        if (lane == 0) y[k] = yk;
        for (int i = k + 1 + lane; i < n; i += 32) y[i] -= L[(size_t)i * n + k] * yk;
        __syncwarp();
    }
    for (int k = n - 1; k >= 0; --k) {
        const float xk = y[k] / L[(size_t)k * n + k];
        __syncwarp();
        if (lane == 0) y[k] = xk;
        for (int i = lane; i < k; i += 32) y[i] -= L[(size_t)k * n + i] * xk;
        __syncwarp();
    }
}

// Blocked FP32 Cholesky A = L L^T of the row-major n x n matrix in global
// memory (lower triangle read and written; the upper one is left as it was),
// all threads of the block (256).  ws: kWsFloats floats of shared memory.
// Returns nonzero (uniformly) if a pivot is not positive.
__device__ int chol32_blocked(float *A, int n, float *ws) {
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid & 15, ty = tid >> 4;            // 16 x 16 threads, 4 x 4 elements each
    float *D = ws;                                     // diagonal block; column kPan holds 1 / L_cc
    float *Li = ws, *Lj = ws + kTile * kLd;            // trailing-update tiles (D is dead by then)
    if (tid == 0) s_bad = 0;
    for (int k0 = 0; k0 < n; k0 += kPan) {
        const int kb = min(kPan, n - k0), m0 = k0 + kb;
        for (int e = tid; e < kPan * kPan; e += blockDim.x) {
            const int r = e / kPan, c = e % kPan;
            D[r * kLd + c] = (r < kb && c <= r) ? A[(size_t)(k0 + r) * n + k0 + c] : 0.f;
        }
        __syncthreads();
        if (warp == 0) {                               // factor the diagonal block, lane r owns row r
            for (int c = 0; c < kb; ++c) {
                const float d = D[c * kLd + c];
                const bool nonpos = !(d > 0.f);
                const float lcc = nonpos ? 1.f : sqrtf(d), inv = 1.f / lcc;
                __syncwarp();
                if (lane == c) { D[c * kLd + c] = lcc; D[c * kLd + kPan] = inv; }
                if (lane > c && lane < kb) D[lane * kLd + c] *= inv;
                __syncwarp();
                if (lane > c && lane < kb) {
                    const float lrc = D[lane * kLd + c];
                    for (int t = c + 1; t <= lane; ++t) D[lane * kLd + t] -= lrc * D[t * kLd + c];
                }
                __syncwarp();
                if (nonpos && lane == 0) s_bad = 1;
            }
        }
        __syncthreads();
        for (int e = tid; e < kb * kb; e += blockDim.x) {
            const int r = e / kb, c = e % kb;
            if (c <= r) A[(size_t)(k0 + r) * n + k0 + c] = D[r * kLd + c];
        }
        // rows below: L21 = A21 L11^-T, one thread per row (a panel with rows
        // below is always full, kb = kPan)
        for (int i = m0 + tid; i < n; i += blockDim.x) {
            float *row = A + (size_t)i * n + k0;
            float x[kPan];
#pragma unroll
            for (int c = 0; c < kPan; ++c) x[c] = row[c];
#pragma unroll
            for (int c = 0; c < kPan; ++c) {
                float v = x[c];
#pragma unroll
                for (int t = 0; t < c; ++t) v = fmaf(-x[t], D[c * kLd + t], v);
                x[c] = v * D[c * kLd + kPan];
            }
#pragma unroll
            for (int c = 0; c < kPan; ++c) row[c] = x[c];
        }
        __syncthreads();
        // trailing update: A22 -= L21 L21^T on the lower triangle, tile by tile
        const int nt = (n - m0 + kTile - 1) / kTile;
        for (int ti = 0; ti < nt; ++ti) {
            for (int tj = 0; tj <= ti; ++tj) {
                const int i0 = m0 + ti * kTile, j0 = m0 + tj * kTile;
                for (int e = tid; e < kTile * kPan; e += blockDim.x) {
                    const int r = e / kPan, c = e % kPan;
                    Li[r * kLd + c] = i0 + r < n ? A[(size_t)(i0 + r) * n + k0 + c] : 0.f;
                    Lj[r * kLd + c] = j0 + r < n ? A[(size_t)(j0 + r) * n + k0 + c] : 0.f;
                }
                __syncthreads();
                float acc[4][4] = {};
#pragma unroll 8
                for (int t = 0; t < kPan; ++t) {
                    float li[4], lj[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) li[r] = Li[(ty + 16 * r) * kLd + t];
#pragma unroll
                    for (int c = 0; c < 4; ++c) lj[c] = Lj[(tx + 16 * c) * kLd + t];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(li[r], lj[c], acc[r][c]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int i = i0 + ty + 16 * r;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int j = j0 + tx + 16 * c;
                        if (i < n && j <= i) A[(size_t)i * n + j] -= acc[r][c];
                    }
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    return s_bad;
}

// Solves L L^T y = y in place (y in shared memory) with the factor of
// chol32_blocked, all threads of the block, in blocks of kPan rows: the
// off-diagonal part of each block as warp dot products over rows of L (forward)
// or columns of L (backward), the diagonal block by warp 0 from registers.
// red: 8 x 32 floats of shared memory.
__device__ void solve32_blocked(const float *L, int n, float *y, float *red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int k0 = 0; k0 < n; k0 += kPan) {             // L z = y
        const int kb = min(kPan, n - k0);
        for (int r = warp; r < kb; r += nw) {
            const float *row = L + (size_t)(k0 + r) * n;
            float p = 0.f;
            for (int j = lane; j < k0; j += 32) p = fmaf(row[j], y[j], p);
            p = warp_sum(p);
            if (lane == 0) y[k0 + r] -= p;
        }
        __syncthreads();
        if (warp == 0) {
            const float *row = L + (size_t)(k0 + lane) * n + k0;
            float l[kPan], d = 1.f;
#pragma unroll
            for (int c = 0; c < kPan; ++c) {
                l[c] = (lane < kb && c <= lane) ? row[c] : 0.f;
                if (c == lane && lane < kb) d = l[c];
            }
            const float inv = 1.f / d;
            float s = lane < kb ? y[k0 + lane] : 0.f;
#pragma unroll
            for (int c = 0; c < kPan; ++c) {
                const float zc = __shfl_sync(kFull, s * inv, c);
                if (lane > c) s = fmaf(-l[c], zc, s);
            }
            if (lane < kb) y[k0 + lane] = s * inv;
        }
        __syncthreads();
    }
    for (int k0 = ((n - 1) / kPan) * kPan; k0 >= 0; k0 -= kPan) {     // L^T x = z
        const int kb = min(kPan, n - k0), m0 = k0 + kb;
        float p = 0.f;
        if (lane < kb)
            for (int j = m0 + warp; j < n; j += nw) p = fmaf(L[(size_t)j * n + k0 + lane], y[j], p);
        red[warp * 32 + lane] = p;
        __syncthreads();
        if (warp == 0) {
            float s = 0.f;
            for (int w = 0; w < nw; ++w) s += red[w * 32 + lane];
            float col[kPan], d = 1.f;                  // lane r: column r of the diagonal block
#pragma unroll
            for (int j = 0; j < kPan; ++j) {
                col[j] = (lane < kb && j >= lane && j < kb) ? L[(size_t)(k0 + j) * n + k0 + lane] : 0.f;
                if (j == lane && lane < kb) d = col[j];
            }
            const float inv = 1.f / d;
            s = lane < kb ? y[k0 + lane] - s : 0.f;
#pragma unroll
            for (int c = kPan - 1; c >= 0; --c) {
                const float xc = __shfl_sync(kFull, s * inv, c);
                if (lane < c) s = fmaf(-col[c], xc, s);
            }
            if (lane < kb) y[k0 + lane] = s * inv;
        }
        __syncthreads();
    }
}

// FP64 Cholesky + solve of A x = b in place (x overwrites b), all threads.
__device__ int chol64_solve(double *A, int n2, double *b) {
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n2; ++k) {
        if (tid == 0) {
            const double d = A[(size_t)k * n2 + k];
            if (!(d > 0.0)) { s_bad = 1; A[(size_t)k * n2 + k] = 1.0; }
            else A[(size_t)k * n2 + k] = sqrt(d);
        }
        __syncthreads();
        const double lkk = A[(size_t)k * n2 + k];
        for (int i = k + 1 + tid; i < n2; i += blockDim.x) A[(size_t)i * n2 + k] /= lkk;
        __syncthreads();
        const int tx = tid & 15, ty = tid >> 4;
        for (int i = k + 1 + ty; i < n2; i += 16) {
            const double lik = A[(size_t)i * n2 + k];
            for (int j = k + 1 + tx; j <= i; j += 16) A[(size_t)i * n2 + j] -= lik * A[(size_t)j * n2 + k];
        }
        __syncthreads();
    }
    for (int k = 0; k < n2; ++k) {
        if (tid == 0) b[k] /= A[(size_t)k * n2 + k];
        __syncthreads();
        const double yk = b[k];
        for (int i = k + 1 + tid; i < n2; i += blockDim.x) b[i] -= A[(size_t)i * n2 + k] * yk;
        __syncthreads();
    }
    for (int k = n2 - 1; k >= 0; --k) {
        if (tid == 0) b[k] /= A[(size_t)k * n2 + k];
        __syncthreads();
        const double xk = b[k];
        for (int i = tid; i < k; i += blockDim.x) b[i] -= A[(size_t)k * n2 + i] * xk;
        __syncthreads();
    }
    return s_bad;
}

__global__ void __launch_bounds__(kLmThreads) lm_update_kernel(const LMArgs a0, const LMArgs *__restrict__ la) {
    extern __shared__ double s_dyn[];
    const LMArgs a = la != nullptr ? la[blockIdx.x] : a0;     // batched: one block per context
    const int small = 2 * a.n_ant <= kSmallN2;
    LMState *st = a.st;
    if (st->done) return;
    __shared__ int s_accept, s_stop;
    __shared__ double s_lam;
    __shared__ int s_fail;
    __shared__ double s_tmp[kLmThreads];
    const int tid = threadIdx.x;
    const int n = a.n_ant, n2 = 2 * n;
    const size_t len = ev_len(n, a.n_bl);

    // the step that produced this trial (its largest component)
    double tstep = 0.0;
    for (int p = tid; p < n2; p += blockDim.x) tstep = fmax(tstep, fabs(a.lm_trial[p] - a.lm_cur[p]));
    tstep = block_max(tstep, s_tmp);

    if (tid == 0) {
        const double chi2_t = a.ev[0];
        int accept = 0, stop = PSC_STOP_NONE;
        double lam = st->lam;
        if (st->n_eval == 0) {
            if (isfinite(chi2_t)) accept = 1;
            else stop = PSC_STOP_NUMERIC;
        } else if (isfinite(chi2_t) && chi2_t < st->chi2) {
            accept = 1;
            const double rel = st->chi2 > 0.0 ? (st->chi2 - chi2_t) / st->chi2 : 0.0;
            lam = fmax(lam / 10.0, st->lam_min);
            if (rel < st->chi2_rtol) stop = PSC_STOP_CHI2;
        } else {
            lam *= 10.0;
            if (lam > st->lam_max) stop = PSC_STOP_LAMBDA;
            // a rejected step already below ten times the step tolerance: the
            // minimum is found to within the evaluation's own noise, and a
            // rising lam would only shrink the step to the tolerance
            else if (isfinite(chi2_t) && tstep < 10.0 * st->step_tol) stop = PSC_STOP_STEP;
        }
        st->n_eval += 1;
        if (accept) st->chi2 = chi2_t;
        if (stop == PSC_STOP_NONE && st->n_iter >= st->max_iter) stop = PSC_STOP_MAX_ITER;
        st->lam = lam;
        s_lam = lam;
        s_accept = accept;
        s_stop = stop;
        s_fail = 0;
    }
    __syncthreads();
    if (s_accept) {
        for (size_t k = tid; k < len; k += blockDim.x) a.cur[k] = a.ev[k];
        for (int k = tid; k < n2; k += blockDim.x) a.lm_cur[k] = a.lm_trial[k];
    }
    __syncthreads();
    if (s_stop != PSC_STOP_NONE) {
        if (tid == 0) { st->reason = s_stop; st->done = 1; }
        return;
    }
    if (tid == 0) st->n_iter += 1;

    const double lam = s_lam;
    const double *g = a.cur + 1;
    const double *H = a.cur + 1 + n2;
    const double *X = a.cur + 1 + n2 + 3 * (size_t)n;
    double *delta = a.rhs;

    if (st->mode == PSC_LM_BLOCK) {
        for (int an = tid; an < n; an += blockDim.x) {
            const double p = H[3 * an] * (1.0 + lam), b = H[3 * an + 1], d = H[3 * an + 2] * (1.0 + lam);
            const double det = p * d - b * b;
            double x0 = 0.0, x1 = 0.0;
            if (det > 0.0 && p > 0.0) {
                x0 = -(d * g[2 * an] - b * g[2 * an + 1]) / det;
                x1 = -(-b * g[2 * an] + p * g[2 * an + 1]) / det;
            }
            delta[2 * an] = st->block_gain * x0;
            delta[2 * an + 1] = st->block_gain * x1;
        }
        __syncthreads();
    } else {
        // dynamic shared memory: [A64 | A32] (small systems only) then b, r (FP64),
        // y32, and the blocked factorisation's tiles (large systems only)
        double *A = small ? s_dyn : a.mat;
        float *A32 = small ? (float *)(s_dyn + (size_t)n2 * n2) : a.mat32;
        double *vb = small ? s_dyn + (size_t)n2 * n2 + ((size_t)n2 * n2 + 1) / 2 : s_dyn;
        double *vr = vb + n2;
        float *y32 = (float *)(vr + n2);
        float *ws = y32 + n2;

        // assemble H + lam diag(H) (FP64, both triangles) and b = -g
        for (size_t k = tid; k < (size_t)n2 * n2; k += blockDim.x) A[k] = 0.0;
        __syncthreads();
        for (int an = tid; an < n; an += blockDim.x) {
            const double hll = H[3 * an], hlm = H[3 * an + 1], hmm = H[3 * an + 2];
            const int p = 2 * an;
            A[(size_t)p * n2 + p] = hll * (1.0 + lam);
            A[(size_t)p * n2 + p + 1] = hlm;
            A[(size_t)(p + 1) * n2 + p] = hlm;
            A[(size_t)(p + 1) * n2 + p + 1] = hmm * (1.0 + lam);
            vb[p] = -g[p];
            vb[p + 1] = -g[p + 1];
        }
        for (int bl = tid; bl < a.n_bl; bl += blockDim.x) {
            const int2 ij = a.pairs[bl];
            const int p = 2 * ij.x, q = 2 * ij.y;
            const double *x = X + 4 * (size_t)bl;
            A[(size_t)p * n2 + q] = x[0];       A[(size_t)q * n2 + p] = x[0];
            A[(size_t)p * n2 + q + 1] = x[1];   A[(size_t)(q + 1) * n2 + p] = x[1];
            A[(size_t)(p + 1) * n2 + q] = x[2]; A[(size_t)q * n2 + p + 1] = x[2];
            A[(size_t)(p + 1) * n2 + q + 1] = x[3]; A[(size_t)(q + 1) * n2 + p + 1] = x[3];
        }
        __syncthreads();
        // hold parameters without data fixed
        for (int p = tid; p < n2; p += blockDim.x) {
            if (!(A[(size_t)p * n2 + p] > 0.0)) {
                for (int q = 0; q < n2; ++q) { A[(size_t)p * n2 + q] = 0.0; A[(size_t)q * n2 + p] = 0.0; }
            }
        }
        __syncthreads();
        for (int p = tid; p < n2; p += blockDim.x) {
            if (A[(size_t)p * n2 + p] == 0.0) { A[(size_t)p * n2 + p] = 1.0; vb[p] = 0.0; }
            delta[p] = 0.0;
        }
        __syncthreads();
        for (size_t k = tid; k < (size_t)n2 * n2; k += blockDim.x) A32[k] = (float)A[k];
        __syncthreads();

        const int bad = small ? chol32(A32, n2) : chol32_blocked(A32, n2, ws);
        double bmax = 0.0;
        for (int p = tid; p < n2; p += blockDim.x) { bmax = fmax(bmax, fabs(vb[p])); vr[p] = vb[p]; }
        bmax = block_max(bmax, s_tmp);
        bool converged = false;
        for (int it = 0; it < kRefineMax && !bad && !converged; ++it) {
            for (int p = tid; p < n2; p += blockDim.x) y32[p] = (float)vr[p];
            __syncthreads();
            if (small) {
                if (tid < 32) solve32_warp(A32, n2, y32);
            } else {
                solve32_blocked(A32, n2, y32, ws);
            }
            __syncthreads();
            for (int p = tid; p < n2; p += blockDim.x) delta[p] += (double)y32[p];
            __syncthreads();
            double rmax = 0.0;
            if (small) {
                for (int p = tid; p < n2; p += blockDim.x) {     // r = b - A x in FP64
                    double acc = vb[p];
                    const double *row = A + (size_t)p * n2;
                    for (int q = 0; q < n2; ++q) acc = fma(-row[q], delta[q], acc);
                    vr[p] = acc;
                    rmax = fmax(rmax, fabs(acc));
                }
            } else {
                const int lane = tid & 31, nw = blockDim.x >> 5;
                for (int p = tid >> 5; p < n2; p += nw) {       // one warp per row
                    const double *row = A + (size_t)p * n2;
                    double acc = 0.0;
                    for (int q = lane; q < n2; q += 32) acc = fma(row[q], delta[q], acc);
                    const double r = vb[p] - warp_sum(acc);
                    if (lane == 0) vr[p] = r;
                    rmax = fmax(rmax, fabs(r));
                }
            }
            rmax = block_max(rmax, s_tmp);
            converged = rmax <= kRefineTol * bmax;
        }
        if (bad || !converged) {
            // FP64 fallback: factor the FP64 matrix itself
            for (int p = tid; p < n2; p += blockDim.x) delta[p] = vb[p];
            __syncthreads();
            const int bad64 = chol64_solve(A, n2, delta);
            if (bad64 && tid == 0) s_fail = 1;
            __syncthreads();
        }
    }

    double mx = 0.0;
    bool finite = true;
    for (int p = tid; p < n2; p += blockDim.x) {
        mx = fmax(mx, fabs(delta[p]));
        if (!isfinite(delta[p])) finite = false;
    }
    mx = block_max(finite ? mx : INFINITY, s_tmp);
    if (tid == 0) {
        if (s_fail || !isfinite(mx)) { st->reason = PSC_STOP_NUMERIC; st->done = 1; }
        else if (mx < st->step_tol) { st->reason = PSC_STOP_STEP; st->done = 1; }
    }
    __syncthreads();
    if (st->done) return;
    for (int p = tid; p < n2; p += blockDim.x) a.lm_trial[p] = a.lm_cur[p] + delta[p];
}

__global__ void lm_restart_kernel(const LMArgs a0, const LMState *st00, const double *lm00,
                                  const LMArgs *__restrict__ la, const LMState *const *st0s,
                                  const double *const *lm0s) {
    const bool batched = la != nullptr;
    const LMArgs a = batched ? la[blockIdx.x] : a0;
    const LMState *st0 = batched ? st0s[blockIdx.x] : st00;
    const double *lm0 = batched ? lm0s[blockIdx.x] : lm00;
    if (threadIdx.x == 0) *a.st = *st0;
    for (int p = threadIdx.x; p < 2 * a.n_ant; p += blockDim.x) {
        a.lm_trial[p] = lm0[p];
        a.lm_cur[p] = lm0[p];
    }
}

// Dynamic shared memory of the LM kernel: the FP64 matrix and its FP32 copy
// for small systems, then b, r (FP64) and y (FP32), 2 n_ant each, then the
// blocked factorisation's tiles for large systems.
size_t lm_dyn_smem(int n_ant) {
    const size_t n2 = 2 * (size_t)n_ant;
    const size_t vec = sizeof(double) * 2 * n2 + sizeof(float) * n2;
    if ((int)n2 <= kSmallN2) return sizeof(double) * (n2 * n2 + (n2 * n2 + 1) / 2) + vec;
    return vec + sizeof(float) * kWsFloats;
}

}  // namespace

cudaError_t lm_prepare(int n_ant) {
    (void)n_ant;
    const size_t most = lm_dyn_smem(kSmallN2 / 2) > lm_dyn_smem(512) ? lm_dyn_smem(kSmallN2 / 2) : lm_dyn_smem(512);
    return cudaFuncSetAttribute(lm_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
}

size_t lm_smem_bytes(int n_ant) { return lm_dyn_smem(n_ant); }

cudaError_t launch_lm_restart(const LMArgs &a, const LMState *st0, const double *lm0, cudaStream_t s) {
    lm_restart_kernel<<<1, 128, 0, s>>>(a, st0, lm0, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_lm_restart_batch(const LMArgs *la_dev, const LMState *const *st0_dev,
                                    const double *const *lm0_dev, int n_ctx, cudaStream_t s) {
    LMArgs none{};
    lm_restart_kernel<<<n_ctx, 128, 0, s>>>(none, nullptr, nullptr, la_dev, st0_dev, lm0_dev);
    return cudaGetLastError();
}

cudaError_t launch_lm_update(const LMArgs &a, cudaStream_t s) {
    lm_update_kernel<<<1, kLmThreads, lm_dyn_smem(a.n_ant), s>>>(a, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_lm_update_batch(const LMArgs *la_dev, int n_ctx, size_t dyn, cudaStream_t s) {
    LMArgs none{};
    lm_update_kernel<<<n_ctx, kLmThreads, dyn, s>>>(none, la_dev);
    return cudaGetLastError();
}

}  // namespace psc

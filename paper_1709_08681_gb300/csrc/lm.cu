// Levenberg-Marquardt update on the device, FP64 (Algorithm 1's Terminate()
// and f(), left to the minimiser by the paper, Sec. 2.2).
//
// One thread block per context.  After each fused evaluation at the trial
// offsets it (1) accepts the trial if chi^2 went down (lam /= 10, floored at
// lam_min) or rejects it (lam *= 10), (2) applies the stop rules, and (3) solves
// the damped system (H + lam diag(H)) delta = -g for the next trial, either
// over all 2 n_ant parameters (Cholesky of the full Gauss-Newton matrix:
// per-antenna 2x2 diagonal blocks and one 2x2 cross block per baseline) or
// per antenna from the diagonal block alone with the step scaled by the loop
// gain block_gain.  Parameters whose diagonal is not positive (antennas with
// no data) are held fixed.
#include <math.h>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kLmThreads = 256;

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

__global__ void __launch_bounds__(kLmThreads) lm_update_kernel(const LMArgs a) {
    LMState *st = a.st;
    if (st->done) return;
    __shared__ int s_accept, s_stop;
    __shared__ double s_lam;
    __shared__ int s_fail;
    __shared__ double s_tmp[kLmThreads];
    const int tid = threadIdx.x;
    const int n = a.n_ant, n2 = 2 * n;
    const size_t len = ev_len(n, a.n_bl);

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
        double *A = a.mat;                       // row-major [n2][n2]
        // assemble H + lam diag(H)
        for (size_t k = tid; k < (size_t)n2 * n2; k += blockDim.x) A[k] = 0.0;
        __syncthreads();
        for (int an = tid; an < n; an += blockDim.x) {
            const double hll = H[3 * an], hlm = H[3 * an + 1], hmm = H[3 * an + 2];
            const int p = 2 * an;
            A[(size_t)p * n2 + p] = hll * (1.0 + lam);
            A[(size_t)p * n2 + p + 1] = hlm;
            A[(size_t)(p + 1) * n2 + p] = hlm;
            A[(size_t)(p + 1) * n2 + p + 1] = hmm * (1.0 + lam);
            delta[p] = -g[p];
            delta[p + 1] = -g[p + 1];
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
            if (A[(size_t)p * n2 + p] == 0.0) { A[(size_t)p * n2 + p] = 1.0; delta[p] = 0.0; }
        }
        __syncthreads();
        // Cholesky A = L L^T in place (lower triangle), right-looking
        for (int k = 0; k < n2; ++k) {
            if (tid == 0) {
                const double d = A[(size_t)k * n2 + k];
                if (!(d > 0.0)) { s_fail = 1; A[(size_t)k * n2 + k] = 1.0; }
                else A[(size_t)k * n2 + k] = sqrt(d);
            }
            __syncthreads();
            const double lkk = A[(size_t)k * n2 + k];
            for (int i = k + 1 + tid; i < n2; i += blockDim.x) A[(size_t)i * n2 + k] /= lkk;
            __syncthreads();
            const int m = n2 - k - 1;
            for (int idx = tid; idx < m * m; idx += blockDim.x) {
                const int i = k + 1 + idx / m, j = k + 1 + idx % m;
                if (j <= i) A[(size_t)i * n2 + j] -= A[(size_t)i * n2 + k] * A[(size_t)j * n2 + k];
            }
            __syncthreads();
        }
        // forward: L y = -g
        for (int k = 0; k < n2; ++k) {
            if (tid == 0) delta[k] /= A[(size_t)k * n2 + k];
            __syncthreads();
            const double yk = delta[k];
            for (int i = k + 1 + tid; i < n2; i += blockDim.x) delta[i] -= A[(size_t)i * n2 + k] * yk;
            __syncthreads();
        }
        // backward: L^T x = y
        for (int k = n2 - 1; k >= 0; --k) {
            if (tid == 0) delta[k] /= A[(size_t)k * n2 + k];
            __syncthreads();
            const double xk = delta[k];
            for (int i = tid; i < k; i += blockDim.x) delta[i] -= A[(size_t)k * n2 + i] * xk;
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

__global__ void lm_restart_kernel(const LMArgs a, const LMState *st0, const double *lm0) {
    if (threadIdx.x == 0) *a.st = *st0;
    for (int p = threadIdx.x; p < 2 * a.n_ant; p += blockDim.x) {
        a.lm_trial[p] = lm0[p];
        a.lm_cur[p] = lm0[p];
    }
}

}  // namespace

cudaError_t launch_lm_restart(const LMArgs &a, const LMState *st0, const double *lm0, cudaStream_t s) {
    lm_restart_kernel<<<1, 128, 0, s>>>(a, st0, lm0);
    return cudaGetLastError();
}

cudaError_t launch_lm_update(const LMArgs &a, cudaStream_t s) {
    lm_update_kernel<<<1, kLmThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace psc

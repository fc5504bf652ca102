// Model grid V° = F[I^M] (Algorithm 1, first pre-compute; Eq. MEDD):
// the unnormalised DFT, sign exp(+2 pi i) as in Eq. ME, of the N x N image
// zero-padded to Ng x Ng,
//   G[gy][gx] = sum_{row,col} I[row][col] W((gx-Ng/2)(col-N/2)) W((gy-Ng/2)(row-N/2)),
//   W(k) = exp(2 pi i k / Ng),
// computed as two complex matrix products, T = I F^T (N x Ng) and G = F T,
// with F[g][c] = W((g - Ng/2)(c - N/2)) generated on the fly from a twiddle
// table (exact integer phase index modulo Ng, table values from FP64 sincospi).
// FP32 SIMT GEMM tiles: 64 x 64 outputs per 256-thread block, 4 x 4 per thread.
#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

__global__ void twiddle_kernel(float2 *W, int ng) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)ng, &s, &c);
        W[k] = make_float2((float)c, (float)s);
    }
}

__device__ __forceinline__ int phase_index(int g, int c, int ng, int n) {
    const long long p = (long long)(g - ng / 2) * (long long)(c - n / 2);
    long long r = p % ng;
    if (r < 0) r += ng;
    return (int)r;
}

// T[r][g] = sum_c I[r][c] F[g][c]      (rows r < N, columns g < Ng, depth c < N)
__global__ void __launch_bounds__(256) dft_rows_kernel(const float *__restrict__ img, const float2 *__restrict__ W,
                                                       int n, int ng, float2 *__restrict__ T) {
    __shared__ float As[kBK][kBM];
    __shared__ float2 Bs[kBK][kBN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += kBK) {
        for (int e = threadIdx.x; e < kBK * kBM; e += blockDim.x) {
            const int kk = e % kBK, mm = e / kBK;
            const int r = m0 + mm, c = k0 + kk;
            As[kk][mm] = (r < n && c < n) ? img[(size_t)r * n + c] : 0.f;
        }
        for (int e = threadIdx.x; e < kBK * kBN; e += blockDim.x) {
            const int nn = e % kBN, kk = e / kBN;
            const int g = n0 + nn, c = k0 + kk;
            Bs[kk][nn] = (g < ng && c < n) ? W[phase_index(g, c, ng, n)] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4];
            float2 b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(a[i], b[j].x, acc[i][j].x);
                    acc[i][j].y = fmaf(a[i], b[j].y, acc[i][j].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + ty + 16 * i, g = n0 + tx + 16 * j;
            if (r < n && g < ng) T[(size_t)r * ng + g] = acc[i][j];
        }
}

// G[gy][gx] = sum_r F[gy][r] T[r][gx]   (rows gy < Ng, columns gx < Ng, depth r < N)
__global__ void __launch_bounds__(256) dft_cols_kernel(const float2 *__restrict__ T, const float2 *__restrict__ W,
                                                       int n, int ng, float2 *__restrict__ G) {
    __shared__ float2 As[kBK][kBM];
    __shared__ float2 Bs[kBK][kBN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += kBK) {
        for (int e = threadIdx.x; e < kBK * kBM; e += blockDim.x) {
            const int kk = e % kBK, mm = e / kBK;
            const int gy = m0 + mm, r = k0 + kk;
            As[kk][mm] = (gy < ng && r < n) ? W[phase_index(gy, r, ng, n)] : make_float2(0.f, 0.f);
        }
        for (int e = threadIdx.x; e < kBK * kBN; e += blockDim.x) {
            const int nn = e % kBN, kk = e / kBN;
            const int gx = n0 + nn, r = k0 + kk;
            Bs[kk][nn] = (gx < ng && r < n) ? T[(size_t)r * ng + gx] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gy = m0 + ty + 16 * i, gx = n0 + tx + 16 * j;
            if (gy < ng && gx < ng) G[(size_t)gy * ng + gx] = acc[i][j];
        }
}

}  // namespace

cudaError_t launch_model_grid(int n_img, int n_grid, const float *image, float2 *tmp, float2 *twiddle,
                              float2 *grid_out, cudaStream_t s) {
    twiddle_kernel<<<(n_grid + 255) / 256, 256, 0, s>>>(twiddle, n_grid);
    dim3 g1((n_grid + kBN - 1) / kBN, (n_img + kBM - 1) / kBM);
    dft_rows_kernel<<<g1, 256, 0, s>>>(image, twiddle, n_img, n_grid, tmp);
    dim3 g2((n_grid + kBN - 1) / kBN, (n_grid + kBM - 1) / kBM);
    dft_cols_kernel<<<g2, 256, 0, s>>>(tmp, twiddle, n_img, n_grid, grid_out);
    return cudaGetLastError();
}

}  // namespace psc

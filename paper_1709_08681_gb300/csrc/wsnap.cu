// W-snapshots (Sec. 6.1 and the conclusions: for short solution intervals the
// array is treated as co-planar, so the w-term costs nothing in the degridding).
//
// With w = a u + b v within an interval, the phase u l + v m + w (n - 1) of a
// source at (l, m), n = sqrt(1 - l^2 - m^2), equals u l' + v m' with
// l' = l + a (n - 1), m' = m + b (n - 1): the co-planar path applies to the sky
// moved to (l', m').  The degridding kernel weights a source by the primary
// beam at its grid position, so each flux is rescaled by PB(l) / PB(l'), PB
// the pointing-free power pattern of the aperture at the given frequency.
//
// plane_sums_kernel accumulates the normal equations of the least-squares
// plane (FP64, one atomicAdd per block and sum); the host solves the 2 x 2
// system.  The source move runs on the host (n_comp values).
//
// What the plane leaves, w - a u - b v, is the residual w of the stacked
// model grids: wrange_kernel gives each block's (min, max) of it, which the
// host combines to size a stack or to check that one covers a context.
#include <algorithm>
#include <cmath>

#include "psc_internal.cuh"

namespace psc {
namespace {

__global__ void plane_sums_kernel(const double *__restrict__ uvw, long long n_rows, double *__restrict__ sums) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rows;
         r += (long long)gridDim.x * blockDim.x) {
        const double u = uvw[3 * r], v = uvw[3 * r + 1], w = uvw[3 * r + 2];
        acc[0] += u * u; acc[1] += u * v; acc[2] += v * v; acc[3] += u * w; acc[4] += v * w;
    }
    __shared__ double red[32][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double x = acc[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double x = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x + 31) / 32; ++wi) x += red[wi][threadIdx.x];
        atomicAdd(&sums[threadIdx.x], x);
    }
}

__global__ void wrange_kernel(const double *__restrict__ uvw, long long n_rows, double a, double b,
                              double *__restrict__ out) {
    double lo = INFINITY, hi = -INFINITY;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rows;
         r += (long long)gridDim.x * blockDim.x) {
        const double wr = uvw[3 * r + 2] - a * uvw[3 * r] - b * uvw[3 * r + 1];
        lo = fmin(lo, wr);
        hi = fmax(hi, wr);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ double red[32][2];
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = lo;
        red[threadIdx.x >> 5][1] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int wi = 1; wi < (int)(blockDim.x + 31) / 32; ++wi) {
            lo = fmin(lo, red[wi][0]);
            hi = fmax(hi, red[wi][1]);
        }
        out[2 * blockIdx.x] = lo;
        out[2 * blockIdx.x + 1] = hi;
    }
}

}  // namespace

cudaError_t launch_wrange(const double *uvw, long long n_rows, double a, double b, double *out_dev, int *blocks,
                          cudaStream_t s) {
    *blocks = (int)std::max<long long>(1, std::min<long long>((n_rows + 255) / 256, 1024));
    wrange_kernel<<<*blocks, 256, 0, s>>>(uvw, n_rows, a, b, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_plane_sums(const double *uvw, long long n_rows, double *sums_dev, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sums_dev, 0, 5 * sizeof(double), s);
    if (e != cudaSuccess || n_rows <= 0) return e;
    const int blocks = (int)std::min<long long>((n_rows + 255) / 256, 1024);
    plane_sums_kernel<<<blocks, 256, 0, s>>>(uvw, n_rows, sums_dev);
    return cudaGetLastError();
}

}  // namespace psc

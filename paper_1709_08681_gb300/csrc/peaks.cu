// FP32 FMA throughput of the device: the denominator check of the fused
// kernel's roofline (its bound is the FP32 pipe).  Every thread runs eight
// independent FMA chains; the result is folded into one store per thread so
// that nothing is eliminated.
#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_rate_kernel(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace psc

using namespace psc;

extern "C" psc_status psc_fp32_fma_rate(double *tflops, void *stream) {
    if (!tflops) return set_global_error(PSC_ERR_ARG, "tflops is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = n_sm * 8, threads = 256, iters = 1 << 15;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        fma_rate_kernel<<<blocks, threads, 0, s>>>(out, 1024, 0.999f, 1e-4f);        // warm
        cudaEventRecord(e0, s);
        fma_rate_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-4f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_global_error(PSC_ERR_CUDA, cudaGetErrorString(e));
    *tflops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    return PSC_OK;
}

// The learned initial estimate's MLP on the GPU: forward, backward and AdamW
// (an addition to the paper's method, which starts the minimiser from zero or
// from earlier solutions).
//
// Network 52 -> 256 -> 256 -> 256 -> 2, GELU (0.5 x (1 + erf(x / sqrt 2)))
// after the hidden layers, input standardised by fixed (mu, s).  Flat FP32
// parameter vector: W1 [52][256], b1, W2 [256][256], b2, W3 [256][256], b3,
// W4 [256][2], b4, mu [52], s [52]; y = x W + b.  Loss (1/B) sum (y - t)^2.
//
// Precision: FP32 master weights and AdamW state; every GEMM operand is
// bfloat16 (weights, standardised input, GELU outputs, output gradients),
// multiplied on the 5th-generation tensor cores (tcgen05.mma, FP32
// accumulator in tensor memory); biases, GELU, its derivative and the
// optimiser are FP32.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "psc_internal.cuh"

namespace psc {
namespace {

constexpr int kIn = 52, kHid = 256, kOut = 2;
constexpr size_t oW1 = 0, ob1 = oW1 + (size_t)kIn * kHid, oW2 = ob1 + kHid, ob2 = oW2 + (size_t)kHid * kHid,
                 oW3 = ob2 + kHid, ob3 = oW3 + (size_t)kHid * kHid, oW4 = ob3 + kHid, ob4 = oW4 + (size_t)kHid * kOut,
                 omu = ob4 + kOut, os = omu + kIn, kNParams = os + kIn, kNTrained = omu;

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------ GEMM
// C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn].
struct GemmArgs {
    const bf16 *A;
    long long sam, sak;
    const bf16 *B;
    long long sbk, sbn;
    int M, N, K;
    const float *bias;     // [N] or nullptr
    float *out;            // FP32 result (z for GELU layers) [M][ldo] or nullptr
    long long ldo;
    bf16 *out_bf;          // bfloat16 of GELU(result) (gelu) or of the result, [M][ldb] or nullptr
    long long ldb;
    int gelu;
};

// Tile of one block: kGM x kGN outputs, K in chunks of kGK, two chunk buffers.
constexpr int kGM = 128, kGN = 64, kGK = 32;
constexpr long kWaitLimit = 1L << 24;       // mbarrier polls before a GEMM gives up (sets *err)

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// Shared-memory matrix descriptor of tcgen05.mma for a K-major operand in the
// no-swizzle core-matrix layout: core matrices of 8 rows x 16 bytes, those
// adjacent along K `lbo` bytes apart, those adjacent along M/N `sbo` bytes
// apart (descriptor version 1, layout type 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Byte offset of element (r, k) of a rows x kGK chunk in that layout
// (lbo = 128: the two 8-wide K halves of a 16-wide step are adjacent;
// sbo = kGK / 8 * 128: one 8-row group holds all of the chunk's K).
__device__ __forceinline__ uint32_t core_off(int r, int k) {
    return (uint32_t)((r >> 3) * (kGK / 8 * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (long it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
                     : "=r"(ok) : "r"(addr), "r"(parity));
        if (ok) return true;
    }
    return false;
}

// C = A B on the 5th-generation tensor cores: bfloat16 operands staged into
// shared memory (any strides, zero-filled past M, N, K), tcgen05.mma with the
// 128 x 64 FP32 accumulator in tensor memory (one elected thread issues the
// MMAs and commits them to a chunk buffer's mbarrier), tcgen05.ld into
// registers for the epilogue (bias, GELU, FP32 and bfloat16 stores).  Block
// = 4 warps; warp w owns accumulator rows 32w..32w+31.  A chunk buffer is
// restaged only after the MMAs that read it have completed.
__global__ void __launch_bounds__(128) gemm_tc_kernel(const GemmArgs g, int *err) {
    __shared__ __align__(128) bf16 sA[2][kGM * kGK];
    __shared__ __align__(128) bf16 sB[2][kGN * kGK];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    const uint32_t mb1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "r"(kGN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // kind::f16 instruction descriptor: D FP32, A and B bfloat16, both K-major, N = kGN, M = kGM
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGN >> 3) << 17) |
                           ((uint32_t)(kGM >> 4) << 24);
    const bf16 zero = __float2bfloat16(0.f);
    const int nk = (g.K + kGK - 1) / kGK;
    bool ok = true;
    for (int c = 0; c < nk && ok; ++c) {
        const int b = c & 1;
        if (c >= 2) ok = mbar_wait(b ? mb1 : mb0, (uint32_t)((c - 2) >> 1) & 1u);   // MMAs of chunk c-2 done
        if (!ok) break;
        const int k0 = c * kGK;
        char *ab = reinterpret_cast<char *>(sA[b]);
        char *bb = reinterpret_cast<char *>(sB[b]);
        for (int e = tid; e < kGM * kGK; e += blockDim.x) {
            const int mm = e / kGK, kk = e % kGK;
            const int m = m0 + mm, k = k0 + kk;
            *reinterpret_cast<bf16 *>(ab + core_off(mm, kk)) =
                (m < g.M && k < g.K) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : zero;
        }
        for (int e = tid; e < kGN * kGK; e += blockDim.x) {
            const int nn = e / kGK, kk = e % kGK;
            const int n = n0 + nn, k = k0 + kk;
            *reinterpret_cast<bf16 *>(bb + core_off(nn, kk)) =
                (n < g.N && k < g.K) ? g.B[(long long)k * g.sbk + (long long)n * g.sbn] : zero;
        }
        asm volatile("fence.proxy.async.shared::cta;");      // the stores above, visible to the tensor core
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sA[b]);
            const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(sB[b]);
#pragma unroll
            for (int kk = 0; kk < kGK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + 256u * kk, 128u, kGK / 8 * 128);
                const uint64_t bd = smem_desc(b0 + 256u * kk, 128u, kGK / 8 * 128);
                const uint32_t accum = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(b ? mb1 : mb0));
        }
    }
    // the last commit completes after every earlier MMA of this thread
    if (ok && nk > 0) ok = mbar_wait(((nk - 1) & 1) ? mb1 : mb0, (uint32_t)((nk - 1) >> 1) & 1u);
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // MMAs may still be in flight: wait once more (bounded) before freeing TMEM
        if (nk > 0) mbar_wait(((nk - 1) & 1) ? mb1 : mb0, (uint32_t)((nk - 1) >> 1) & 1u);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int m = m0 + 32 * warp + lane;              // accumulator lane = output row
#pragma unroll
        for (int c0 = 0; c0 < kGN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (m < g.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n >= g.N) break;
                    float v = __uint_as_float(r[j]);
                    if (g.bias) v += g.bias[n];
                    if (g.out) g.out[(long long)m * g.ldo + n] = v;
                    if (g.out_bf) g.out_bf[(long long)m * g.ldb + n] = __float2bfloat16(g.gelu ? gelu_f(v) : v);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kGN));
}

// ------------------------------------------------------------------ small kernels
__global__ void standardise_kernel(const float *x, const float *mu, const float *s, int B, bf16 *a0) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * kIn; e += gridDim.x * blockDim.x) {
        const int i = e % kIn;
        a0[e] = __float2bfloat16((x[e] - mu[i]) / s[i]);
    }
}

// dy = 2 (y - t) / B (FP32 and bfloat16) and the loss, one block, fixed order.
__global__ void loss_kernel(const float *y, const float *t, int B, float *dy, bf16 *dy_bf, double *loss) {
    __shared__ double s_l[256];
    double l = 0.0;
    for (int e = threadIdx.x; e < B * kOut; e += blockDim.x) {
        const float d = y[e] - t[e];
        l += (double)d * d;
        const float g = 2.0f * d / (float)B;
        dy[e] = g;
        dy_bf[e] = __float2bfloat16(g);
    }
    s_l[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_l[threadIdx.x] += s_l[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s_l[0] / B;
}

__global__ void gelu_back_kernel(const float *da, const float *z, int n, float *dz, bf16 *dz_bf) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float v = da[e] * gelu_grad_f(z[e]);
        dz[e] = v;
        dz_bf[e] = __float2bfloat16(v);
    }
}

// db[n] = sum_m dz[m][n], one warp per column, fixed order.
__global__ void colsum_kernel(const float *dz, int M, int N, float *db) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (col >= N) return;
    float s = 0.f;
    for (int m = lane; m < M; m += 32) s += dz[(size_t)m * N + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[col] = s;
}

// AdamW (decoupled weight decay) on the trained parameters; c1, c2 are the
// bias corrections 1 - beta^step.
__global__ void adamw_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                             float eps, float wd, float c1, float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.f - b1) * ge;
        const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        const float mh = me / c1, vh = ve / c2;
        const float pe = p[e] - lr * (mh / (sqrtf(vh) + eps) + wd * p[e]);
        p[e] = pe;
    }
}

__global__ void to_bf16_kernel(const float *src, int n, bf16 *dst) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16(src[e]);
}

int blocks_for(size_t n, int threads = 256) {
    size_t b = (n + threads - 1) / threads;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace psc

using namespace psc;

struct psc_mlp {
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // [kNParams]
    bf16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *w4 = nullptr;
    bf16 *a0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr; // activations (bfloat16)
    float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *y = nullptr;
    float *dy = nullptr, *da = nullptr, *dz = nullptr;
    bf16 *dy_bf = nullptr, *dz_bf = nullptr;
    double *d_loss = nullptr;
    int *d_err = nullptr;        // set by a GEMM whose tensor-core wait ran out
    long long step = 0;
    std::vector<float> host;
    std::string err;
};

namespace {

psc_status mfail(psc_mlp *m, psc_status st, const std::string &msg) {
    if (m) m->err = msg;
    return set_global_error(st, msg.c_str());
}

#define PSC_MCUDA(mm, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return mfail((mm), e_ == cudaErrorMemoryAllocation ? PSC_ERR_OOM : PSC_ERR_CUDA,     \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

template <class T>
cudaError_t mall(T **p, size_t n) { return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)); }

// After a synchronisation: PSC_ERR_TIMEOUT (and the flag cleared) if a GEMM
// gave up waiting for its tensor-core work since the last check.
psc_status check_device_err(psc_mlp *m) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mfail(m, PSC_ERR_CUDA, std::string("device error flag: ") + cudaGetErrorString(e));
    if (h == 0) return PSC_OK;
    cudaMemset(m->d_err, 0, sizeof(int));
    return mfail(m, PSC_ERR_TIMEOUT, "a tensor-core GEMM timed out waiting for its MMAs");
}

void mfree(psc_mlp *m) {
    if (!m) return;
    void *ptrs[] = {m->p, m->g, m->m, m->v, m->w1, m->w2, m->w3, m->w4, m->a0, m->a1, m->a2, m->a3, m->z1, m->z2,
                    m->z3, m->y, m->dy, m->da, m->dz, m->dy_bf, m->dz_bf, m->d_loss, m->d_err};
    for (void *q : ptrs) cudaFree(q);
    delete m;
}

// Each block holds kGN TMEM columns; 4 KB of unused dynamic shared memory
// keeps a block at >= 28 KB, so at most 7 blocks (448 of the 512 columns)
// are resident on an SM and a TMEM allocation never has to wait.
constexpr size_t kTmemGuardSmem = 4096;

cudaError_t gemm(const GemmArgs &a, int *err, cudaStream_t s) {
    dim3 grid((a.N + kGN - 1) / kGN, (a.M + kGM - 1) / kGM);
    gemm_tc_kernel<<<grid, 128, kTmemGuardSmem, s>>>(a, err);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(psc_mlp *m) {
    cudaStream_t s = m->stream;
    to_bf16_kernel<<<blocks_for(kIn * kHid), 256, 0, s>>>(m->p + oW1, kIn * kHid, m->w1);
    to_bf16_kernel<<<blocks_for(kHid * kHid), 256, 0, s>>>(m->p + oW2, kHid * kHid, m->w2);
    to_bf16_kernel<<<blocks_for(kHid * kHid), 256, 0, s>>>(m->p + oW3, kHid * kHid, m->w3);
    to_bf16_kernel<<<blocks_for(kHid * kOut), 256, 0, s>>>(m->p + oW4, kHid * kOut, m->w4);
    return cudaGetLastError();
}

GemmArgs fwd_layer(const bf16 *A, int B, int K, const bf16 *W, int N, const float *bias, float *z, bf16 *abf, int gelu) {
    GemmArgs a{};
    a.A = A; a.sam = K; a.sak = 1;
    a.B = W; a.sbk = N; a.sbn = 1;
    a.M = B; a.N = N; a.K = K;
    a.bias = bias;
    a.out = z; a.ldo = N;
    a.out_bf = abf; a.ldb = N;
    a.gelu = gelu;
    return a;
}

psc_status forward(psc_mlp *m, const float *x, int B) {
    cudaStream_t s = m->stream;
    standardise_kernel<<<blocks_for((size_t)B * kIn), 256, 0, s>>>(x, m->p + omu, m->p + os, B, m->a0);
    PSC_MCUDA(m, cudaGetLastError());
    PSC_MCUDA(m, gemm(fwd_layer(m->a0, B, kIn, m->w1, kHid, m->p + ob1, m->z1, m->a1, 1), m->d_err, s));
    PSC_MCUDA(m, gemm(fwd_layer(m->a1, B, kHid, m->w2, kHid, m->p + ob2, m->z2, m->a2, 1), m->d_err, s));
    PSC_MCUDA(m, gemm(fwd_layer(m->a2, B, kHid, m->w3, kHid, m->p + ob3, m->z3, m->a3, 1), m->d_err, s));
    PSC_MCUDA(m, gemm(fwd_layer(m->a3, B, kHid, m->w4, kOut, m->p + ob4, m->y, nullptr, 0), m->d_err, s));
    return PSC_OK;
}

// dW[K][N] = X^T dZ  with X [B][K] (bfloat16) and dZ [B][N] (bfloat16)
GemmArgs wgrad(const bf16 *X, int B, int K, const bf16 *dZ, int N, float *dW) {
    GemmArgs a{};
    a.A = X; a.sam = 1; a.sak = K;        // A(m = k_in, k = b) = X[b][k_in]
    a.B = dZ; a.sbk = N; a.sbn = 1;       // B(k = b, n) = dZ[b][n]
    a.M = K; a.N = N; a.K = B;
    a.out = dW; a.ldo = N;
    return a;
}

// dX[B][K] = dZ W^T with dZ [B][N] and W [K][N] (both bfloat16)
GemmArgs dgrad(const bf16 *dZ, int B, int N, const bf16 *W, int K, float *dX) {
    GemmArgs a{};
    a.A = dZ; a.sam = N; a.sak = 1;       // A(m = b, k = n) = dZ[b][n]
    a.B = W; a.sbk = 1; a.sbn = N;        // B(k = n, n' = k_in) = W[k_in][n]
    a.M = B; a.N = K; a.K = N;
    a.out = dX; a.ldo = K;
    return a;
}

psc_status backward(psc_mlp *m, const float *t, int B) {
    cudaStream_t s = m->stream;
    loss_kernel<<<1, 256, 0, s>>>(m->y, t, B, m->dy, m->dy_bf, m->d_loss);
    PSC_MCUDA(m, cudaGetLastError());
    float *g = m->g;
    PSC_MCUDA(m, cudaMemsetAsync(g, 0, sizeof(float) * kNParams, s));
    PSC_MCUDA(m, gemm(wgrad(m->a3, B, kHid, m->dy_bf, kOut, g + oW4), m->d_err, s));
    colsum_kernel<<<1, 32 * kOut, 0, s>>>(m->dy, B, kOut, g + ob4);
    PSC_MCUDA(m, gemm(dgrad(m->dy_bf, B, kOut, m->w4, kHid, m->da), m->d_err, s));
    const float *zs[3] = {m->z1, m->z2, m->z3};
    const bf16 *as[3] = {m->a0, m->a1, m->a2};
    const bf16 *ws[3] = {m->w1, m->w2, m->w3};
    const size_t ow[3] = {oW1, oW2, oW3}, ob[3] = {ob1, ob2, ob3};
    const int kin[3] = {kIn, kHid, kHid};
    for (int L = 2; L >= 0; --L) {
        gelu_back_kernel<<<blocks_for((size_t)B * kHid), 256, 0, s>>>(m->da, zs[L], B * kHid, m->dz, m->dz_bf);
        PSC_MCUDA(m, cudaGetLastError());
        PSC_MCUDA(m, gemm(wgrad(as[L], B, kin[L], m->dz_bf, kHid, g + ow[L]), m->d_err, s));
        colsum_kernel<<<(kHid * 32 + 255) / 256, 256, 0, s>>>(m->dz, B, kHid, g + ob[L]);
        PSC_MCUDA(m, cudaGetLastError());
        if (L > 0) PSC_MCUDA(m, gemm(dgrad(m->dz_bf, B, kHid, ws[L], kin[L], m->da), m->d_err, s));
    }
    return PSC_OK;
}

psc_status check_batch(psc_mlp *m, const void *x, int B) {
    if (!m) return set_global_error(PSC_ERR_ARG, "mlp is NULL");
    if (!x) return mfail(m, PSC_ERR_ARG, "input is NULL");
    if (B < 1 || B > m->max_batch) return mfail(m, PSC_ERR_ARG, "batch must be in [1, max_batch]");
    return PSC_OK;
}

}  // namespace

extern "C" {

int psc_mlp_n_params(void) { return (int)kNParams; }

psc_status psc_mlp_create(psc_mlp **out, int max_batch, void *stream) {
    if (!out) return set_global_error(PSC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 24)) return set_global_error(PSC_ERR_ARG, "max_batch must be in [1, 2^24]");
    psc_mlp *m = new psc_mlp();
    m->stream = (cudaStream_t)stream;
    m->max_batch = max_batch;
    const size_t B = max_batch;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = mall(&m->p, kNParams);
    if (e == cudaSuccess) e = mall(&m->g, kNParams);
    if (e == cudaSuccess) e = mall(&m->m, kNParams);
    if (e == cudaSuccess) e = mall(&m->v, kNParams);
    if (e == cudaSuccess) e = mall(&m->w1, (size_t)kIn * kHid);
    if (e == cudaSuccess) e = mall(&m->w2, (size_t)kHid * kHid);
    if (e == cudaSuccess) e = mall(&m->w3, (size_t)kHid * kHid);
    if (e == cudaSuccess) e = mall(&m->w4, (size_t)kHid * kOut);
    if (e == cudaSuccess) e = mall(&m->a0, B * kIn);
    if (e == cudaSuccess) e = mall(&m->a1, B * kHid);
    if (e == cudaSuccess) e = mall(&m->a2, B * kHid);
    if (e == cudaSuccess) e = mall(&m->a3, B * kHid);
    if (e == cudaSuccess) e = mall(&m->z1, B * kHid);
    if (e == cudaSuccess) e = mall(&m->z2, B * kHid);
    if (e == cudaSuccess) e = mall(&m->z3, B * kHid);
    if (e == cudaSuccess) e = mall(&m->y, B * kOut);
    if (e == cudaSuccess) e = mall(&m->dy, B * kOut);
    if (e == cudaSuccess) e = mall(&m->da, B * kHid);
    if (e == cudaSuccess) e = mall(&m->dz, B * kHid);
    if (e == cudaSuccess) e = mall(&m->dy_bf, B * kOut);
    if (e == cudaSuccess) e = mall(&m->dz_bf, B * kHid);
    if (e == cudaSuccess) e = mall(&m->d_loss, 1);
    if (e == cudaSuccess) e = mall(&m->d_err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream);
    if (e != cudaSuccess) {
        mfree(m);
        return set_global_error(e == cudaErrorMemoryAllocation ? PSC_ERR_OOM : PSC_ERR_CUDA, "psc_mlp_create: allocation");
    }
    *out = m;
    return PSC_OK;
}

void psc_mlp_destroy(psc_mlp *m) { mfree(m); }

psc_status psc_mlp_set_params(psc_mlp *m, const float *params) {
    if (!m || !params) return set_global_error(PSC_ERR_ARG, "mlp and params must be non-NULL");
    for (int i = 0; i < kIn; ++i)
        if (!(params[os + i] > 0.f)) return mfail(m, PSC_ERR_ARG, "input scales s must be > 0");
    PSC_MCUDA(m, cudaMemcpyAsync(m->p, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, m->stream));
    PSC_MCUDA(m, cudaMemsetAsync(m->m, 0, sizeof(float) * kNParams, m->stream));
    PSC_MCUDA(m, cudaMemsetAsync(m->v, 0, sizeof(float) * kNParams, m->stream));
    PSC_MCUDA(m, refresh_bf16(m));
    PSC_MCUDA(m, cudaStreamSynchronize(m->stream));
    m->step = 0;
    return PSC_OK;
}

psc_status psc_mlp_get_params(psc_mlp *m, float *params) {
    if (!m || !params) return set_global_error(PSC_ERR_ARG, "mlp and params must be non-NULL");
    PSC_MCUDA(m, cudaMemcpyAsync(params, m->p, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, m->stream));
    PSC_MCUDA(m, cudaStreamSynchronize(m->stream));
    return check_device_err(m);
}

psc_status psc_mlp_forward(psc_mlp *m, const float *x_dev, int batch, float *y_dev) {
    psc_status st = check_batch(m, x_dev, batch);
    if (st != PSC_OK) return st;
    if (!y_dev) return mfail(m, PSC_ERR_ARG, "output is NULL");
    st = forward(m, x_dev, batch);
    if (st != PSC_OK) return st;
    PSC_MCUDA(m, cudaMemcpyAsync(y_dev, m->y, sizeof(float) * batch * kOut, cudaMemcpyDeviceToDevice, m->stream));
    return PSC_OK;
}

psc_status psc_mlp_grad(psc_mlp *m, const float *x_dev, const float *t_dev, int batch, float *grad_host, double *loss) {
    psc_status st = check_batch(m, x_dev, batch);
    if (st != PSC_OK) return st;
    if (!t_dev) return mfail(m, PSC_ERR_ARG, "targets are NULL");
    st = forward(m, x_dev, batch);
    if (st == PSC_OK) st = backward(m, t_dev, batch);
    if (st != PSC_OK) return st;
    if (grad_host) PSC_MCUDA(m, cudaMemcpyAsync(grad_host, m->g, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, m->stream));
    if (loss) PSC_MCUDA(m, cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (grad_host || loss) {
        PSC_MCUDA(m, cudaStreamSynchronize(m->stream));
        return check_device_err(m);
    }
    return PSC_OK;
}

psc_status psc_mlp_train_step(psc_mlp *m, const float *x_dev, const float *t_dev, int batch, double lr, double *loss) {
    psc_status st = check_batch(m, x_dev, batch);
    if (st != PSC_OK) return st;
    if (!t_dev) return mfail(m, PSC_ERR_ARG, "targets are NULL");
    if (!(lr > 0.0) || !std::isfinite(lr)) return mfail(m, PSC_ERR_ARG, "lr must be > 0");
    st = forward(m, x_dev, batch);
    if (st == PSC_OK) st = backward(m, t_dev, batch);
    if (st != PSC_OK) return st;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)m->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)m->step));
    adamw_kernel<<<blocks_for(kNTrained), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, (int)kNTrained, (float)lr, b1, b2,
                                                               1e-8f, 1e-4f, c1, c2);
    PSC_MCUDA(m, cudaGetLastError());
    PSC_MCUDA(m, refresh_bf16(m));
    if (loss) {
        PSC_MCUDA(m, cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        PSC_MCUDA(m, cudaStreamSynchronize(m->stream));
        return check_device_err(m);
    }
    return PSC_OK;
}

psc_status psc_mlp_infer_offsets(psc_mlp *m, const float *feat_dev, int n_ant, double sigma_prior_rad, double *lm_out) {
    psc_status st = check_batch(m, feat_dev, n_ant);
    if (st != PSC_OK) return st;
    if (!lm_out) return mfail(m, PSC_ERR_ARG, "lm_out is NULL");
    st = forward(m, feat_dev, n_ant);
    if (st != PSC_OK) return st;
    if (m->host.size() < (size_t)n_ant * kOut) m->host.resize((size_t)n_ant * kOut);
    PSC_MCUDA(m, cudaMemcpyAsync(m->host.data(), m->y, sizeof(float) * n_ant * kOut, cudaMemcpyDeviceToHost, m->stream));
    PSC_MCUDA(m, cudaStreamSynchronize(m->stream));
    st = check_device_err(m);
    if (st != PSC_OK) return st;
    for (int i = 0; i < n_ant * kOut; ++i) lm_out[i] = (double)m->host[i] * sigma_prior_rad;
    return PSC_OK;
}

}  // extern "C"

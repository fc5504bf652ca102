// Model grid V° = F[I^M] (Algorithm 1, first pre-compute; Eq. MEDD):
// the unnormalised DFT, sign exp(+2 pi i) as in Eq. ME, of the N x N image
// zero-padded to Ng x Ng,
//   G[gy][gx] = sum_{row,col} I[row][col] W((gx-Ng/2)(col-N/2)) W((gy-Ng/2)(row-N/2)),
//   W(k) = exp(2 pi i k / Ng),
// computed as two complex matrix products, T = I F^T (N x Ng) and G = F T,
// with F[g][c] = W((g - Ng/2)(c - N/2)) generated on the fly from a twiddle
// table (exact integer phase index modulo Ng, table values from FP64 sincospi).
// FP32 SIMT GEMM tiles: 64 x 64 outputs per 256-thread block, 4 x 4 per thread.
#include <algorithm>
#include <cstdint>

#include <cuda.h>
#include <cuda_bf16.h>

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


// ---------------------------------------------------------------------------
// Tensor-core path (N % 8 == 0): the same two products on the 5th-generation
// tensor cores in split bfloat16.  Every FP32 operand x is written as three
// bfloat16 planes x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x - h
// - m), each residual exact in FP32), and a product x y is accumulated in FP32
// from the six plane pairs (h,h) (h,m) (m,h) (m,m) (h,l) (l,h); the dropped
// pairs are below 2^-24 of |x y|, FP32's own rounding.
//   pass 1: T[r][g] = sum_c I[r][c] E[g][c]       (tile rows r, columns g)
//   pass 2: G[gy][gx]^T tile: rows gx, columns gy, sum over r of T[r][gx] E[gy][r]
// with E[g][c] = W((g - Ng/2)(c - N/2)).  Pass 1 writes T already split and
// transposed (planes [3][Ng][N]) so that both passes read K-major operands.
// A block owns a 128 x 64 tile with FP32 accumulators in tensor memory; K
// advances in chunks of 32 through shared-memory buffers of all operand
// planes.  One thread runs the pipeline over three shared-memory buffers: it
// loads chunks two ahead with TMA (cp.async.bulk.tensor, one copy per source
// and 8-wide K column: the box 8 x rows x 3 planes lands as [plane][row][8
// elements], i.e. the no-swizzle K-major core-matrix layout, K columns
// 3 * rows * 16 bytes apart), waits for a chunk's copies on its buffer's load
// mbarrier, issues the MMAs (kind::f16, the negative term of the complex
// product by the descriptor's negate-A bit), commits them to the buffer's MMA
// mbarrier, and refills the previous chunk's buffer once those MMAs are done.
// Rows past the operands' edges read TMA's zero fill; the depth K is padded
// with zeros to a multiple of the chunk.  Every wait is bounded (*err).

typedef __nv_bfloat16 bf16;
constexpr int kTM = 128, kTN = 64, kTK = 32;
constexpr int kColA = 3 * kTM * 16;                 // one 8-wide K column of an A source, 3 planes (6 KB)
constexpr int kColB = 3 * kTN * 16;                 // the same of a B source (3 KB)
constexpr int kSrcA = kTK / 8 * kColA;              // an A source's share of a chunk (24 KB)
constexpr int kSrcB = kTK / 8 * kColB;              // a B source's share (12 KB)
constexpr int kEpoch = 4;                            // chunks (K = 128) between promotions to registers
constexpr int kStages = 3;                           // shared-memory buffers of the TMA pipeline
constexpr long kTcWait = 1L << 24;

__device__ __forceinline__ void split3(float x, bf16 &h, bf16 &m, bf16 &l) {
    h = __float2bfloat16_rn(x);
    const float r = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r);
    l = __float2bfloat16_rn(r - __bfloat162float(m));
}

// The same split of an FP64 value (the twiddles), residuals in FP64.
__device__ __forceinline__ void split3d(double x, bf16 &h, bf16 &m, bf16 &l) {
    h = __double2bfloat16(x);
    const double r = x - (double)__bfloat162float(h);
    m = __double2bfloat16(r);
    l = __double2bfloat16(r - (double)__bfloat162float(m));
}

__global__ void twiddle64_kernel(double2 *W, int ng) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)ng, &s, &c);
        W[k] = make_double2(c, s);
    }
}

// I3[p][r][c] of the N x N image, each row padded with zeros to kp columns
// (the GEMM depth, a multiple of the K chunk, so that no chunk is ragged).
__global__ void split_image_kernel(const float *__restrict__ img, int n, int kp, bf16 *__restrict__ I3) {
    const long long total = (long long)n * kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / kp), c = (int)(e % kp);
        bf16 h, m, l;
        split3(c < n ? img[(size_t)r * n + c] : 0.f, h, m, l);
        I3[e] = h; I3[total + e] = m; I3[2 * total + e] = l;
    }
}

// E3re[p][g][c], E3im[p][g][c] (g < Ng, c < kp; zero for c >= N).
__global__ void split_dft_matrix_kernel(const double2 *__restrict__ W, int n, int ng, int kp, bf16 *__restrict__ Er,
                                        bf16 *__restrict__ Ei) {
    const long long total = (long long)ng * kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(e / kp), c = (int)(e % kp);
        const double2 w = c < n ? W[phase_index(g, c, ng, n)] : make_double2(0.0, 0.0);
        bf16 h, m, l;
        split3d(w.x, h, m, l);
        Er[e] = h; Er[total + e] = m; Er[2 * total + e] = l;
        split3d(w.y, h, m, l);
        Ei[e] = h; Ei[total + e] = m; Ei[2 * total + e] = l;
    }
}

// Component operands of the grid G[gy][gx] = sum_k S_k exp(2 pi i (u_gx l_k + v_gy m_k)),
// u_g = v_g = (g - Ng/2) du, as the second tensor-core pass with
// A[gx][k] = S_k exp(2 pi i u_gx l_k) and B[gy][k] = exp(2 pi i v_gy m_k): split planes
// [3][Ng][kp] of the real and imaginary parts, phases from FP64 sincospi,
// columns k >= n_comp zero (kp = n_comp rounded up to a multiple of the K chunk).
__global__ void split_comp_kernel(const double *__restrict__ comp, int n_comp, int stride, double wp, int kp, int ng,
                                  double du, bf16 *__restrict__ Ar, bf16 *__restrict__ Ai, bf16 *__restrict__ Br,
                                  bf16 *__restrict__ Bi) {
    const long long total = (long long)ng * kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(e / kp), k = (int)(e % kp);
        double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
        if (k < n_comp) {
            const double x = (double)(g - ng / 2) * du;
            const double *ck = comp + (size_t)stride * k;
            // flux phase of a w-plane: 2 pi wp (n - 1), folded into the u factor
            const double wph = stride == 4 ? wp * ck[3] : 0.0;
            double sn, cs;
            sincospi(2.0 * (x * ck[0] + wph), &sn, &cs);
            ar = ck[2] * cs;
            ai = ck[2] * sn;
            sincospi(2.0 * x * ck[1], &sn, &cs);
            br = cs;
            bi = sn;
        }
        bf16 h, m, l;
        split3d(ar, h, m, l); Ar[e] = h; Ar[total + e] = m; Ar[2 * total + e] = l;
        split3d(ai, h, m, l); Ai[e] = h; Ai[total + e] = m; Ai[2 * total + e] = l;
        split3d(br, h, m, l); Br[e] = h; Br[total + e] = m; Br[2 * total + e] = l;
        split3d(bi, h, m, l); Bi[e] = h; Bi[total + e] = m; Bi[2 * total + e] = l;
    }
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t k_stride) {
    // K-major, no swizzle: K-adjacent core matrices k_stride bytes apart, 8-row groups 128 B apart
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((k_stride >> 4) & 0x3FFF) << 16) |
           ((uint64_t)(128 >> 4) << 32) | ((uint64_t)1 << 46);
}

// TMA load of one box of a 3-D tensor map into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t mbar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t addr, uint32_t parity) {
    for (long it = 0; it < kTcWait; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
                     : "=r"(ok) : "r"(addr), "r"(parity));
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

struct TcPassArgs {
    const bf16 *A[2];       // split planes [3][a_rows][k] of each A source (pass 1: image; pass 2: T re, T im)
    const bf16 *B[2];       // split planes [3][b_rows][k] of each B source (E re, E im)
    int n_a;                // A sources: 1 (pass 1) or 2 (pass 2)
    int a_rows, b_rows, k;  // rows of the A and B operands, depth (= N, also the plane pitch)
    bf16 *Tr, *Ti;          // pass 1 output planes [3][Ng][N]
    float2 *G;              // pass 2 output [Ng][Ng]
    int ng;
    int *err;
};

template <int kPass>
__global__ void __launch_bounds__(128, 1) dft_tc_kernel(const TcPassArgs g, const __grid_constant__ CUtensorMap mA0,
                                                        const __grid_constant__ CUtensorMap mA1,
                                                        const __grid_constant__ CUtensorMap mB0,
                                                        const __grid_constant__ CUtensorMap mB1) {
    constexpr int kNA = kPass == 1 ? 1 : 2;
    constexpr int kStage = kNA * kSrcA + 2 * kSrcB;           // A sources, then B sources (E re, E im)
    constexpr uint32_t kBytes = (uint32_t)kStage;              // TMA bytes of one chunk (zero fill included)
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kStages];            // MMAs of the buffer's chunk done
    __shared__ __align__(8) uint64_t lbar[kStages];            // TMA copies of the buffer's chunk done
    __shared__ __align__(8) uint64_t pbar;                     // MMAs up to an epoch's last chunk done
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    uint32_t mb[kStages], lb[kStages];
    for (int i = 0; i < kStages; ++i) {
        mb[i] = (uint32_t)__cvta_generic_to_shared(&mbar[i]);
        lb[i] = (uint32_t)__cvta_generic_to_shared(&lbar[i]);
    }
    const uint32_t pb = (uint32_t)__cvta_generic_to_shared(&pbar);
    const CUtensorMap *mapA[2] = {&mA0, &mA1};
    const CUtensorMap *mapB[2] = {&mB0, &mB1};
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb[i]));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(lb[i]));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(pb));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "r"(4 * kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // accumulators of kTN columns: 0 real, 1 imaginary (head x head plane
    // products), 2 real, 3 imaginary (the smaller cross-plane products, kept
    // apart so that the tensor core's accumulation does not round them away
    // against the head terms).  Every kEpoch chunks all four are added into
    // FP32 registers (round to nearest) and restarted, which bounds the depth
    // of any tensor-core sum at kEpoch * kTK = 128.
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                           ((uint32_t)(kTM >> 4) << 24);
    const uint32_t idesc_neg = idesc | (1u << 13);  // negate A
    const int nk = (g.k + kTK - 1) / kTK;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    float sum_re[kTN], sum_im[kTN];
#pragma unroll
    for (int j = 0; j < kTN; ++j) { sum_re[j] = 0.f; sum_im[j] = 0.f; }
    bool ok = true;
    bool started[4] = {false, false, false, false};  // used by thread 0 only
    // Only thread 0 waits on the buffers' barriers (in chunk order, so never
    // two phases behind); the other threads wait on pbar, one phase per epoch,
    // committed after the epoch's last chunk and waited by every thread before
    // the block barrier of the promotion.  Thread 0 keeps the copies kStages - 1
    // chunks ahead: it issues a chunk's MMAs as soon as its copies have landed,
    // then refills the buffer of the previous chunk once that chunk's MMAs are done.
    int loads = 0;                                    // thread 0: chunks whose copies were issued
    int mmas = 0;                                     // thread 0: chunks whose MMAs were issued
    int epoch = 0;                                    // promotions done
    auto issue_copies = [&](int ch) {
        const int bb = ch % kStages;
        const uint32_t sb = smem_base + (uint32_t)(bb * kStage);
        mbar_expect(lb[bb], kBytes);
        const int k0 = ch * kTK;
        for (int j = 0; j < kTK / 8; ++j) {
            for (int s_ = 0; s_ < kNA; ++s_)
                tma_load3(sb + (uint32_t)(s_ * kSrcA + j * kColA), mapA[s_], k0 + 8 * j, m0, 0, lb[bb]);
            for (int s_ = 0; s_ < 2; ++s_)
                tma_load3(sb + (uint32_t)(kNA * kSrcA + s_ * kSrcB + j * kColB), mapB[s_], k0 + 8 * j, n0, 0, lb[bb]);
        }
        loads = ch + 1;
    };
    if (tid == 0)
        for (int ch = 0; ch < kStages - 1 && ch < nk; ++ch) issue_copies(ch);
    for (int c = 0; c < nk && ok; ++c) {
        const int b = c % kStages;
        const bool promote = (c + 1) % kEpoch == 0 || c == nk - 1;
        if (tid == 0) {
            ok = tc_wait(lb[b], (uint32_t)(c / kStages) & 1u);          // this chunk's copies
            const uint32_t sb = smem_base + (uint32_t)(b * kStage);
            if (ok) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                // plane pairs (A split, B split) kept in each product; pair 0 is head x head
                const int pp[6][2] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}, {0, 2}, {2, 0}};
                // terms (accumulator, A source, B source, negate):
                // pass 1: re += I Er, im += I Ei; pass 2: re += Tr Er - Ti Ei, im += Ti Er + Tr Ei
                constexpr int kTerms = kPass == 1 ? 2 : 4;
                const int terms[4][4] = {{0, 0, 0, 0},
                                         {kPass == 1 ? 1 : 0, kPass == 1 ? 0 : 1, 1, kPass == 1 ? 0 : 1},
                                         {1, 1, 0, 0},
                                         {1, 0, 1, 0}};
                for (int t = 0; t < kTerms; ++t) {
                    const int acc = terms[t][0], sa = terms[t][1], sbs = terms[t][2], neg = terms[t][3];
                    for (int q = 0; q < 6; ++q) {
                        // plane p of source s: K column j at + j * kCol, plane p at + p * rows * 16
                        const uint32_t a_pl = sb + (uint32_t)(sa * kSrcA + pp[q][0] * kTM * 16);
                        const uint32_t b_pl = sb + (uint32_t)(kNA * kSrcA + sbs * kSrcB + pp[q][1] * kTN * 16);
                        const int dst = acc + (q == 0 ? 0 : 2);
#pragma unroll
                        for (int kk = 0; kk < kTK / 16; ++kk) {
                            tc_mma(tmem + (uint32_t)(dst * kTN), tc_desc(a_pl + (uint32_t)(2 * kk * kColA), kColA),
                                   tc_desc(b_pl + (uint32_t)(2 * kk * kColB), kColB), neg ? idesc_neg : idesc,
                                   started[dst] ? 1u : 0u);
                            started[dst] = true;
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mb[b]));
                if (promote)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(pb));
                mmas = c + 1;
            }
            // refill: chunk c + kStages - 1 goes into the buffer of chunk c - 1
            const int nx = c + kStages - 1;
            if (ok && nx < nk) {
                if (c >= 1) ok = tc_wait(mb[(c - 1) % kStages], (uint32_t)((c - 1) / kStages) & 1u);
                if (ok) issue_copies(nx);
            }
            if (!ok) break;
        }
        if (promote) {
            // promote: wait for this chunk's MMAs (and with them all earlier ones),
            // add the four accumulators into the FP32 sums, restart them
            ok = tc_wait(pb, (uint32_t)epoch & 1u);
            ++epoch;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int c0 = 0; c0 < kTN; c0 += 16) {
                uint32_t re[16], im[16], rs[16], is[16];
                tc_ld16(lane_base + (uint32_t)c0, re);
                tc_ld16(lane_base + (uint32_t)(kTN + c0), im);
                tc_ld16(lane_base + (uint32_t)(2 * kTN + c0), rs);
                tc_ld16(lane_base + (uint32_t)(3 * kTN + c0), is);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    sum_re[c0 + j] += __uint_as_float(re[j]) + __uint_as_float(rs[j]);
                    sum_im[c0 + j] += __uint_as_float(im[j]) + __uint_as_float(is[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();                               // every warp has read before the accumulators restart
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) started[0] = started[1] = started[2] = started[3] = false;
        }
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(g.err, 1);
            // copies and MMAs still in flight, bounded: the last issued chunk's copies and
            // the MMAs of the chunks before it
            for (int c = mmas; c < loads; ++c) tc_wait(lb[c % kStages], (uint32_t)(c / kStages) & 1u);
            for (int c = std::max(0, mmas - kStages); c < mmas; ++c)
                tc_wait(mb[c % kStages], (uint32_t)(c / kStages) & 1u);
        }
    }
    if (ok) {
        const int m = m0 + 32 * warp + lane;         // accumulator lane: pass 1 image row, pass 2 grid column gx
        if (m < g.a_rows) {
#pragma unroll
            for (int j = 0; j < kTN; ++j) {
                const int col = n0 + j;                      // pass 1: grid column g; pass 2: grid row gy
                if (col >= g.b_rows) break;
                if constexpr (kPass == 1) {
                    const size_t plane_t = (size_t)g.b_rows * g.k;
                    const size_t o = (size_t)col * g.k + m;  // T planes [3][Ng][N]: row g, column image row m
                    bf16 h, mm, l;
                    split3(sum_re[j], h, mm, l);
                    g.Tr[o] = h; g.Tr[plane_t + o] = mm; g.Tr[2 * plane_t + o] = l;
                    split3(sum_im[j], h, mm, l);
                    g.Ti[o] = h; g.Ti[plane_t + o] = mm; g.Ti[2 * plane_t + o] = l;
                } else {
                    g.G[(size_t)col * g.ng + m] = make_float2(sum_re[j], sum_im[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(4 * kTN));
}
}  // namespace

namespace {
size_t al256(size_t x) { return (x + 255) / 256 * 256; }
bool use_tc(int n_img) { return n_img % 8 == 0; }
// GEMM depth: padded with zeros to a multiple of the K chunk (no ragged chunk;
// TMA boxes never start past an operand's end)
int kpad(int n) { return std::max(kTK, (n + kTK - 1) / kTK * kTK); }
int comp_depth(int n_comp) { return kpad(n_comp); }

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, through the runtime (no link against libcuda).
cudaError_t encode_fn(EncodeTiled *out) {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    *out = fn;
    return cudaSuccess;
}

// Tensor map of split bfloat16 planes [3][rows][k] (k % 8 == 0, 16-byte aligned
// base): dimensions (k, rows, 3), box 8 x box_rows x 3 (one 8-wide K column of a
// tile, all planes), zero fill outside.
cudaError_t plane_map(CUtensorMap *m, const bf16 *base, int rows, int k, int box_rows) {
    if (k % 8 || ((uintptr_t)base & 15)) return cudaErrorInvalidValue;
    EncodeTiled fn = nullptr;
    cudaError_t e = encode_fn(&fn);
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, 3};
    const cuuint64_t strides[2] = {(cuuint64_t)k * 2, (cuuint64_t)rows * (cuuint64_t)k * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, 3};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// One pass on the tensor cores: maps of the A sources (rows a_rows) and B
// sources (rows b_rows), then the launch.
template <int kPass>
cudaError_t launch_tc_pass(const TcPassArgs &a, cudaStream_t s) {
    constexpr int kNA = kPass == 1 ? 1 : 2;
    const int smem = kStages * (kNA * kSrcA + 2 * kSrcB);
    CUtensorMap mA[2], mB[2];
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kNA && e == cudaSuccess; ++i) e = plane_map(&mA[i], a.A[i], a.a_rows, a.k, kTM);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = plane_map(&mB[i], a.B[i], a.b_rows, a.k, kTN);
    if (e != cudaSuccess) return e;
    if (kNA == 1) mA[1] = mA[0];
    e = cudaFuncSetAttribute(dft_tc_kernel<kPass>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.b_rows + kTN - 1) / kTN, (a.a_rows + kTM - 1) / kTM);
    dft_tc_kernel<kPass><<<grid, 128, smem, s>>>(a, mA[0], mA[1], mB[0], mB[1]);
    return cudaGetLastError();
}
}  // namespace

size_t model_grid_ws_bytes(int n_img, int n_grid) {
    const size_t n = (size_t)n_img, ng = (size_t)n_grid;
    if (use_tc(n_img))
    {
        const size_t kp = (size_t)kpad(n_img);
        return al256(ng * sizeof(double2)) + al256(3 * n * kp * 2) + 4 * al256(3 * ng * kp * 2) + 256;
    }
    return al256(n * ng * sizeof(float2)) + al256(ng * sizeof(float2)) + 256;
}

cudaError_t launch_model_grid(int n_img, int n_grid, const float *image, void *ws, float2 *grid_out, int **err_dev,
                              cudaStream_t s) {
    const size_t n = (size_t)n_img, ng = (size_t)n_grid;
    unsigned char *p = (unsigned char *)ws;
    if (!use_tc(n_img)) {
        float2 *tmp = (float2 *)p;
        float2 *twiddle = (float2 *)(p + al256(n * ng * sizeof(float2)));
        *err_dev = (int *)(p + al256(n * ng * sizeof(float2)) + al256(ng * sizeof(float2)));
        cudaError_t e = cudaMemsetAsync(*err_dev, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        twiddle_kernel<<<(n_grid + 255) / 256, 256, 0, s>>>(twiddle, n_grid);
        dim3 g1((n_grid + kBN - 1) / kBN, (n_img + kBM - 1) / kBM);
        dft_rows_kernel<<<g1, 256, 0, s>>>(image, twiddle, n_img, n_grid, tmp);
        dim3 g2((n_grid + kBN - 1) / kBN, (n_grid + kBM - 1) / kBM);
        dft_cols_kernel<<<g2, 256, 0, s>>>(tmp, twiddle, n_img, n_grid, grid_out);
        return cudaGetLastError();
    }
    const int kp = kpad(n_img);
    const size_t kz = (size_t)kp;
    double2 *tw = (double2 *)p;
    p += al256(ng * sizeof(double2));
    bf16 *I3 = (bf16 *)p;
    p += al256(3 * n * kz * 2);
    bf16 *Er = (bf16 *)p; p += al256(3 * ng * kz * 2);
    bf16 *Ei = (bf16 *)p; p += al256(3 * ng * kz * 2);
    bf16 *Tr = (bf16 *)p; p += al256(3 * ng * kz * 2);
    bf16 *Ti = (bf16 *)p; p += al256(3 * ng * kz * 2);
    *err_dev = (int *)p;
    cudaError_t e = cudaMemsetAsync(*err_dev, 0, sizeof(int), s);
    // pass 1 writes T's first N columns; the padding columns stay zero
    if (e == cudaSuccess) e = cudaMemsetAsync(Tr, 0, 2 * al256(3 * ng * kz * 2), s);
    if (e != cudaSuccess) return e;
    twiddle64_kernel<<<(n_grid + 255) / 256, 256, 0, s>>>(tw, n_grid);
    split_image_kernel<<<(int)std::min<size_t>((n * kz + 255) / 256, 4096), 256, 0, s>>>(image, n_img, kp, I3);
    split_dft_matrix_kernel<<<(int)std::min<size_t>((ng * kz + 255) / 256, 8192), 256, 0, s>>>(tw, n_img, n_grid, kp, Er,
                                                                                                  Ei);
    TcPassArgs a1{};
    a1.A[0] = I3; a1.n_a = 1;
    a1.B[0] = Er; a1.B[1] = Ei;
    a1.a_rows = n_img; a1.b_rows = n_grid; a1.k = kp;
    a1.Tr = Tr; a1.Ti = Ti; a1.ng = n_grid; a1.err = *err_dev;
    e = launch_tc_pass<1>(a1, s);
    if (e != cudaSuccess) return e;
    TcPassArgs a2{};
    a2.A[0] = Tr; a2.A[1] = Ti; a2.n_a = 2;
    a2.B[0] = Er; a2.B[1] = Ei;
    a2.a_rows = n_grid; a2.b_rows = n_grid; a2.k = kp;
    a2.G = grid_out; a2.ng = n_grid; a2.err = *err_dev;
    return launch_tc_pass<2>(a2, s);
}

size_t model_grid_comp_ws_bytes(int n_comp, int n_grid, int stride) {
    const size_t kp = (size_t)comp_depth(n_comp), ng = (size_t)n_grid;
    return al256((size_t)n_comp * stride * sizeof(double)) + 4 * al256(3 * ng * kp * 2) + 256;
}

cudaError_t launch_model_grid_comp(int n_comp, const double *comp_host, int stride, double wp, int n_grid, double du,
                                   void *ws, float2 *grid_out, int **err_dev, cudaStream_t s) {
    const int kp = comp_depth(n_comp);
    const size_t ng = (size_t)n_grid;
    unsigned char *p = (unsigned char *)ws;
    double *comp = (double *)p; p += al256((size_t)n_comp * stride * sizeof(double));
    bf16 *Ar = (bf16 *)p; p += al256(3 * ng * kp * 2);
    bf16 *Ai = (bf16 *)p; p += al256(3 * ng * kp * 2);
    bf16 *Br = (bf16 *)p; p += al256(3 * ng * kp * 2);
    bf16 *Bi = (bf16 *)p; p += al256(3 * ng * kp * 2);
    *err_dev = (int *)p;
    cudaError_t e = cudaMemsetAsync(*err_dev, 0, sizeof(int), s);
    if (e == cudaSuccess && n_comp > 0)
        e = cudaMemcpyAsync(comp, comp_host, (size_t)n_comp * stride * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    split_comp_kernel<<<(int)std::min<size_t>((ng * kp + 255) / 256, 8192), 256, 0, s>>>(
        comp, n_comp, stride, wp, kp, n_grid, du, Ar, Ai, Br, Bi);
    TcPassArgs a2{};
    a2.A[0] = Ar; a2.A[1] = Ai; a2.n_a = 2;
    a2.B[0] = Br; a2.B[1] = Bi;
    a2.a_rows = n_grid; a2.b_rows = n_grid; a2.k = kp;
    a2.G = grid_out; a2.ng = n_grid; a2.err = *err_dev;
    return launch_tc_pass<2>(a2, s);
}

}  // namespace psc

// Device helpers of the fused evaluation kernels (eval.cu, track.cu): complex
// products, hardware square roots, packed FP32x2 arithmetic, the grid
// position of a visibility from the FP32 split of its baseline, and the
// per-row tap loops of the kernel of Eq. AIJPOINTING (radial A° table in
// shared memory as intercept/slope pairs, the phase ramp factored out of the
// taps).  Internal; included by the .cu files only.
#pragma once

#include <cuda_runtime.h>

namespace psc {
namespace tap {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float rsqrt_fast(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// (px, py) += a (gx, gy) as one packed FP32x2 FMA: each lane rounds exactly
// like fmaf, and the pair costs one instruction instead of two.
__device__ __forceinline__ void fma2_acc(float &px, float &py, float a, float gx, float gy) {
    asm("{\n.reg .b64 aa, gg, pp;\nmov.b64 aa, {%2, %2};\nmov.b64 gg, {%3, %4};\nmov.b64 pp, {%0, %1};\n"
        "fma.rn.f32x2 pp, aa, gg, pp;\nmov.b64 {%0, %1}, pp;\n}"
        : "+f"(px), "+f"(py) : "f"(a), "f"(gx), "f"(gy));
}

// Shared-memory load at a 32-bit shared address.  Not volatile: the loads
// are pure, and the compiler may schedule them early (they are only issued
// inside tap loops that follow the barrier publishing the tables).
__device__ __forceinline__ float2 lds_f2(unsigned addr) {
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// Grid position x = u sc + Ng/2 of a baseline coordinate given as two floats
// (u = uh + ul, metres) and the channel's scale sc = sh + sl, without FP64:
// the product's rounding error comes from an FMA (exact), the small cross
// terms are added to it, and Ng/2 is added with Knuth's TwoSum, whose error
// term is exact.  Returns floor(x) in n and x - floor(x) in f (rounded once
// to FP32).
__device__ __forceinline__ void grid_pos(float uh, float ul, float sh, float sl, float half, int &n, float &f) {
    // _rn intrinsics: no FMA contraction may merge these steps
    const float p = __fmul_rn(uh, sh);
    float e = fmaf(uh, sh, -p);
    e = fmaf(uh, sl, e);
    e = fmaf(ul, sh, e);
    const float s = __fadd_rn(half, p);
    const float bb = __fsub_rn(s, half);
    const float r = __fadd_rn(__fsub_rn(half, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float fl = floorf(s);
    f = __fadd_rn(__fsub_rn(s, fl), __fadd_rn(r, e));     // s - fl is exact
    n = (int)fl;
    if (f < 0.f) { f += 1.f; n -= 1; }
    else if (f >= 1.f) { f -= 1.f; n += 1; }
}

// Packed FP32x2 helpers on float2 pairs (each lane rounds like the scalar op).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n.reg .b64 aa, bb, cc;\nmov.b64 aa, {%2, %3};\nmov.b64 bb, {%4, %5};\nmov.b64 cc, {%6, %7};\n"
        "fma.rn.f32x2 cc, aa, bb, cc;\nmov.b64 {%0, %1}, cc;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 aa, bb;\nmov.b64 aa, {%2, %3};\nmov.b64 bb, {%4, %5};\n"
        "mul.rn.f32x2 aa, aa, bb;\nmov.b64 {%0, %1}, aa;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 aa, bb;\nmov.b64 aa, {%2, %3};\nmov.b64 bb, {%4, %5};\n"
        "add.rn.f32x2 aa, aa, bb;\nmov.b64 {%0, %1}, aa;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fadd2_rz(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 aa, bb;\nmov.b64 aa, {%2, %3};\nmov.b64 bb, {%4, %5};\n"
        "add.rz.f32x2 aa, aa, bb;\nmov.b64 {%0, %1}, aa;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// The row loop for two visibilities with their per-visibility scalars
// packed in pairs: s2, floor(t) + 2^23, A dxo and the dxo step are one packed
// instruction for both.
__device__ __forceinline__ void row_taps2(const float2 *__restrict__ row, int n, float2 dxo, float2 dyo2, float ov,
                                          unsigned tab_adj, float (&pr)[2], float (&pi)[2], float (&qr)[2],
                                          float (&qi)[2]) {
    const float2 step = make_float2(-ov, -ov);
    const float2 magic = make_float2(8388608.0f, 8388608.0f);
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
        const float2 g = row[k];
        const float2 s2 = ffma2(dxo, dxo, dyo2);
        const float2 t = make_float2(sqrt_fast(s2.x), sqrt_fast(s2.y));
        const float2 tf = fadd2_rz(t, magic);                       // floor(t) + 2^23, both
        const float2 e0 = lds_f2(tab_adj + ((unsigned)__float_as_int(tf.x) << 3));
        const float2 e1 = lds_f2(tab_adj + ((unsigned)__float_as_int(tf.y) << 3));
        const float2 A = make_float2(fmaf(t.x, e0.y, e0.x), fmaf(t.y, e1.y, e1.x));
        const float2 Ad = fmul2(A, dxo);
        fma2_acc(pr[0], pi[0], A.x, g.x, g.y);
        fma2_acc(pr[1], pi[1], A.y, g.x, g.y);
        fma2_acc(qr[0], qi[0], Ad.x, g.x, g.y);
        fma2_acc(qr[1], qi[1], Ad.y, g.x, g.y);
        dxo = fadd2(dxo, step);
    }
}

// One row of taps for kV visibilities: n consecutive staged cells starting at
// row (shared memory); visibility v's first tap is at dxo[v] (= dx ov).  The
// table address is tab_adj + (bits of floor(t) + 2^23) * 8.  Accumulates
// P = sum A G' and Q = sum A dxo G' per visibility.
template <int kV>
__device__ __forceinline__ void row_taps(const float2 *__restrict__ row, int n, float (&dxo)[kV],
                                         const float (&dyo2)[kV], float ov, unsigned tab_adj, float (&pr)[kV],
                                         float (&pi)[kV], float (&qr)[kV], float (&qi)[kV]) {
    constexpr int kUnroll = 4;
#pragma unroll kUnroll
    for (int k = 0; k < n; ++k) {
        const float2 g = row[k];
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float s2 = fmaf(dxo[v], dxo[v], dyo2[v]);
            const float t = sqrt_fast(s2);
            const float tf = __fadd_rz(t, 8388608.0f);          // floor(t) + 2^23
            const float2 e = lds_f2(tab_adj + ((unsigned)__float_as_int(tf) << 3));
            const float A = fmaf(t, e.y, e.x);
            fma2_acc(pr[v], pi[v], A, g.x, g.y);
            fma2_acc(qr[v], qi[v], A * dxo[v], g.x, g.y);
            dxo[v] -= ov;
        }
    }
}

}  // namespace tap
}  // namespace psc

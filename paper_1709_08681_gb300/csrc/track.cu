// Track kernel: the fused evaluation of Algorithm 1's inner loop for small
// apertures (a few to a few tens of taps per visibility), one warp per
// baseline track.
//
// Paper basis (Bhatnagar & Cornwell 2017): the kernel A_ij of Eq.
// AIJPOINTING and its derivatives of Eq. DAIJPOINTING (extended to m, Sec. 3),
// chi^2 of Eq. Chisq and its gradient, Eq. DCHIDD -- the same arithmetic as
// eval.cu, organised for a different regime.
//
// Work decomposition.  An item is one baseline and one chunk of 32 kV
// consecutive time steps; lane l owns the kV visibilities at times
// chunk 32 kV + l kV + v of one channel, and the warp loops over all channels.
// Within one channel the chunk's visibilities sit on a short arc of the uv
// track (a 60 s chunk of a 16 km baseline moves under 20 cells), so the
// warp's footprint -- the box of cells within rho_max of its visibilities --
// is small.  Each channel's box (8, 16 or 32 cells wide, in copies of 8 rows)
// and the channel's radial table are staged by TMA (cp.async.bulk.tensor for
// the grid, cp.async.bulk for the table) into one of the warp's two shared
// buffers, completing on that buffer's mbarrier; the copies of channel c + 1
// are issued before channel c is computed, so their latency hides behind it.
// The staged cells are then multiplied in place by the cell half of the phase
// ramp (origin: the box corner), exactly as eval.cu stages its tiles, and the
// taps run the same inner loop.  Warps never wait on one another: there is no
// block barrier.  Boxes wider than 32 cells or taller than the tile fall back
// to taps read from global memory with the ramp applied per tap.
//
// Sums.  Over the channels, each lane keeps ten moments from which the
// item's fifteen sums follow (see the epilogue), in shared memory rather than
// registers, which the tap loops need: chi^2 and the three gradient
// moments with Knuth's TwoSum (compensated FP32: a running sum and its
// rounding error), the six normal-equation moments in plain FP32.  One
// butterfly over the warp per item (TwoSum again for the compensated four)
// gives the item's moments; the fifteen sums are formed from them in FP64 and
// written as the item's record.  Records are summed per baseline in FP64 in a
// fixed order (bl_reduce_kernel), so the results do not depend on which warp
// ran which item.
//
// Waits.  Every mbarrier wait is bounded (wait_limit polls).  A wait that runs
// out sets *err; the warp then waits, with a fixed larger bound, for its own
// copies still in flight and returns.  The host reports PSC_ERR_TIMEOUT.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "psc_internal.cuh"
#include "tap_math.cuh"

namespace psc {
namespace {

using namespace tap;

constexpr int kTrkWarps = kTrkThreads / 32;
constexpr int kBoxRows = 8;                 // rows of one TMA copy
constexpr int kMaxBoxW = 32;                // widest staged box (cells)
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kDrainPolls = 1LL << 26;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t mb) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb));
}

// Bounded wait for a phase of mbarrier mb: at most `limit` polls, each of
// which may suspend the warp for up to a microsecond (a hint to the
// hardware) instead of spinning.
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n"
                     "selp.u32 %0, 1, 0, q;\n}"
                     : "=r"(ok) : "r"(mb), "r"(parity), "r"(1000u) : "memory");
        if (ok) return true;
    }
    return false;
}

// The asynchronous copies, each issued by the lanes whose p is nonzero (no
// branch around it): the arrival that sets a phase's expected bytes; one 2-D
// TMA copy of a W x 8 box of the grid (x = column, y = row) to dst; one
// contiguous bulk copy (16-byte aligned addresses, size a multiple of 16).
// All complete on mbarrier mb.
__device__ __forceinline__ void mbar_expect_if(int p, uint32_t mb, uint32_t bytes) {
    asm volatile("{\n.reg .pred q;\nsetp.ne.s32 q, %2, 0;\n@q mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n}"
                 :: "r"(mb), "r"(bytes), "r"(p) : "memory");
}

__device__ __forceinline__ void tma_box_if(int p, uint32_t dst, const void *map, int x, int y, uint32_t mb) {
    asm volatile("{\n.reg .pred q;\nsetp.ne.s32 q, %5, 0;\n"
                 "@q cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n}"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mb), "r"(p) : "memory");
}

__device__ __forceinline__ void bulk_copy_if(int p, uint32_t dst, const void *src, uint32_t bytes, uint32_t mb) {
    asm volatile("{\n.reg .pred q;\nsetp.ne.s32 q, %4, 0;\n"
                 "@q cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n}"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mb), "r"(p) : "memory");
}

// Grid position x = u sc + Ng/2 from the FP32 split u = uh + ul and
// sc = sh + sl: the product's rounding error by an FMA (exact) plus the cross
// terms; p - floor(p) is exact, so f carries the bits below p's ulp.
__device__ __forceinline__ void trk_pos(float uh, float ul, float sh, float sl, int half, int &n, float &f) {
    const float p = __fmul_rn(uh, sh);
    float e = fmaf(uh, sh, -p);
    e = fmaf(uh, sl, e);
    e = fmaf(ul, sh, e);
    const float fl = floorf(p);
    f = __fadd_rn(__fsub_rn(p, fl), e);
    n = (int)fl + half;
    if (f < 0.f) { f += 1.f; n -= 1; }
    else if (f >= 1.f) { f -= 1.f; n += 1; }
}

// s + c += x with Knuth's TwoSum: s keeps the rounded sum, c the exact rounding errors.
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, err);
}

struct Box {
    int x0, x1, y0, y1;   // inclusive cell range of the warp's footprint; x0 rounded down to even
    int n0, m0;           // this lane's first visibility: base cell and fraction in the channel
    float f0, g0;
};

// The warp's footprint in a channel of scale (sh, sl): the union over lanes
// of each lane's tap pattern, the cells (n0 + a, m0 + b), a, b in [1 - R, R],
// around the base cell (n0, m0) of its first visibility (u, v split q0; R the
// ceiling of the pattern radius rp, see the tap pattern below).
__device__ __forceinline__ Box chan_box(const float4 &q0, float sh, float sl, int half, float rp) {
    int n0, m0;
    float f0, g0;
    trk_pos(q0.x, q0.y, sh, sl, half, n0, f0);
    trk_pos(q0.z, q0.w, sh, sl, half, m0, g0);
    const int R = (int)ceilf(rp);
    Box b;
    b.n0 = n0;
    b.m0 = m0;
    b.f0 = f0;
    b.g0 = g0;
    b.x0 = __reduce_min_sync(kFull, n0 + 1 - R) & ~1;     // TMA: the first column at a 16-byte boundary
    b.x1 = __reduce_max_sync(kFull, n0 + R);
    b.y0 = __reduce_min_sync(kFull, m0 + 1 - R);
    b.y1 = __reduce_max_sync(kFull, m0 + R);
    return b;
}

// Box width class (8, 16 or 32 cells; 0 = does not fit) and its TMA copies.
__device__ __forceinline__ int box_width(const Box &b) {
    const int w = b.x1 - b.x0 + 1;
    return w <= 8 ? 8 : w <= 16 ? 16 : w <= kMaxBoxW ? 32 : 0;
}

__device__ __forceinline__ void sts_f2(uint32_t addr, float2 v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" :: "r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

__device__ __forceinline__ unsigned tab_addr(unsigned tab_adj, float tf) {
    return tab_adj + ((unsigned)__float_as_int(tf) << 3);
}

// Two rows of the tap pattern at once, for a lane's two visibilities,
// unrolled.  Rows b and 1 - b have the same width (the pattern is symmetric
// about the unit cell): 2 kCW cells each from shared addresses row_a and
// row_b (the rows' first column a = 1 - kCW), so they share the column offsets
// dxo.v = (x_v - a) ov; their squared row offsets differ (dyo2a, dyo2b).
// Returns each row's sums P_v = sum A G' (pa0, pa1; pb0, pb1) and adds both
// rows' sum A dxo G' to su0, su1.  Twice the independent work per unrolled
// body, half the row set-ups and dispatches.
template <int kCW>
__device__ __forceinline__ void pat_pair2(uint32_t row_a, uint32_t row_b, float2 dxo, float2 dyo2a, float2 dyo2b,
                                          float2 step, uint32_t tab_adj, float2 &pa0, float2 &pa1, float2 &pb0,
                                          float2 &pb1, float2 &su0, float2 &su1) {
    const float2 magic = make_float2(8388608.0f, 8388608.0f);
#pragma unroll
    for (int k = 0; k < 2 * kCW; ++k) {
        const float2 ga = lds_f2(row_a + 8u * k);
        const float2 gb = lds_f2(row_b + 8u * k);
        const float2 sa = ffma2(dxo, dxo, dyo2a);
        const float2 sb = ffma2(dxo, dxo, dyo2b);
        const float2 ta = make_float2(sqrt_fast(sa.x), sqrt_fast(sa.y));
        const float2 tb = make_float2(sqrt_fast(sb.x), sqrt_fast(sb.y));
        const float2 fa = fadd2_rz(ta, magic);
        const float2 fb = fadd2_rz(tb, magic);
        const float2 ea0 = lds_f2(tab_addr(tab_adj, fa.x));
        const float2 ea1 = lds_f2(tab_addr(tab_adj, fa.y));
        const float2 eb0 = lds_f2(tab_addr(tab_adj, fb.x));
        const float2 eb1 = lds_f2(tab_addr(tab_adj, fb.y));
        const float2 Aa = make_float2(fmaf(ta.x, ea0.y, ea0.x), fmaf(ta.y, ea1.y, ea1.x));
        const float2 Ab = make_float2(fmaf(tb.x, eb0.y, eb0.x), fmaf(tb.y, eb1.y, eb1.x));
        const float2 Ada = fmul2(Aa, dxo);
        const float2 Adb = fmul2(Ab, dxo);
        if (k == 0) {
            pa0 = fmul2(make_float2(Aa.x, Aa.x), ga);
            pa1 = fmul2(make_float2(Aa.y, Aa.y), ga);
            pb0 = fmul2(make_float2(Ab.x, Ab.x), gb);
            pb1 = fmul2(make_float2(Ab.y, Ab.y), gb);
        } else {
            fma2_acc(pa0.x, pa0.y, Aa.x, ga.x, ga.y);
            fma2_acc(pa1.x, pa1.y, Aa.y, ga.x, ga.y);
            fma2_acc(pb0.x, pb0.y, Ab.x, gb.x, gb.y);
            fma2_acc(pb1.x, pb1.y, Ab.y, gb.x, gb.y);
        }
        fma2_acc(su0.x, su0.y, Ada.x, ga.x, ga.y);
        fma2_acc(su1.x, su1.y, Ada.y, ga.x, ga.y);
        fma2_acc(su0.x, su0.y, Adb.x, gb.x, gb.y);
        fma2_acc(su1.x, su1.y, Adb.y, gb.x, gb.y);
        dxo = fadd2(dxo, step);
    }
}

// One row of the pattern for one visibility per lane, unrolled: 2 kCW cells
// from `row`, the first at dxo = (x - a) ov.  Returns P = sum A G' in p and
// adds sum A dxo G' to su.
template <int kCW>
__device__ __forceinline__ void pat_row1(uint32_t row, float dxo, float dyo2, float ov, uint32_t tab_adj, float2 &p,
                                         float2 &su) {
#pragma unroll
    for (int k = 0; k < 2 * kCW; ++k) {
        const float2 g = lds_f2(row + 8u * k);
        const float t = sqrt_fast(fmaf(dxo, dxo, dyo2));
        const float2 e = lds_f2(tab_addr(tab_adj, __fadd_rz(t, 8388608.0f)));
        const float A = fmaf(t, e.y, e.x);
        if (k == 0) p = make_float2(A * g.x, A * g.y);
        else fma2_acc(p.x, p.y, A, g.x, g.y);
        fma2_acc(su.x, su.y, A * dxo, g.x, g.y);
        dxo -= ov;
    }
}

// Rows wider than the unrolled ones (apertures past 6 cells): the same taps in a loop.
__device__ __forceinline__ void pat_row2_n(uint32_t row, int n, float2 dxo, float2 dyo2, float2 step, uint32_t tab_adj,
                                           float2 &p0, float2 &p1, float2 &su0, float2 &su1) {
    const float2 magic = make_float2(8388608.0f, 8388608.0f);
    p0 = p1 = make_float2(0.f, 0.f);
    for (int k = 0; k < n; ++k) {
        const float2 g = lds_f2(row + 8u * k);
        const float2 s2 = ffma2(dxo, dxo, dyo2);
        const float2 t = make_float2(sqrt_fast(s2.x), sqrt_fast(s2.y));
        const float2 tf = fadd2_rz(t, magic);
        const float2 e0 = lds_f2(tab_addr(tab_adj, tf.x));
        const float2 e1 = lds_f2(tab_addr(tab_adj, tf.y));
        const float2 A = make_float2(fmaf(t.x, e0.y, e0.x), fmaf(t.y, e1.y, e1.x));
        const float2 Ad = fmul2(A, dxo);
        fma2_acc(p0.x, p0.y, A.x, g.x, g.y);
        fma2_acc(p1.x, p1.y, A.y, g.x, g.y);
        fma2_acc(su0.x, su0.y, Ad.x, g.x, g.y);
        fma2_acc(su1.x, su1.y, Ad.y, g.x, g.y);
        dxo = fadd2(dxo, step);
    }
}

__device__ __forceinline__ void pat_row1_n(uint32_t row, int n, float dxo, float dyo2, float ov, uint32_t tab_adj,
                                           float2 &p, float2 &su) {
    p = make_float2(0.f, 0.f);
    for (int k = 0; k < n; ++k) {
        const float2 g = lds_f2(row + 8u * k);
        const float t = sqrt_fast(fmaf(dxo, dxo, dyo2));
        const float2 e = lds_f2(tab_addr(tab_adj, __fadd_rz(t, 8388608.0f)));
        const float A = fmaf(t, e.y, e.x);
        fma2_acc(p.x, p.y, A, g.x, g.y);
        fma2_acc(su.x, su.y, A * dxo, g.x, g.y);
        dxo -= ov;
    }
}

template <int kV>
__global__ void __launch_bounds__(kTrkThreads, 4)
track_kernel(const EvalArgs a0, const EvalArgs *__restrict__ args, const long long *__restrict__ prefix, int n_ctx,
             unsigned long long *queue, int cap, int tabc) {
    extern __shared__ __align__(128) unsigned char trk_raw[];
    __shared__ EvalArgs s_args[kTrkWarps];
    __shared__ __align__(8) unsigned long long s_mbar[kTrkWarps][2];
    __shared__ float s_mom[kTrkWarps][14][32];      // the lanes' running channel moments
    __shared__ float4 s_q[kTrkWarps][2][32];         // per lane: first (u, v) split; (du1, dv1, wv0, wv1)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool persistent = queue != nullptr;
    EvalArgs &a = s_args[warp];
    // this warp's two buffers, [tile cap][table tabc] each (shared addresses),
    // from a 128-byte boundary
    const uint32_t dyn0 = (saddr(trk_raw) + 127u) & ~127u;
    const uint32_t buf_bytes = (uint32_t)(cap + tabc) * 8u;
    const uint32_t tile0 = dyn0 + (uint32_t)warp * 2u * buf_bytes;
    const uint32_t mb0 = saddr(&s_mbar[warp][0]), mb1 = saddr(&s_mbar[warp][1]);
    if (lane == 0) {
        mbar_init(mb0);
        mbar_init(mb1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!persistent) a = a0;
    }
    __syncwarp();
    uint32_t par = 0;                  // bit b: parity of buffer b's next completion
    uint32_t pending = 0;              // bit b: a copy into buffer b not yet waited for
    int cur = -1;
    long long first = 0;
    long long gi_static = (long long)blockIdx.x * kTrkWarps + warp;
    const float pi_f = 3.14159265358979f;

    for (;;) {
        long long gi;
        if (persistent) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(queue, 1ull);
            gi = (long long)__shfl_sync(kFull, t, 0);
            if (gi >= prefix[n_ctx]) break;
            if (cur < 0 || gi < prefix[cur] || gi >= prefix[cur + 1]) {
                int lo = 0, hi = n_ctx - 1;            // last context with prefix[k] <= gi
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (prefix[mid] <= gi) lo = mid; else hi = mid - 1;
                }
                cur = lo;
                first = prefix[lo];
                __syncwarp();                          // every lane is done reading the old arguments
                const int *src = reinterpret_cast<const int *>(&args[lo]);
                int *dst = reinterpret_cast<int *>(&a);
                for (int i = lane; i < (int)(sizeof(EvalArgs) / 4); i += 32) dst[i] = src[i];
                __syncwarp();
            }
        } else {
            gi = gi_static;
            gi_static += (long long)gridDim.x * kTrkWarps;
            if (gi >= a.n_bricks) break;
        }
        if (a.skip != nullptr && *a.skip) continue;
        const int item = (int)(gi - first);
        const int chunks = a.trk_chunks;
        const int qbl = item / chunks, chunk = item - qbl * chunks;
        const int bl = a.bl_order != nullptr ? a.bl_order[qbl] : qbl;
        const int brick = bl * chunks + chunk;
        const int2 ij = a.pairs[bl];
        const double li = a.lm[2 * ij.x], mi = a.lm[2 * ij.x + 1];
        const double lj = a.lm[2 * ij.y], mj = a.lm[2 * ij.y + 1];
        const float L = (float)(li + lj), M = (float)(mi + mj);       // ramp
        const float dL = (float)(li - lj), dM = (float)(mi - mj);     // decorrelation
        const int nt = a.nt, nc = a.nc, n_bl = a.n_bl, half = a.ng / 2;
        const float du = a.du, ov = (float)a.ov;
        const int tb = chunk * 32 * kV + lane * kV;
        // rows of the lane's visibilities in uvs (past the interval's end: the
        // last step again, with weight 0) and of their first channel in vis_obs
        const int t0 = min(tb, nt - 1);
        const int tstep = kV == 2 && tb + 1 < nt ? 1 : 0;
        const float4 *uvs0 = a.uvs + (size_t)t0 * n_bl + bl;
        const size_t uvs_step = (size_t)tstep * n_bl;
        const size_t kb0 = ((size_t)t0 * n_bl + bl) * nc;
        const size_t kstep = uvs_step * nc;
        // (u, v) of the second visibility minus the first, metres: the split
        // parts' differences are exact (neighbouring time steps)
        float du1 = 0.f, dv1 = 0.f;
        if (kV == 2 && tstep) {
            const float4 q0 = uvs0[0], q1 = uvs0[uvs_step];
            du1 = __fadd_rn(__fsub_rn(q1.x, q0.x), __fsub_rn(q1.y, q0.y));
            dv1 = __fadd_rn(__fsub_rn(q1.z, q0.z), __fsub_rn(q1.w, q0.w));
        }
        const float wv0 = tb < nt ? a.w_scale : 0.f;
        const float wv1 = tb + 1 < nt ? a.w_scale : 0.f;
        // the lane's running sums (see the epilogue): chi^2 and the gradient
        // moments compensated (TwoSum), the normal-equation moments plain
        float (*mom)[32] = s_mom[warp];
#pragma unroll
        for (int k = 0; k < 14; ++k) mom[k][lane] = 0.f;
        // pattern radius: the aperture's reach plus the largest distance between
        // a lane's visibilities in this item (metres here; times the channel's
        // scale, cells), plus a margin
        const float sp_m = kV == 2 ? __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(sqrtf(du1 * du1 + dv1 * dv1))))
                                   : 0.f;

        ChanConst ch = a.chan[0];
        // per-lane item constants live in shared memory, not registers (the tap
        // loops need every register): the first visibility's (u, v) split,
        // read for every channel's box, and (du1, dv1, weight 0, weight 1)
        const float4 &q00 = s_q[warp][0][lane];
        const float4 &qd = s_q[warp][1][lane];
        s_q[warp][0][lane] = uvs0[0];
        s_q[warp][1][lane] = make_float4(du1, dv1, wv0, wv1);
        Box box = chan_box(q00, ch.sc_hi, ch.sc_lo, half, ch.rho_max + fmaf(sp_m, ch.sc_hi, 1e-3f));
        bool ok = true;
        // issues the copies of channel cc (box bx, table length tl) into buffer bb
        auto issue = [&](int cc, int tl, const Box &bx, int bb) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes before async-proxy writes
            __syncwarp();
            // lane 0 arrives with the expected bytes; lanes 0..ncp-1 copy one
            // 8-row box each and lane 31 the table (a phase completes once the
            // arrival and all bytes are in, in whatever order)
            const int W = box_width(bx);
            const int ncp = (bx.y1 - bx.y0 + 1 + kBoxRows - 1) / kBoxRows;
            const bool fits = W > 0 && W * kBoxRows * ncp <= a.trk_cap;
            const int n_tab = min(a.trk_stride, (tl + a.trk_pad + 1) & ~1);
            const uint32_t tab_bytes = (uint32_t)n_tab * 8u;
            const uint32_t mb = bb ? mb1 : mb0;
            const uint32_t tile = tile0 + (uint32_t)bb * buf_bytes;
            mbar_expect_if(lane == 0, mb, tab_bytes + (fits ? (uint32_t)(W * kBoxRows * ncp) * 8u : 0u));
            __syncwarp();
            {
                const char *map = reinterpret_cast<const char *>(a.tmap) + (W == 8 ? 0 : W == 16 ? 128 : 256);
                tma_box_if(fits && lane < ncp, tile + (uint32_t)(lane * kBoxRows * W * 8), map, bx.x0,
                           bx.y0 + lane * kBoxRows, mb);
            }
            bulk_copy_if(lane == 31, tile + (uint32_t)cap * 8u, a.tabs_cs + (size_t)cc * a.trk_stride, tab_bytes, mb);
            pending |= 1u << bb;
        };
        issue(0, ch.tab_len, box, 0);

        for (int c = 0; c < nc; ++c) {
            const int b = c & 1;
            // prefetch channel c + 1 into the other buffer (its last reader was channel c - 1)
            Box boxn = box;
            ChanConst chn = ch;
            if (c + 1 < nc) {
                chn = a.chan[c + 1];
                boxn = chan_box(q00, chn.sc_hi, chn.sc_lo, half, chn.rho_max + fmaf(sp_m, chn.sc_hi, 1e-3f));
                issue(c + 1, chn.tab_len, boxn, b ^ 1);
            }
            const bool got = mbar_wait(b ? mb1 : mb0, (par >> b) & 1u, a.wait_limit);
            if (__any_sync(kFull, !got)) { ok = false; break; }
            par ^= 1u << b;
            pending &= ~(1u << b);

            // positions of the lane's visibilities in this channel
            int nx[kV], ny[kV];
            float fx[kV], fy[kV];
            nx[0] = box.n0;                            // computed with the channel's box
            ny[0] = box.m0;
            fx[0] = box.f0;
            fy[0] = box.g0;
            if constexpr (kV == 2) {
                // the second visibility moved by (du1, dv1) metres: a fraction of a cell
                float gx = fmaf(qd.x, ch.sc_hi, fx[0]), gy = fmaf(qd.y, ch.sc_hi, fy[0]);
                const float flx = floorf(gx), fly = floorf(gy);
                nx[1] = nx[0] + (int)flx;
                ny[1] = ny[0] + (int)fly;
                fx[1] = gx - flx;
                fy[1] = gy - fly;
            }
            // the channel's observed visibilities and weights, loaded now so that
            // their latency hides behind the taps
            float2 vo[kV];
            float wk[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const size_t k = kb0 + (size_t)v * kstep + c;
                vo[v] = a.vis_obs[k];
                wk[v] = (v == 0 ? qd.z : qd.w) * (a.w != nullptr ? a.w[k] : 1.f);
            }
            const float rmax = ch.rho_max, rmax2 = rmax * rmax;
            const int W = box_width(box);
            const int ncp = (box.y1 - box.y0 + 1 + kBoxRows - 1) / kBoxRows;
            const bool staged = W > 0 && W * kBoxRows * ncp <= a.trk_cap;
            const uint32_t tile = tile0 + (uint32_t)b * buf_bytes;
            const unsigned tab_adj = tile + (uint32_t)cap * 8u - (0x4B000000u << 3);
            float2 S0[kV], Su[kV], Sv[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) S0[v] = Su[v] = Sv[v] = make_float2(0.f, 0.f);
            float parg[kV];                            // the visibility half of the ramp: its phase
            if (staged) {
                // cell half of the ramp, in place: cell (col, r) *= exp(-i pi du (col L + r M))
                const int lw = W == 8 ? 3 : W == 16 ? 4 : 5;
                const int col = lane & (W - 1);
                const int rstep = 32 >> lw;
                const int rows = box.y1 - box.y0 + 1;
                if (col <= box.x1 - box.x0) {
                    int r = lane >> lw;
                    float zs, zc, ss, sc;
                    __sincosf(-pi_f * du * ((float)col * L + (float)r * M), &zs, &zc);
                    __sincosf(-pi_f * du * ((float)rstep * M), &ss, &sc);
                    float2 z = make_float2(zc, zs);
                    const float2 stp = make_float2(sc, ss);
                    uint32_t cell = tile + (uint32_t)(r * W + col) * 8u;
                    const uint32_t cstep = (uint32_t)(rstep * W) * 8u;
                    for (; r < rows; r += rstep, cell += cstep) {
                        sts_f2(cell, cmul(lds_f2(cell), z));
                        z = cmul(z, stp);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    parg[v] = pi_f * du * (((float)(nx[v] - box.x0) + fx[v]) * L + ((float)(ny[v] - box.y0) + fy[v]) * M);
                }
                // The tap pattern, the same for every lane of the warp (no
                // divergence, no per-lane spans): relative to the lane's base
                // cell (n0, m0), the cells (a, b) within rp of some point of
                // the unit cell [0, 1)^2 -- rows b in [1 - R, R], row b's
                // columns a in [1 - ceil(w_b), ceil(w_b)], w_b = sqrt(rp^2 - d_b^2)
                // with d_b the row's distance from the unit cell.  Every cell
                // within rho_max of any of the lane's visibilities is in it;
                // the others read zero table entries (the tables are padded
                // past the aperture's reach + sqrt(2) + the context's largest step).
                const float rp = rmax + fmaf(sp_m, ch.sc_hi, 1e-3f), rp2 = rp * rp;
                const int R = (int)ceilf(rp);
                const uint32_t base = tile + (uint32_t)((ny[0] - box.y0) * W + (nx[0] - box.x0)) * 8u;
                if constexpr (kV == 2) {
                    const float2 ux = make_float2(fx[0], (float)(nx[1] - nx[0]) + fx[1]);
                    const float2 uy = make_float2(fy[0], (float)(ny[1] - ny[0]) + fy[1]);
                    const float2 ov2 = make_float2(ov, ov), step2 = make_float2(-ov, -ov);
                    float2 su0 = make_float2(0.f, 0.f), su1 = su0, s00 = su0, s01 = su0, sv0 = su0, sv1 = su0;
                    const float2 eps2 = make_float2(1e-20f, 1e-20f);
                    // rows b = -j and b = j + 1 (distance j from the unit cell) together
                    for (int j = 0; j < R; ++j) {
                        const float d = (float)j;
                        const float rem = fmaf(-d, d, rp2);
                        const int cw = (int)ceilf(rem * rsqrt_fast(rem));
                        const float fa = (float)(1 - cw);
                        const float2 dya = fadd2(uy, make_float2(d, d));
                        const float2 dyb = fadd2(uy, make_float2(-d - 1.f, -d - 1.f));
                        const float2 dyoa = fmul2(dya, ov2), dyob = fmul2(dyb, ov2);
                        const float2 dyo2a = ffma2(dyoa, dyoa, eps2), dyo2b = ffma2(dyob, dyob, eps2);
                        const float2 dxo = fmul2(fadd2(ux, make_float2(-fa, -fa)), ov2);
                        const uint32_t row_a = base + (uint32_t)(1 - cw - j * W) * 8u;
                        const uint32_t row_b = base + (uint32_t)((j + 1) * W + 1 - cw) * 8u;
                        float2 pa0, pa1, pb0, pb1;
                        switch (cw) {
                            case 1: pat_pair2<1>(row_a, row_b, dxo, dyo2a, dyo2b, step2, tab_adj, pa0, pa1, pb0, pb1, su0, su1); break;
                            case 2: pat_pair2<2>(row_a, row_b, dxo, dyo2a, dyo2b, step2, tab_adj, pa0, pa1, pb0, pb1, su0, su1); break;
                            case 3: pat_pair2<3>(row_a, row_b, dxo, dyo2a, dyo2b, step2, tab_adj, pa0, pa1, pb0, pb1, su0, su1); break;
                            case 4: pat_pair2<4>(row_a, row_b, dxo, dyo2a, dyo2b, step2, tab_adj, pa0, pa1, pb0, pb1, su0, su1); break;
                            case 5: pat_pair2<5>(row_a, row_b, dxo, dyo2a, dyo2b, step2, tab_adj, pa0, pa1, pb0, pb1, su0, su1); break;
                            case 6: pat_pair2<6>(row_a, row_b, dxo, dyo2a, dyo2b, step2, tab_adj, pa0, pa1, pb0, pb1, su0, su1); break;
                            default:
                                pat_row2_n(row_a, 2 * cw, dxo, dyo2a, step2, tab_adj, pa0, pa1, su0, su1);
                                pat_row2_n(row_b, 2 * cw, dxo, dyo2b, step2, tab_adj, pb0, pb1, su0, su1);
                        }
                        s00 = fadd2(s00, fadd2(pa0, pb0));
                        s01 = fadd2(s01, fadd2(pa1, pb1));
                        sv0 = ffma2(make_float2(dya.x, dya.x), pa0, sv0);
                        sv0 = ffma2(make_float2(dyb.x, dyb.x), pb0, sv0);
                        sv1 = ffma2(make_float2(dya.y, dya.y), pa1, sv1);
                        sv1 = ffma2(make_float2(dyb.y, dyb.y), pb1, sv1);
                    }
                    S0[0] = s00; S0[1] = s01; Su[0] = su0; Su[1] = su1; Sv[0] = sv0; Sv[1] = sv1;
                } else {
                    const float ux = fx[0], uy = fy[0];
                    for (int rb = 1 - R; rb <= R; ++rb) {
                        const float d = (float)(rb <= 0 ? -rb : rb - 1);
                        const float rem = fmaf(-d, d, rp2);
                        const int cw = (int)ceilf(rem * rsqrt_fast(rem));
                        const float dy = uy - (float)rb;
                        const float dyo = dy * ov;
                        const float dyo2 = fmaf(dyo, dyo, 1e-20f);
                        const float dxo = (ux - (float)(1 - cw)) * ov;
                        const uint32_t row = base + (uint32_t)(rb * W + 1 - cw) * 8u;
                        float2 p;
                        switch (cw) {
                            case 1: pat_row1<1>(row, dxo, dyo2, ov, tab_adj, p, Su[0]); break;
                            case 2: pat_row1<2>(row, dxo, dyo2, ov, tab_adj, p, Su[0]); break;
                            case 3: pat_row1<3>(row, dxo, dyo2, ov, tab_adj, p, Su[0]); break;
                            case 4: pat_row1<4>(row, dxo, dyo2, ov, tab_adj, p, Su[0]); break;
                            case 5: pat_row1<5>(row, dxo, dyo2, ov, tab_adj, p, Su[0]); break;
                            case 6: pat_row1<6>(row, dxo, dyo2, ov, tab_adj, p, Su[0]); break;
                            default: pat_row1_n(row, 2 * cw, dxo, dyo2, ov, tab_adj, p, Su[0]);
                        }
                        S0[0].x += p.x; S0[0].y += p.y;
                        Sv[0].x = fmaf(dy, p.x, Sv[0].x);
                        Sv[0].y = fmaf(dy, p.y, Sv[0].y);
                    }
                }
            } else {
                // fallback: taps read the grid (L1/L2), ramp per tap from each
                // visibility's own cell (nx, ny)
                float zxs, zxc;
                __sincosf(-pi_f * du * L, &zxs, &zxc);
                const float2 zx = make_float2(zxc, zxs);
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    parg[v] = pi_f * du * (fx[v] * L + fy[v] * M);
                    const int b_lo = max((int)floorf(fy[v] - rmax) + 1, -ny[v]);
                    const int b_hi = min((int)ceilf(fy[v] + rmax) - 1, a.ng - 1 - ny[v]);
                    for (int bb = b_lo; bb <= b_hi; ++bb) {
                        const float dy = fy[v] - (float)bb;
                        const float rem = rmax2 - dy * dy;
                        if (!(rem > 0.f)) continue;
                        const float r = fminf(rem * rsqrt_fast(rem), rmax);
                        const int a_lo = max((int)floorf(fx[v] - r) + 1, -nx[v]);
                        const int a_hi = min((int)ceilf(fx[v] + r) - 1, a.ng - 1 - nx[v]);
                        if (a_lo > a_hi) continue;
                        const float dyo = dy * ov;
                        const float dyo2 = fmaf(dyo, dyo, 1e-20f);
                        float zs, zc;
                        __sincosf(-pi_f * du * ((float)a_lo * L + (float)bb * M), &zs, &zc);
                        float2 z = make_float2(zc, zs);
                        float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
                        const float2 *rowp = a.grid + (size_t)(ny[v] + bb) * a.ng + nx[v];
                        float dd = (fx[v] - (float)a_lo) * ov;
                        // unrolled: four grid loads in flight per lane instead of one
#pragma unroll 4
                        for (int aa = a_lo; aa <= a_hi; ++aa, dd -= ov) {
                            const float2 g = cmul(__ldg(&rowp[aa]), z);
                            z = cmul(z, zx);
                            const float s2 = fmaf(dd, dd, dyo2);
                            const float tv = sqrt_fast(s2);
                            const float2 e = lds_f2(tab_addr(tab_adj, __fadd_rz(tv, 8388608.0f)));
                            const float A = fmaf(tv, e.y, e.x);
                            pr = fmaf(A, g.x, pr);
                            pi = fmaf(A, g.y, pi);
                            const float Ad = A * dd;
                            qr = fmaf(Ad, g.x, qr);
                            qi = fmaf(Ad, g.y, qi);
                        }
                        S0[v].x += pr; S0[v].y += pi;
                        Su[v].x += qr; Su[v].y += qi;
                        Sv[v].x = fmaf(dy, pr, Sv[v].x);
                        Sv[v].y = fmaf(dy, pi, Sv[v].y);
                    }
                }
            }

            // ---- epilogue: visibility half of the ramp, residuals, sums ----
            // With T = T0, Px = i pi Tu, Py = i pi Tv (Tu, Tv in wavelengths),
            // el = -dL alpha^2, em = -dM alpha^2, the derivatives are
            // dV/dl_i = D (el T + Px), dV/dl_j = D (-el T + Px),
            // dV/dm_i = D (em T + Py), dV/dm_j = D (-em T + Py).  Every chi^2,
            // gradient and normal sum then follows from the weighted inner
            // products <X, Y> = Re(conj(X) Y) of R, T, Px, Py over the lane's
            // visibilities of the channel, and the channel's D and alpha^2
            // enter only as factors of moments summed over channels:
            //   chi^2 = sum <R,R>,  E0 = sum 2 D a2 <R,T>,  E1 = -sum 2 D <R,Px>,
            //   E2 = -sum 2 D <R,Py>,  A0 = sum 2 D^2 <Px,Px>,  A1 = .. <Py,Py>,
            //   A2 = .. <Px,Py>,  B1 = sum 2 D^2 a2 <T,Px>,  B2 = .. <T,Py>,
            //   C = sum 2 D^2 a2^2 <T,T>
            // (a2 = alpha^2 with decorrelation, else 0 and D = 1); the item's
            // fifteen sums are formed from them and (dL, dM) once per item.
            float D = 1.f, a2 = 0.f;
            if (a.decorrelation) {
                a2 = ch.alpha2;
                D = __expf(-0.5f * a2 * (dL * dL + dM * dM));
            }
            const float su = pi_f * du / ov;         // Q was accumulated with dx ov; Px = i pi Tu
            const float sv = pi_f * du;
            float rr = 0.f, rt = 0.f, rx = 0.f, ry = 0.f, tt = 0.f, tx = 0.f, ty = 0.f, xx = 0.f, xy = 0.f, yy = 0.f;
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                float s, co;
                __sincosf(parg[v], &s, &co);
                const float2 ph = make_float2(co, s);
                const float2 T = cmul(ph, S0[v]);
                const float2 U = cmul(ph, Su[v]), W2 = cmul(ph, Sv[v]);
                const float2 Px = make_float2(-su * U.y, su * U.x);
                const float2 Py = make_float2(-sv * W2.y, sv * W2.x);
                const float w = wk[v];
                const float2 R = make_float2(fmaf(-D, T.x, vo[v].x), fmaf(-D, T.y, vo[v].y));
                const float2 wR = make_float2(w * R.x, w * R.y);
                const float2 wT = make_float2(w * T.x, w * T.y);
                const float2 wX = make_float2(w * Px.x, w * Px.y);
                // the ten inner products as five packed pairs
                {
                    float2 p;
                    p = ffma2(make_float2(wR.y, wR.y), make_float2(R.y, T.y), ffma2(make_float2(wR.x, wR.x), make_float2(R.x, T.x), make_float2(rr, rt)));
                    rr = p.x; rt = p.y;
                    p = ffma2(make_float2(wR.y, wR.y), make_float2(Px.y, Py.y), ffma2(make_float2(wR.x, wR.x), make_float2(Px.x, Py.x), make_float2(rx, ry)));
                    rx = p.x; ry = p.y;
                    p = ffma2(make_float2(wT.y, wT.y), make_float2(T.y, Px.y), ffma2(make_float2(wT.x, wT.x), make_float2(T.x, Px.x), make_float2(tt, tx)));
                    tt = p.x; tx = p.y;
                    p = ffma2(make_float2(wT.y, wX.y), make_float2(Py.y, Py.y), ffma2(make_float2(wT.x, wX.x), make_float2(Py.x, Py.x), make_float2(ty, xy)));
                    ty = p.x; xy = p.y;
                    p = ffma2(make_float2(wX.y, w * Py.y), make_float2(Px.y, Py.y), ffma2(make_float2(wX.x, w * Py.x), make_float2(Px.x, Py.x), make_float2(xx, yy)));
                    xx = p.x; yy = p.y;
                }
            }
            const float d2 = 2.f * D, dd2 = d2 * D;
            {
                float ms, mc;
                ms = mom[0][lane]; mc = mom[1][lane]; two_sum_acc(ms, mc, rr); mom[0][lane] = ms; mom[1][lane] = mc;
                ms = mom[2][lane]; mc = mom[3][lane]; two_sum_acc(ms, mc, d2 * a2 * rt); mom[2][lane] = ms; mom[3][lane] = mc;
                ms = mom[4][lane]; mc = mom[5][lane]; two_sum_acc(ms, mc, -d2 * rx); mom[4][lane] = ms; mom[5][lane] = mc;
                ms = mom[6][lane]; mc = mom[7][lane]; two_sum_acc(ms, mc, -d2 * ry); mom[6][lane] = ms; mom[7][lane] = mc;
                mom[8][lane] = fmaf(dd2, xx, mom[8][lane]);
                mom[9][lane] = fmaf(dd2, yy, mom[9][lane]);
                mom[10][lane] = fmaf(dd2, xy, mom[10][lane]);
                mom[11][lane] = fmaf(dd2 * a2, tx, mom[11][lane]);
                mom[12][lane] = fmaf(dd2 * a2, ty, mom[12][lane]);
                mom[13][lane] = fmaf(dd2 * a2 * a2, tt, mom[13][lane]);
            }
            ch = chn;
            box = boxn;
        }
        if (!ok) {
            // a wait ran out: report it, wait (longer bound) for this warp's own
            // copies still in flight, and stop
            if (lane == 0) atomicExch(a.err, 1);
            for (int bb = 0; bb < 2; ++bb)
                if (pending & (1u << bb)) mbar_wait(bb ? mb1 : mb0, (par >> bb) & 1u, kDrainPolls);
            __syncwarp();
            return;
        }
        // ---- the item's record: butterfly over the warp, then the fifteen sums in FP64 ----
        float cmp[4][2] = {{mom[0][lane], mom[1][lane]}, {mom[2][lane], mom[3][lane]}, {mom[4][lane], mom[5][lane]},
                           {mom[6][lane], mom[7][lane]}};
        float pln[6] = {mom[8][lane], mom[9][lane], mom[10][lane], mom[11][lane], mom[12][lane], mom[13][lane]};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float so = __shfl_xor_sync(kFull, cmp[k][0], o);
                const float co = __shfl_xor_sync(kFull, cmp[k][1], o);
                float cs = 0.f;
                two_sum_acc(cmp[k][0], cs, so);
                cmp[k][1] = __fadd_rn(__fadd_rn(cmp[k][1], co), cs);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) pln[k] += __shfl_xor_sync(kFull, pln[k], o);
        }
        const double chi2 = (double)cmp[0][0] + (double)cmp[0][1];
        const double E0 = (double)cmp[1][0] + (double)cmp[1][1];
        const double E1 = (double)cmp[2][0] + (double)cmp[2][1];
        const double E2 = (double)cmp[3][0] + (double)cmp[3][1];
        const double A0 = pln[0], A1 = pln[1], A2 = pln[2], B1 = pln[3], B2 = pln[4], C = pln[5];
        const double xl = dL, xm = dM;
        double out;
        switch (lane) {
            case 0: out = chi2; break;
            case 1: out = xl * E0 + E1; break;                                  // g l_i
            case 2: out = xm * E0 + E2; break;                                  // g m_i
            case 3: out = -xl * E0 + E1; break;                                 // g l_j
            case 4: out = -xm * E0 + E2; break;                                 // g m_j
            case 5: out = xl * xl * C - 2.0 * xl * B1 + A0; break;              // l_i l_i
            case 6: out = xl * xm * C - xl * B2 - xm * B1 + A2; break;          // l_i m_i
            case 7: out = xm * xm * C - 2.0 * xm * B2 + A1; break;              // m_i m_i
            case 8: out = xl * xl * C + 2.0 * xl * B1 + A0; break;              // l_j l_j
            case 9: out = xl * xm * C + xl * B2 + xm * B1 + A2; break;          // l_j m_j
            case 10: out = xm * xm * C + 2.0 * xm * B2 + A1; break;             // m_j m_j
            case 11: out = A0 - xl * xl * C; break;                             // l_i l_j
            case 12: out = -xl * B2 + xm * B1 - xl * xm * C + A2; break;        // l_i m_j
            case 13: out = xl * B2 - xm * B1 - xl * xm * C + A2; break;         // m_i l_j
            case 14: out = A1 - xm * xm * C; break;                             // m_i m_j
            default: out = 0.0;
        }
        if (lane < kRed) a.partials[(size_t)lane * a.n_bricks + brick] = out;
    }
}

// (intercept, slope) tables of every channel at a common stride, zero padded:
// entry n of channel c is (A°(n) - n s_n, s_n) with s_n = A°(n+1) - A°(n).
__global__ void track_tables_kernel(const ChanConst *__restrict__ chan, const float2 *__restrict__ tabs, int nc,
                                    int stride, float2 *__restrict__ out) {
    const size_t total = (size_t)nc * stride;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(k / stride), n = (int)(k - (size_t)c * stride);
        float2 v = make_float2(0.f, 0.f);
        if (n < chan[c].tab_len) {
            const float2 e = tabs[chan[c].tab_off + n];
            v = make_float2(fmaf(-(float)n, e.y, e.x), e.y);
        }
        out[k] = v;
    }
}

}  // namespace

size_t track_dyn_smem(int cap, int tabc) {
    return (size_t)kTrkWarps * 2 * (size_t)(cap + tabc) * sizeof(float2) + 128;    // + alignment slack
}

cudaError_t set_track_smem(size_t dyn) {
    for (const void *k : {(const void *)track_kernel<1>, (const void *)track_kernel<2>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t track_occupancy(int kv, size_t dyn, int *blocks_per_sm) {
    if (kv == 2)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<2>, kTrkThreads, dyn);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<1>, kTrkThreads, dyn);
}

cudaError_t launch_track(const EvalArgs &a, cudaStream_t s) {
    const int cap = a.trk_cap, tabc = a.trk_tabc;
    const size_t dyn = track_dyn_smem(cap, tabc);
    cudaError_t e = set_track_smem(dyn);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, n_sm = 0;
    e = track_occupancy(a.trk_kv, dyn, &per_sm);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long need = (a.n_bricks + kTrkWarps - 1) / kTrkWarps;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)std::max(1, per_sm) * n_sm));
    if (a.trk_kv == 2) track_kernel<2><<<grid, kTrkThreads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr, cap, tabc);
    else track_kernel<1><<<grid, kTrkThreads, dyn, s>>>(a, nullptr, nullptr, 0, nullptr, cap, tabc);
    return cudaGetLastError();
}

cudaError_t launch_track_batch(const EvalArgs *args_dev, const long long *prefix_dev, int n_ctx,
                               unsigned long long *queue, int kv, int cap, int tabc, int grid, cudaStream_t s) {
    EvalArgs none{};
    const size_t dyn = track_dyn_smem(cap, tabc);
    if (kv == 2) track_kernel<2><<<grid, kTrkThreads, dyn, s>>>(none, args_dev, prefix_dev, n_ctx, queue, cap, tabc);
    else track_kernel<1><<<grid, kTrkThreads, dyn, s>>>(none, args_dev, prefix_dev, n_ctx, queue, cap, tabc);
    return cudaGetLastError();
}

cudaError_t launch_track_tables(const ChanConst *chan, const float2 *tabs, int nc, int stride, float2 *out,
                                cudaStream_t s) {
    const size_t total = (size_t)nc * stride;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 1024);
    track_tables_kernel<<<blocks, 256, 0, s>>>(chan, tabs, nc, stride, out);
    return cudaGetLastError();
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
}

// Three tensor maps over the complex64 grid [ng][ng] viewed as 8-byte cells:
// boxes of 8, 16 and 32 cells by 8 rows, zero fill outside the grid.
cudaError_t make_grid_maps(const float2 *grid, int ng, void *maps_dev, cudaStream_t s) {
    if (((uintptr_t)grid & 15) || ng % 2) return cudaErrorInvalidValue;
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    CUtensorMap maps[3];
    const int widths[3] = {8, 16, 32};
    for (int k = 0; k < 3; ++k) {
        const cuuint64_t dims[2] = {(cuuint64_t)ng, (cuuint64_t)ng};
        const cuuint64_t strides[1] = {(cuuint64_t)ng * 8};
        const cuuint32_t box[2] = {(cuuint32_t)widths[k], (cuuint32_t)kBoxRows};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = fn(&maps[k], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<float2 *>(grid), dims, strides,
                              box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaMemcpyAsync(maps_dev, maps, sizeof(maps), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace psc

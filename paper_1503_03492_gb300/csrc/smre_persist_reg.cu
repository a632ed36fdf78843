// Persistent cooperative kernel of the standard Dykstra path with the band of
// x held in registers (sm_103a).
//
// The launch runs the whole projection (Sec. 2.3, Algorithm 2) on the same
// per-CTA schedule as the shared-memory band kernel (smre_persist.cu): for
// each side L a CTA owns a band of window-rows ("units") for all offsets a,
// the band slides down one row from offset a to a + 1, and one grid barrier
// per cycle gathers the FP64 norms of the stopping test.  What differs is the
// mapping of pixels to threads and the way data leaves the SM:
//
//  - lane l of consumer warp w owns the image columns c = 64 w + 2 l and
//    c + 1 for the whole launch, and holds those two columns of every band row
//    in registers (at most kRegRows rows).  A pass (L, a, b) therefore never
//    moves x: each lane forms y = x + q, the FP32 column sums of y^2 (rows in
//    order, both columns at once with the FP32x2 operations), and the only
//    data that crosses lanes are the column sums, through a shared-memory
//    array double-buffered by pass parity -- one CTA barrier per pass;
//  - every lane then adds the L column sums of its window in column order
//    (the same additions, in the same order, as every other schedule of this
//    library), takes the ball test, keeps y * scale in its registers and
//    writes y - x over the increments it read in the shared-memory stage;
//  - increments stream through a ring of stages: a producer warp fills a
//    stage with bulk async copies (TMA engine) up to the ring depth ahead,
//    and a storer warp copies each consumed stage back to its plane with bulk
//    stores, so no SM store instruction touches the increment stream;
//  - at an offset transition each warp hands its 64 columns of the band's
//    top row to the same warp of the upper neighbour as 64-bit words
//    (value, tag): the receiving warp polls the words until their tag is the
//    current cycle's, so the transition needs no flag and no memory fence.
//    The flags that later sides wait on are released once per side, after
//    the band is stored.
//
// Windows whose FP32 sum lies within 1e-6 of the bound are summed again in
// FP64: the warps of such a window publish FP64 column sums in shared memory
// and meet the neighbour warp through a per-warp flag.  Every wait is
// time-limited; on expiry the kernel records SMRE_ETIMEOUT, every warp leaves
// at the next barrier, and the context stays usable.
#include <cuda_runtime.h>

#include <cstdint>

#include "smre_internal.h"
#include "smre_ptx.cuh"

namespace smre {

namespace {

constexpr float kNearBand = 1e-6f;
constexpr unsigned kFull = 0xffffffffu;

// ---- shared memory by 32-bit address (explicit ld/st.shared)

__device__ __forceinline__ float2 lds2(unsigned a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ float lds1(unsigned a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void sts2(unsigned a, float2 v)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

__device__ __forceinline__ double ldsd(unsigned a)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void stsd2(unsigned a, double x, double y)
{
    asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(x), "d"(y) : "memory");
}

__device__ __forceinline__ void mbar_arrive_a(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_a(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_try_sleep_a(unsigned bar, unsigned parity, unsigned ns)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// ---- global memory helpers

__device__ __forceinline__ float2 ldcg2(const float *p)
{
    return __ldcg(reinterpret_cast<const float2 *>(p));
}

__device__ __forceinline__ void st_relaxed_v2(unsigned long long *p, unsigned long long a,
                                              unsigned long long b)
{
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long *p, unsigned long long &a,
                                              unsigned long long &b)
{
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ void st_relaxed_u32(unsigned *p, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void cta_sync_all() { asm volatile("barrier.sync 0;" ::: "memory"); }

// ---- time-limited waits (slow paths out of line)

__device__ __noinline__ void raise_timeout(const PersistArgs &A)
{
    atomicCAS(&A.ctl->status, (int)SMRE_OK, (int)SMRE_ETIMEOUT);
    atomicExch(A.abort_word, 1);
}

// One thread: wait until *p >= target (acquire), or time out / see an abort.
__device__ __noinline__ bool wait_geq(const PersistArgs &A, const unsigned *p, unsigned target)
{
    if (ld_acquire(p) >= target) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 0;; ++it) {
        if (ld_acquire(p) >= target) return true;
        if (it >= 4) __nanosleep(32);
        if ((it & 31) == 31) {
            if (ld_volatile(A.abort_word)) return false;
            if (globaltimer() - t0 > A.timeout_ns) {
                raise_timeout(A);
                return false;
            }
        }
    }
}

__device__ __noinline__ bool mbar_wait_slow(const PersistArgs &A, unsigned bar, unsigned parity)
{
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_sleep_a(bar, parity, 20000u)) return true;
        if (ld_volatile(A.abort_word)) return false;
        if (globaltimer() - t0 > A.timeout_ns) {
            raise_timeout(A);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait_timed(const PersistArgs &A, unsigned bar, unsigned parity)
{
    if (mbar_try_a(bar, parity)) return true;
    return mbar_wait_slow(A, bar, parity);
}

// Lane 0 of a warp waits for a shared-memory flag of another warp of the CTA
// (a volatile read of a monotone tag).
__device__ __noinline__ bool wait_smem_geq(const PersistArgs &A, const volatile unsigned *p,
                                           unsigned target)
{
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 0;; ++it) {
        if (*p >= target) return true;
        if ((it & 63) == 63) {
            if (ld_volatile(A.abort_word)) return false;
            if (globaltimer() - t0 > A.timeout_ns) {
                raise_timeout(A);
                return false;
            }
        }
    }
}

// The warp takes row words published by the same warp of another CTA: every
// lane polls its two 64-bit words until both carry `tag`.  Returns the two
// values in x, y and 1 in z, or z = 0 on time-out or abort.
__device__ __noinline__ float3 take_tagged(const PersistArgs &A, const unsigned long long *w,
                                           unsigned tag, bool lane_ok)
{
    bool ok = !lane_ok;
    float2 v = make_float2(0.f, 0.f);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        if (!ok) {
            unsigned long long a, b;
            ld_relaxed_v2(w, a, b);
            if ((unsigned)(a >> 32) == tag && (unsigned)(b >> 32) == tag) {
                v = make_float2(__uint_as_float((unsigned)a), __uint_as_float((unsigned)b));
                ok = true;
            }
        }
        if (__all_sync(kFull, ok)) return make_float3(v.x, v.y, 1.f);
        if (it == 0) t0 = globaltimer();
        __nanosleep(20);
        if ((it & 15) == 15) {
            const bool give_up = ld_volatile(A.abort_word) != 0 || globaltimer() - t0 > A.timeout_ns;
            if (__any_sync(kFull, give_up)) {
                if ((threadIdx.x & 31) == 0 && !ld_volatile(A.abort_word)) raise_timeout(A);
                return make_float3(v.x, v.y, 0.f);
            }
        }
    }
}

// Rare path of one unit: FP64 sums of the windows near the boundary.  The
// warps of such a window see it alike (same FP32 sum), publish FP64 column
// sums of their columns (r64: the unit's row of FP64 column sums) and meet
// the neighbour warp holding the window's other columns.  Returns the scales
// of the lane's two columns in x, y and 0 in z when a wait was lost.
template <int L>
__device__ __noinline__ float3 near_scales(const PersistArgs &A, unsigned r64, unsigned *near_tag,
                                           int warp, int lane, int pitch, int c0, bool lane_ok,
                                           double c64x, double c64y, unsigned tag, bool nr0,
                                           bool nr1, int s0, int s1, double cS64, float sc0,
                                           float sc1)
{
    if (lane_ok) stsd2(r64 + (unsigned)c0 * 8u, c64x, c64y);
    __syncwarp();
    __threadfence_block();
    const int wc0 = 64 * warp, wc1 = min(wc0 + 64, pitch);
    const bool need_l = __any_sync(kFull, (nr0 && s0 < wc0) || (nr1 && s1 < wc0));
    const bool need_r = __any_sync(kFull, (nr0 && s0 + L > wc1) || (nr1 && s1 + L > wc1));
    bool ok = true;
    if (lane == 0) {
        *(volatile unsigned *)(near_tag + warp) = tag;
        if (need_l) ok = wait_smem_geq(A, near_tag + warp - 1, tag);
        if (ok && need_r) ok = wait_smem_geq(A, near_tag + warp + 1, tag);
    }
    ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
    __syncwarp();
    __threadfence_block();
    if (!ok) return make_float3(sc0, sc1, 0.f);
    if (nr0) {
        double t64 = ldsd(r64 + (unsigned)s0 * 8u);
#pragma unroll
        for (int m = 1; m < L; ++m) t64 += ldsd(r64 + (unsigned)(s0 + m) * 8u);
        sc0 = t64 > cS64 ? (float)sqrt(cS64 / t64) : 1.f;
    }
    if (nr1) {
        double t64 = ldsd(r64 + (unsigned)s1 * 8u);
#pragma unroll
        for (int m = 1; m < L; ++m) t64 += ldsd(r64 + (unsigned)(s1 + m) * 8u);
        sc1 = t64 > cS64 ? (float)sqrt(cS64 / t64) : 1.f;
    }
    return make_float3(sc0, sc1, 1.f);
}

struct RegTask {
    int U;             // units present at this offset (band rows 0 .. U*L-1 take part)
    int pass0;         // q offset entry of pass b = 0
    float cS, sqrt_cS;
    double cS64;
};

struct RegCtx {
    const PersistArgs *A;
    unsigned full, written;     // shared addresses of the mbarrier arrays
    unsigned stage;             // shared address of stage 0
    unsigned stage_bytes;
    unsigned cs32, cs64;        // shared addresses of the column-sum arrays
    unsigned cs_half;           // bytes of one FP32 column-sum buffer
    unsigned *near_tag;         // [warps] last near-window tag each warp published
    volatile int *abort_cta;    // set (never cleared) when a warp of the CTA lost a wait
    int S, NC, warp, lane, pitch, W, c0;
    bool lane_ok;               // c0 < pitch
};

// Pass barrier of the consumer warps; returns true when any of them lost a
// wait (a sticky shared flag, written before the barrier and read after it).
__device__ __forceinline__ bool pass_barrier(const RegCtx &cx, bool bad)
{
    if (bad && cx.lane == 0) *cx.abort_cta = 1;
    named_sync(1, cx.NC);
    return *cx.abort_cta != 0;
}

// Side 1, rare path: the FP64 ball test of single-pixel windows near the
// boundary.  Out of line, so that none of its FP64 work is scheduled on the
// common path (FP64 runs at a small fraction of the FP32 rate on this part).
__device__ __noinline__ float2 near_scales1(float2 y, bool nr0, bool nr1, double cS64, float sc0,
                                            float sc1)
{
    if (nr0) {
        const double t64 = fma((double)y.x, (double)y.x, 0.0);
        sc0 = t64 > cS64 ? (float)sqrt(cS64 / t64) : 1.f;
    }
    if (nr1) {
        const double t64 = fma((double)y.y, (double)y.y, 0.0);
        sc1 = t64 > cS64 ? (float)sqrt(cS64 / t64) : 1.f;
    }
    return make_float2(sc0, sc1);
}

// Side 1: every window is one pixel, so the pass needs no exchange and no
// barrier.  A wait this warp missed stays in `lost` until the next barrier.
__device__ __forceinline__ void reg_task1(const RegCtx &cx, const RegTask &ts,
                                          float2 (&xr)[kRegRows], int &s_cur, unsigned &fph,
                                          unsigned &ptag, bool &lost)
{
    const PersistArgs &A = *cx.A;
    const unsigned rowb = (unsigned)cx.pitch * 4u;
    const int U = ts.U, c0 = cx.c0;
    const float cS = ts.cS, sqrt_cS = ts.sqrt_cS;
    const int s = s_cur;
    bool bad = lost;
    if (!bad) bad = !mbar_wait_timed(A, cx.full + 8u * s, (fph >> s) & 1u);
    bad = __any_sync(kFull, bad);
    fph ^= 1u << s;
    const unsigned stg = cx.stage + (unsigned)s * cx.stage_bytes + (unsigned)c0 * 4u;
    const bool work = !bad && cx.lane_ok;
    const bool in0 = work && c0 < cx.W;
    const bool in1 = work && c0 + 1 < cx.W;
#pragma unroll
    for (int u = 0; u < kRegRows; ++u) {
        if (u < U) {
            float2 y = xr[u];
            if (work) y = __fadd2_rn(y, lds2(stg + (unsigned)u * rowb));
            // window sum: 0 + y^2 rounded once, as in every schedule
            const float2 t = __ffma2_rn(y, y, make_float2(0.f, 0.f));
            float sc0 = 1.f, sc1 = 1.f;
            if (in0 && t.x > cS) sc0 = sqrt_cS * rsqrtf(t.x);
            if (in1 && t.y > cS) sc1 = sqrt_cS * rsqrtf(t.y);
            const bool nr0 = in0 && fabsf(t.x - cS) <= kNearBand * cS;
            const bool nr1 = in1 && fabsf(t.y - cS) <= kNearBand * cS;
            if (__any_sync(kFull, nr0 || nr1)) {
                const float2 r = near_scales1(y, nr0, nr1, ts.cS64, sc0, sc1);
                sc0 = r.x;
                sc1 = r.y;
            }
            if (work) {
                const float2 xn = __fmul2_rn(y, make_float2(sc0, sc1));
                if (in0) xr[u].x = xn.x;
                if (in1) xr[u].y = xn.y;
                sts2(stg + (unsigned)u * rowb, __fadd2_rn(y, make_float2(-xn.x, -xn.y)));
            }
        }
    }
    fence_proxy_async_smem();   // the new increments in the stage, for the bulk store
    __syncwarp();
    if (cx.lane == 0) mbar_arrive_a(cx.written + 8u * s);
    s_cur = s + 1 == cx.S ? 0 : s + 1;
    ++ptag;
    lost = lost || bad;
}

// The L passes b = 0..L-1 of one offset task, side L >= 2 known at compile
// time.  Returns true when the CTA must abandon the launch; `lost` says this
// warp already missed a wait (its work is skipped, it still meets every
// barrier).
template <int L>
__device__ __forceinline__ bool reg_task(const RegCtx &cx, const RegTask &ts,
                                         float2 (&xr)[kRegRows], int &s_cur, unsigned &fph,
                                         unsigned &ptag, bool &lost)
{
    constexpr int UM = kRegRows / L;          // units a band can hold
    const PersistArgs &A = *cx.A;
    const unsigned rowb = (unsigned)cx.pitch * 4u;
    const int U = ts.U, c0 = cx.c0;
    const float cS = ts.cS, sqrt_cS = ts.sqrt_cS;
#pragma unroll 1
    for (int b = 0; b < L; ++b) {
        const int s = s_cur;
        bool bad = lost;
        if (!bad) bad = !mbar_wait_timed(A, cx.full + 8u * s, (fph >> s) & 1u);
        bad = __any_sync(kFull, bad);
        fph ^= 1u << s;
        const unsigned stg = cx.stage + (unsigned)s * cx.stage_bytes + (unsigned)c0 * 4u;
        const unsigned csb = cx.cs32 + (ptag & 1u) * cx.cs_half;
        // windows of pass b cover the columns [b, b + nvL)
        const int nvL = cx.W - b >= L ? (cx.W - b) / L * L : 0;
        const int p0 = c0 - b;
        const bool work = !bad && cx.lane_ok;
        const bool in0 = work && p0 >= 0 && p0 < nvL;
        const bool in1 = work && p0 + 1 >= 0 && p0 + 1 < nvL;
        const int s0 = in0 ? c0 - p0 % L : 0;          // first column of each column's window
        const int s1 = in1 ? c0 + 1 - (p0 + 1) % L : 0;
        // y = x + q replaces x in the registers: columns outside every window
        // of the pass have q = 0 there (each cycle stores y - y * 1 = 0 for
        // them, the first cycle reads zeros), so y * 1 gives their x back
        if (work) {
#pragma unroll
            for (int u = 0; u < UM; ++u) {
                if (u < U) {
                    float2 cs = make_float2(0.f, 0.f);
#pragma unroll
                    for (int i = 0; i < L; ++i) {
                        xr[u * L + i] = __fadd2_rn(xr[u * L + i], lds2(stg + (unsigned)(u * L + i) * rowb));
                        cs = __ffma2_rn(xr[u * L + i], xr[u * L + i], cs);
                    }
                    sts2(csb + (unsigned)u * rowb + (unsigned)c0 * 4u, cs);
                }
            }
        }
        // every column sum of the pass is in shared memory; a copy lost
        // anywhere in the CTA abandons the launch here
        if (pass_barrier(cx, bad)) return true;
        // Each lane adds the column sums of the window of its first column.
        // The window of the second column is the same one, or it starts at
        // that column and then also holds the next lane's first column, whose
        // sum the next lane formed in the same order; only lane 31 forms it
        // itself (its next lane is in the next warp), when a window starts at
        // column 64 w + 63.
        const int c31 = 64 * cx.warp + 63 - b;
        const bool own31 = c31 >= 0 && c31 < nvL && c31 % L == 0;
#pragma unroll
        for (int u = 0; u < UM; ++u) {
            if (u < U) {
                const unsigned rb = csb + (unsigned)u * rowb;
                float v0[L];
#pragma unroll
                for (int m = 0; m < L; ++m) v0[m] = lds1(rb + (unsigned)(s0 + m) * 4u);
                float t0 = v0[0];
#pragma unroll
                for (int m = 1; m < L; ++m) t0 += v0[m];
                const float tn = __shfl_down_sync(kFull, t0, 1);
                float t1 = (in0 && s1 == s0) ? t0 : tn;
                if (own31) {
                    // warp-uniform: only lane 31's value is kept
                    float v1[L];
#pragma unroll
                    for (int m = 0; m < L; ++m) v1[m] = lds1(rb + (unsigned)(s1 + m) * 4u);
                    float t31 = v1[0];
#pragma unroll
                    for (int m = 1; m < L; ++m) t31 += v1[m];
                    if (cx.lane == 31) t1 = t31;
                }
                float sc0 = 1.f, sc1 = 1.f;
                const bool nr0 = in0 && fabsf(t0 - cS) <= kNearBand * cS;
                const bool nr1 = in1 && fabsf(t1 - cS) <= kNearBand * cS;
                if (in0 && t0 > cS) sc0 = sqrt_cS * rsqrtf(t0);
                if (in1 && t1 > cS) sc1 = sqrt_cS * rsqrtf(t1);
                if (__any_sync(kFull, nr0 || nr1)) {
                    double c64x = 0.0, c64y = 0.0;
                    if (work) {
#pragma unroll
                        for (int i = 0; i < L; ++i) {
                            c64x = fma((double)xr[u * L + i].x, (double)xr[u * L + i].x, c64x);
                            c64y = fma((double)xr[u * L + i].y, (double)xr[u * L + i].y, c64y);
                        }
                    }
                    const float3 r = near_scales<L>(
                        A, cx.cs64 + (unsigned)u * (unsigned)cx.pitch * 8u, cx.near_tag, cx.warp,
                        cx.lane, cx.pitch, c0, cx.lane_ok, c64x, c64y,
                        ptag * (unsigned)kRegRows + (unsigned)u + 1u, nr0, nr1, s0, s1, ts.cS64,
                        sc0, sc1);
                    sc0 = r.x;
                    sc1 = r.y;
                    if (r.z == 0.f) lost = true;
                }
                // x = y * scale stays in the registers (scale 1 outside the
                // windows); q = y - x over the stage (copied to the plane)
                if (work) {
                    const float2 sc = make_float2(sc0, sc1);
#pragma unroll
                    for (int i = 0; i < L; ++i) {
                        const float2 yv = xr[u * L + i];
                        const float2 xn = __fmul2_rn(yv, sc);
                        xr[u * L + i] = xn;
                        sts2(stg + (unsigned)(u * L + i) * rowb, __fadd2_rn(yv, make_float2(-xn.x, -xn.y)));
                    }
                }
            }
        }
        fence_proxy_async_smem();   // the new increments in the stage, for the bulk store
        __syncwarp();
        if (cx.lane == 0) mbar_arrive_a(cx.written + 8u * s);
        s_cur = s + 1 == cx.S ? 0 : s + 1;
        ++ptag;
        lost = lost || bad;
    }
    return false;
}

// Row r of the band (runtime index) as a register select.
__device__ __forceinline__ void set_row(float2 (&xr)[kRegRows], int r, float2 v)
{
#pragma unroll
    for (int k = 0; k < kRegRows; ++k)
        if (k == r) xr[k] = v;
}

// x_prev of the rows that a publication of band rows 0 .. n-1 (image rows
// r_first ..) makes final in the cycle, loaded ahead of the passes that end
// in that publication (bit k of `fin`: band row k is final).
template <int PF>
__device__ __forceinline__ void prefetch_prev(const PersistArgs &A, float2 (&pv)[PF], int r_first,
                                              int n, unsigned long long fin, int c0, bool lane_ok)
{
    if (!lane_ok || !fin) return;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int r = r_first + k;
        if (k < n && r < A.H && ((fin >> k) & 1ull))
            pv[k] = __ldcg(reinterpret_cast<const float2 *>(A.xprev + (size_t)r * A.pitch + c0));
    }
}

// Store band rows 0 .. n-1 to image rows r_first ..; rows whose bit is set in
// `fin` are final in the cycle: add their step and previous norm (FP64) and
// keep them as the next cycle's x_prev (taken from pv where PF covers the
// row, else loaded here).
template <int PF, bool USE_PV>
__device__ __forceinline__ void publish_rows(const PersistArgs &A, const float2 (&xr)[kRegRows],
                                             const float2 (&pv)[PF], int r_first, int n,
                                             unsigned long long fin, int c0, bool lane_ok,
                                             double &d2, double &n2)
{
    if (!lane_ok) return;
    const int pitch = A.pitch;
#pragma unroll
    for (int k = 0; k < kRegRows; ++k) {
        const int r = r_first + k;
        if (k < n && r < A.H) {
            const float2 v = xr[k];
            *reinterpret_cast<float2 *>(A.x + (size_t)r * pitch + c0) = v;
            if ((fin >> k) & 1ull) {
                float2 *pp = reinterpret_cast<float2 *>(A.xprev + (size_t)r * pitch + c0);
                const float2 pv_k = USE_PV && k < PF ? pv[k < PF ? k : 0] : __ldcg(pp);
                if (c0 < A.W) {
                    const double dd = (double)v.x - (double)pv_k.x;
                    d2 = fma(dd, dd, d2);
                    n2 = fma((double)pv_k.x, (double)pv_k.x, n2);
                }
                if (c0 + 1 < A.W) {
                    const double dd = (double)v.y - (double)pv_k.y;
                    d2 = fma(dd, dd, d2);
                    n2 = fma((double)pv_k.y, (double)pv_k.y, n2);
                }
                *pp = v;
            }
        }
    }
}

// What a consumer warp carries from one side to the next within a cycle.
struct CycState {
    double d2, n2;     // this thread's share of the cycle norm
    int s_cur;         // stage of the next pass
    unsigned fph;      // parity of the next `full` wait, per stage
    unsigned ptag;     // passes run so far (column-sum buffer parity, near tags)
    bool lost;         // this warp missed a wait
};

// Every offset a of one side for one consumer warp, after the side-start
// wait: the band comes in, slides down one row per offset (the top row goes
// to the upper neighbour, the lower neighbour's comes in), the passes of each
// offset run, and the band is stored at the end.  Returns true when the CTA
// must abandon the launch.  Side L is known at compile time, and the band's
// registers live only here.
template <int L>
__device__ __forceinline__ bool run_side(const RegCtx &cx, const SideS &sd, const GrpS *grps_s,
                                         unsigned want, unsigned tag, CycState &cs)
{
    const PersistArgs &A = *cx.A;
    const int band = sd.U * L, pitch = cx.pitch, c0 = cx.c0;
    const bool lane_ok = cx.lane_ok;
    float2 xr[kRegRows];
#pragma unroll
    for (int k = 0; k < kRegRows; ++k) xr[k] = make_float2(0.f, 0.f);
    if (!cs.lost && lane_ok) {
#pragma unroll
        for (int k = 0; k < kRegRows; ++k)
            if (k < band && sd.r0 + k < A.H) xr[k] = ldcg2(A.x + (size_t)(sd.r0 + k) * pitch + c0);
    }
    for (int a = 0; a < L; ++a) {
        const GrpS gp = grps_s[sd.grp0 + a];
        if (a > 0) {
            // the band slides down one row: drop the (published) top row,
            // take the lower neighbour warp's top row of offset a-1
#pragma unroll
            for (int k = 0; k + 1 < kRegRows; ++k)
                if (k + 1 < band) xr[k] = xr[k + 1];
            const int r = sd.r0 + a - 1 + band;
            if (!cs.lost && r < A.H) {
                float2 v = make_float2(0.f, 0.f);
                if (gp.nb_flag >= 0) {
                    const float3 t = take_tagged(A, A.xch + (size_t)gp.nb_flag * pitch + c0, tag, lane_ok);
                    v = make_float2(t.x, t.y);
                    if (t.z == 0.f) cs.lost = true;
                } else if (lane_ok) {
                    v = ldcg2(A.x + (size_t)r * pitch + c0);   // no task of this side wrote it
                }
                set_row(xr, band - 1, v);
            }
        }
        // x_prev of the rows this offset's publication makes final: loaded
        // now, used after the passes (side 1 only: it is the last side of a
        // cycle whenever the scale set holds it, and then every row becomes
        // final there)
        constexpr int PF = L == 1 ? kRegRows : 1;
        float2 pv[PF];
        const unsigned long long fin = a < L - 1 ? (unsigned long long)((sd.top_final >> a) & 1u)
                                                 : sd.end_final;
        if (L == 1 && !cs.lost) prefetch_prev<PF>(A, pv, sd.r0 + a, a < L - 1 ? 1 : band, fin, c0, lane_ok);
        if (gp.U > 0) {
            const RegTask rt{gp.U, sd.pass0 + a * L, sd.cS, sd.sqrt_cS, sd.cS64};
            bool ab;
            if (L == 1) {
                reg_task1(cx, rt, xr, cs.s_cur, cs.fph, cs.ptag, cs.lost);
                ab = false;
            } else {
                ab = reg_task<L == 1 ? 2 : L>(cx, rt, xr, cs.s_cur, cs.fph, cs.ptag, cs.lost);
            }
            if (ab) return true;
        }
        if (cs.lost) continue;
        if (a < L - 1) {
            // the top row leaves the band: to the image, and tagged to the
            // upper neighbour, which takes it at offset a + 1
            publish_rows<PF, (L == 1)>(A, xr, pv, sd.r0 + a, 1, fin, c0, lane_ok, cs.d2, cs.n2);
            if (lane_ok) {
                const unsigned long long tg = (unsigned long long)tag << 32;
                st_relaxed_v2(A.xch + (size_t)(sd.flag0 + a) * pitch + c0,
                              tg | __float_as_uint(xr[0].x), tg | __float_as_uint(xr[0].y));
            }
        } else {
            // side end: the whole band to the image, then the flags of every
            // event of the side (later sides wait on them)
            publish_rows<PF, (L == 1)>(A, xr, pv, sd.r0 + a, band, fin, c0, lane_ok, cs.d2, cs.n2);
            __syncwarp();
            if (cx.lane == 0) {
                __threadfence();
                const int NCW = A.consumer_warps;
                for (int e = 0; e < L; ++e)
                    st_relaxed_u32(A.flags + (size_t)(sd.flag0 + e) * NCW + cx.warp, want);
            }
        }
    }
    return false;
}

enum { kGo = 0, kStop = 1, kAbort = 2 };

// Cursor over the passes of one cycle that carry increments: (side, offset, pass).
struct Cur {
    int si, a, b;
};

__device__ __forceinline__ void cur_first(Cur &c, const SideS *sides_s, const GrpS *grps_s, int nside)
{
    c.si = 0;
    c.a = 0;
    c.b = 0;
    while (c.si < nside && grps_s[sides_s[c.si].grp0 + c.a].U == 0) {
        if (++c.a >= sides_s[c.si].L) {
            c.a = 0;
            ++c.si;
        }
    }
}

__device__ __forceinline__ void cur_next(Cur &c, const SideS *sides_s, const GrpS *grps_s, int nside)
{
    if (++c.b < sides_s[c.si].L) return;
    c.b = 0;
    for (;;) {
        if (++c.a >= sides_s[c.si].L) {
            c.a = 0;
            if (++c.si >= nside) return;
        }
        if (grps_s[sides_s[c.si].grp0 + c.a].U > 0) return;
    }
}

// ------------------------------------------------------------------ kernel
//
// Warps 0 .. NCW-1 consume (NCW = ceil(pitch / 64)); warp NCW produces and
// warp NCW + 1 stores; in both, lane 0 drives the bulk copies.
//   full[s]    completes when stage s holds the increments of its next pass
//              (U L rows of `pitch` floats; in the first cycle q = 0 and the
//              copies come from a zeroed block)
//   written[s] completes when every consumer warp wrote its new increments
//              into stage s
//   stored[s]  completes when the bulk stores of stage s have read it, so the
//              producer may refill it
// Flags in HBM are per (event, warp): flags[e * NCW + w] = cycle + 1 once
// warp w of the event's CTA stored its columns of the event's rows.
template <int NW>
__global__ void __launch_bounds__((NW + 2) * 32, 1) persist_reg_kernel(const __grid_constant__ PersistArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = A.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);              // [kMaxStages]
    uint64_t *written = full + kMaxStages;                            // [kMaxStages]
    uint64_t *stored = written + kMaxStages;                          // [kMaxStages]
    int *s_prov = reinterpret_cast<int *>(stored + kMaxStages);       // [kMaxStages]
    unsigned *near_tag = reinterpret_cast<unsigned *>(s_prov + kMaxStages);   // [kRegMaxWarps]
    unsigned char *tbl = smem + kRegHeaderBytes;                      // schedule
    float *stage0 = reinterpret_cast<float *>(smem + A.stage_offset); // [S][stage_floats]
    float *cs32 = stage0 + (size_t)S * A.stage_floats;                // [2][kRegRows/2][pitch]
    double *cs64 = reinterpret_cast<double *>(cs32 + (size_t)kRegRows * A.pitch);
    __shared__ int s_dec;
    __shared__ int s_abort;
    __shared__ double s_red[2][32];

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int NCW = A.consumer_warps, NC = NCW * 32;
    const int G = gridDim.x;
    const int pitch = A.pitch;
    __shared__ int s_cta;

    // Schedule index of this CTA: its rank among the SM ids of the launch
    // (one CTA per SM), so that neighbouring bands -- which hand rows to each
    // other at every offset -- run on SMs with neighbouring ids.
    if (tid == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        int rank = (int)blockIdx.x;
        A.smid_tab[blockIdx.x] = smid;
        __threadfence();
        atomicAdd(A.barrier + 16, 1u);
        if (wait_geq(A, A.barrier + 16, (unsigned)G)) {
            rank = 0;
            for (int i = 0; i < G; ++i) {
                const unsigned o = __ldcg(A.smid_tab + i);
                rank += o < smid || (o == smid && i < (int)blockIdx.x);
            }
        }
        s_cta = rank;
    }
    __syncthreads();
    const int cta = s_cta;

    {
        const int *hdr = reinterpret_cast<const int *>(A.sched + A.cta_off[cta]);
        const int nsd = hdr[0], ngr = hdr[1], npa = hdr[2], nde = hdr[3];
        const int n16 = (int)((16 + sizeof(SideS) * nsd + sizeof(GrpS) * ngr +
                               sizeof(long long) * npa + sizeof(int) * nde + 15) / 16);
        const int4 *src = reinterpret_cast<const int4 *>(hdr);
        int4 *dst = reinterpret_cast<int4 *>(tbl);
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    if (tid < kRegMaxWarps) near_tag[tid] = 0u;
    __syncthreads();
    const int nside = reinterpret_cast<const int *>(tbl)[0];
    const int ngrp = reinterpret_cast<const int *>(tbl)[1];
    const int npass_tab = reinterpret_cast<const int *>(tbl)[2];
    const SideS *sides_s = reinterpret_cast<const SideS *>(tbl + 16);
    const GrpS *grps_s = reinterpret_cast<const GrpS *>(sides_s + nside);
    const long long *pass_qoff = reinterpret_cast<const long long *>(grps_s + ngrp);
    const int *deps_s = reinterpret_cast<const int *>(pass_qoff + npass_tab);
    int npass = 0;
    for (int si = 0; si < nside; ++si)
        for (int a = 0; a < sides_s[si].L; ++a)
            if (grps_s[sides_s[si].grp0 + a].U > 0) npass += sides_s[si].L;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&written[s], (unsigned)NCW);
            mbar_init(&stored[s], 1);
            s_prov[s] = 0;
        }
        fence_mbar_init();
        s_dec = kGo;
        s_abort = 0;
    }
    __syncthreads();

    if (warp == NCW) {
        // ===================================================== producer warp
        bool dead = false;
        int s_head = 0;
        unsigned sph = 0;      // parity of the next `stored` wait, per stage
        for (int cyc = 0;; ++cyc) {
            const bool first = cyc == 0;
            if (lane == 0 && npass > 0 && !dead) {
                auto provide = [&](const Cur &c, int stg) {
                    s_prov[stg] += 1;
                    const SideS &sd = sides_s[c.si];
                    const int L = sd.L, U = grps_s[sd.grp0 + c.a].U;
                    const unsigned unit_bytes = (unsigned)(L * pitch * sizeof(float));
                    mbar_arrive_expect_tx(&full[stg], unit_bytes * U);
                    const float *src = first ? A.zeros : A.q + pass_qoff[sd.pass0 + c.a * L + c.b];
                    float *dst = stage0 + (size_t)stg * A.stage_floats;
                    for (int j = 0; j < U; ++j)
                        bulk_load(dst + (size_t)j * L * pitch, first ? src : src + (size_t)j * L * pitch,
                                  unit_bytes, &full[stg]);
                };
                // the stages of the cycle's first passes were stored (waited
                // for below) before the end of the previous cycle
                Cur rc;
                cur_first(rc, sides_s, grps_s, nside);
                int rs = s_head;
                const int pre = npass < S ? npass : S;
                for (int k = 0; k < pre; ++k) {
                    provide(rc, rs);
                    cur_next(rc, sides_s, grps_s, nside);
                    rs = rs + 1 == S ? 0 : rs + 1;
                }
                for (int p = 0; p < npass; ++p) {
                    // the storer has read stage s_head (pass p): refill it S passes ahead
                    if (!mbar_wait_timed(A, smem_u32(&stored[s_head]), (sph >> s_head) & 1u)) {
                        dead = true;
                        break;
                    }
                    sph ^= 1u << s_head;
                    if (p + S < npass) {
                        provide(rc, s_head);
                        cur_next(rc, sides_s, grps_s, nside);
                    }
                    s_head = s_head + 1 == S ? 0 : s_head + 1;
                }
            }
            __syncwarp();
            cta_sync_all();
            const int dec = s_dec;
            cta_sync_all();
            if (dec != kGo || dead) break;
        }
        if (lane == 0) {
            // let every load in flight land before the shared memory is released
            for (int s = 0; s < S; ++s) {
                if (s_prov[s] == 0) continue;
                const unsigned par = (unsigned)((s_prov[s] - 1) & 1);
                for (unsigned it = 0; !mbar_try_wait(&full[s], par) && it < (1u << 22); ++it) {
                }
            }
        }
        return;
    }

    if (warp == NCW + 1) {
        // ======================================================= storer warp
        bool dead = false;
        int s_tail = 0;
        unsigned wph = 0;      // parity of the next `written` wait, per stage
        for (int cyc = 0;; ++cyc) {
            if (lane == 0 && npass > 0 && !dead) {
                Cur c;
                cur_first(c, sides_s, grps_s, nside);
                for (int p = 0; p < npass; ++p) {
                    if (!mbar_wait_timed(A, smem_u32(&written[s_tail]), (wph >> s_tail) & 1u)) {
                        dead = true;
                        break;
                    }
                    wph ^= 1u << s_tail;
                    const SideS &sd = sides_s[c.si];
                    const int L = sd.L, U = grps_s[sd.grp0 + c.a].U;
                    const unsigned unit_bytes = (unsigned)(L * pitch * sizeof(float));
                    float *dst = A.q + pass_qoff[sd.pass0 + c.a * L + c.b];
                    const float *src = stage0 + (size_t)s_tail * A.stage_floats;
                    for (int j = 0; j < U; ++j)
                        bulk_store(dst + (size_t)j * L * pitch, src + (size_t)j * L * pitch, unit_bytes);
                    bulk_commit();
                    bulk_wait_read0();             // the stage may be refilled now
                    mbar_arrive(&stored[s_tail]);
                    cur_next(c, sides_s, grps_s, nside);
                    s_tail = s_tail + 1 == S ? 0 : s_tail + 1;
                }
                // this cycle's increments are in HBM before the next cycle loads them
                bulk_wait_all();
            }
            __syncwarp();
            cta_sync_all();
            const int dec = s_dec;
            cta_sync_all();
            if (dec != kGo || dead) break;
        }
        if (lane == 0) bulk_wait_all();
        return;
    }

    // ======================================================== consumer warps
    const int c0 = 64 * warp + 2 * lane;
    const bool lane_ok = c0 < pitch;
    const RegCtx cx{&A,
                    smem_u32(full),
                    smem_u32(written),
                    smem_u32(stage0),
                    (unsigned)A.stage_floats * 4u,
                    smem_u32(cs32),
                    smem_u32(cs64),
                    (unsigned)(kRegRows / 2) * (unsigned)pitch * 4u,
                    near_tag,
                    &s_abort,
                    S, NC, warp, lane, pitch, A.W, c0, lane_ok};
    CycState cs{0.0, 0.0, 0, 0u, 0u, false};
    bool aborted = false;
    bool &lost = cs.lost;

    for (int cyc = 0;; ++cyc) {
        const unsigned want = (unsigned)(cyc + 1);
        const unsigned tag = A.tag_base + want;
        for (int si = 0; si < nside && !aborted; ++si) {
            const SideS &sd = sides_s[si];
            // side start: wait for the same warp of the last publishers of the
            // band's rows (or a self-test flag nothing sets), one publisher a
            // lane, so flags already set cost one round trip, not one each;
            // the __syncwarp orders every lane's acquire before the band loads
            lost = __any_sync(kFull, lost);
            if (!lost) {
                int ok = 1;
                if (lane == 0 && A.selftest_timeout && cta == 0 && si == 0 && warp == 0)
                    ok = wait_geq(A, A.selftest_flag, 1u) ? 1 : 0;
                ok = __shfl_sync(kFull, ok, 0);
                for (int k0 = 0; ok && k0 < sd.dep_count; k0 += 32) {
                    const int k = k0 + lane;
                    const bool mine = k >= sd.dep_count ||
                                      wait_geq(A, A.flags + (size_t)deps_s[sd.dep_begin + k] * NCW + warp, want);
                    ok = __all_sync(kFull, mine) ? 1 : 0;
                }
                lost = !ok;
            }
            __syncwarp();
            // one dispatch per side: the band lives inside the side's own code
            switch (sd.L) {
#define RS(l) case l: aborted = run_side<l>(cx, sd, grps_s, want, tag, cs); break;
                RS(1) RS(2) RS(3) RS(4) RS(5) RS(6) RS(7) RS(8)
#undef RS
                default: aborted = true; break;
            }
        }

        // ---- end of cycle: publish norms, grid barrier, same decision everywhere
        int dec = kGo;
        if (!aborted) {
            double *slot = A.partials + (size_t)(cyc & 1) * 2 * G;   // double-buffered
            double sa = cs.d2, sb = cs.n2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sa += __shfl_xor_sync(kFull, sa, o);
                sb += __shfl_xor_sync(kFull, sb, o);
            }
            if (lane == 0) {
                s_red[0][warp] = sa;
                s_red[1][warp] = sb;
            }
            // a wait missed by any warp of the CTA ends the launch here
            if (named_sync_or(1, lost, NC)) aborted = true;
            bool late = false;
            if (!aborted && tid == 0) {
                double D = 0.0, N = 0.0;
                for (int w = 0; w < NCW; ++w) {
                    D += s_red[0][w];
                    N += s_red[1][w];
                }
                slot[2 * (size_t)cta] = D;
                slot[2 * (size_t)cta + 1] = N;
                __threadfence();
                atomicAdd(A.barrier, 1u);
                late = !wait_geq(A, A.barrier, (unsigned)G * want);
            }
            if (!aborted) late = named_sync_or(1, late, NC);
            cs.d2 = 0.0;
            cs.n2 = 0.0;
            if (aborted || late) {
                aborted = true;
            } else {
                double ra = 0.0, rb = 0.0;
                for (int i = tid; i < G; i += NC) {
                    ra += __ldcg(slot + 2 * (size_t)i);
                    rb += __ldcg(slot + 2 * (size_t)i + 1);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ra += __shfl_xor_sync(kFull, ra, o);
                    rb += __shfl_xor_sync(kFull, rb, o);
                }
                if (lane == 0) {   // thread 0 read s_red before the barrier above
                    s_red[0][warp] = ra;
                    s_red[1][warp] = rb;
                }
                named_sync(1, NC);
                double D = 0.0, N = 0.0;
                for (int w = 0; w < NCW; ++w) {
                    D += s_red[0][w];
                    N += s_red[1][w];
                }
                const double step = sqrt(D), prev = sqrt(N);
                // a NaN or Inf in x0 shows in the first cycle's norms (|x_prev| is
                // |x0| there); any non-finite norm ends the run with EINVAL
                const bool bad_in = !isfinite(step) || !isfinite(prev);
                const bool conv = !bad_in && A.tol >= 0.0 &&
                                  (A.tol_relative ? step <= A.tol * prev : step <= A.tol);
                const bool cap = cyc + 1 >= A.max_cycles;
                dec = (conv || cap || bad_in) ? kStop : kGo;
                if (cta == 0 && tid == 0) {
                    if (cyc < A.hist_cap) {
                        A.hist[2 * cyc] = step;
                        A.hist[2 * cyc + 1] = prev;
                    }
                    A.ctl->cycles = cyc + 1;
                    A.ctl->step = step;
                    A.ctl->prev_norm = prev;
                    if (dec == kStop) {
                        A.ctl->stop = 1;
                        if (bad_in)
                            atomicCAS(&A.ctl->status, (int)SMRE_OK, (int)SMRE_EINVAL);
                        else if (!conv && A.tol >= 0.0)
                            atomicCAS(&A.ctl->status, (int)SMRE_OK, (int)SMRE_ENOTCONVERGED);
                    }
                }
            }
        }
        if (aborted) dec = kAbort;
        if (tid == 0) s_dec = dec;
        cta_sync_all();
        cta_sync_all();
        if (dec != kGo) break;
    }
}

// Two builds: up to 8 consumer warps (pitch <= 512: ten warps, at most three
// per SM sub-partition, so a thread may take 168 registers) and up to 16
// (pitch <= 1024: eighteen warps, 96 registers a thread).
const void *reg_kernel_for(int threads)
{
    return threads <= 10 * 32 ? (const void *)persist_reg_kernel<8>
                              : (const void *)persist_reg_kernel<kRegMaxWarps>;
}

}  // namespace

bool persist_reg_fits(int pitch, int max_side, int max_band_rows)
{
    return pitch <= 64 * kRegMaxWarps && max_side >= 1 && max_side <= kRegRows &&
           max_band_rows <= kRegRows;
}

size_t persist_reg_exchange_bytes(int pitch)
{
    // FP32 column sums (two buffers of kRegRows / 2 rows) and FP64 column sums
    // (kRegRows / 2 rows)
    return (size_t)kRegRows * pitch * sizeof(float) + (size_t)(kRegRows / 2) * pitch * sizeof(double);
}

cudaError_t persist_reg_occupancy(int threads, size_t smem, int *blocks_per_sm)
{
    const void *k = reg_kernel_for(threads);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

cudaError_t launch_persist_reg(const PersistArgs &A, int grid, int threads, size_t smem,
                               cudaStream_t s)
{
    const void *k = reg_kernel_for(threads);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<PersistArgs *>(&A)};
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace smre

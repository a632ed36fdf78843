// Batched standard Dykstra path on sm_103a: the images of a batch (any mix of
// sizes up to 2048 columns) share every launch.
//
// Paper: Sec. 2.3 (Algorithm 2 with the projection p_s of Sec. 2.3) with the increment
// update of the Sec. 3.2 listing, applied set by set in the order sides
// descending, row offset a, column offset b.
//
// One cycle is one launch of the step kernel per group (L, a) -- the L
// tilings (L, a, b) share their window-rows ("units"), so a CTA that holds a
// unit runs its L passes b = 0..L-1 back to back -- followed by one launch of
// the norm kernel and one of the decide kernel.  Units of one group are
// disjoint, in one image and across images, so the step kernel treats the
// whole batch as one list of items: an item is k consecutive units of one
// image (k * pitch <= the kernel's virtual width), CTAs take items
// blockIdx.x, blockIdx.x + gridDim.x, ...
//
// Inside a CTA a producer warp streams each item's blocks -- the k L rows of
// x, then the increment block of every pass (and, for BF16/FP16 increments,
// the per-window scales) -- into a byte ring of shared memory with bulk
// asynchronous copies (TMA engine), as far ahead as the ring allows.  The 512
// consumer threads keep the item's x in registers (thread t owns the column
// pairs 2 (t + 512 j), FP32x2 arithmetic), form y = x + q and the column sums
// of y^2 in shared memory; after a barrier every consumer thread takes some
// of the pass's windows, sums their column sums in a fixed column order (the
// same order as the single-image kernels, so FP32 results agree bit for bit),
// takes the ball test and leaves the window's factors in shared memory; every
// column then applies its window's factors.  The new increments go back into
// the ring chunk, which a storer warp copies to HBM with bulk stores; x goes
// to HBM at the item's end.
//
// Mixed precision (BF16 / FP16 increments): each window's increment block is
// stored as q_s = sw * h with h in the 16-bit type and sw a power of two per
// window (FP32, in a scale plane beside the increments) chosen from the
// window's increment norm (1 - scale) sqrt(t) >= max |q_i|, so |h| <= 2^15
// fits FP16.  The update is consistent: x = y - sw * h, so x + sum_s q_s = x0
// holds for the stored increments up to FP32 rounding.
//
// Every wait has a time limit; on expiry the kernel records SMRE_ETIMEOUT,
// lets its copies in flight land and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "smre_internal.h"
#include "smre_ptx.cuh"

namespace smre {

namespace batch {

constexpr float kNearBand = 1e-6f;   // FP64 recheck band of the ball test, relative to cS
constexpr int kNC = kBatchConsumers;
constexpr int kNCW = kNC / 32;
constexpr int kD = kBatchDescs;
constexpr int kThreads = kNC + 64;   // consumers, producer warp, storer warp
constexpr int kNormThreads = 256;

// Element type of the stored increments: pairs of adjacent columns are
// loaded and stored together (8 bytes for FP32, 4 for BF16 / FP16); store2
// returns the stored values converted back to FP32 (before any scale).
template <typename QT>
struct QConv;
template <>
struct QConv<float> {
    static constexpr bool mixed = false;
    __device__ static float2 load2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    __device__ static float2 store2(float *p, float a, float b)
    {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
        return make_float2(a, b);
    }
};
template <>
struct QConv<__nv_bfloat16> {
    static constexpr bool mixed = true;
    __device__ static float2 load2(const __nv_bfloat16 *p)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    __device__ static float2 store2(__nv_bfloat16 *p, float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        *reinterpret_cast<__nv_bfloat162 *>(p) = h;
        return __bfloat1622float2(h);
    }
    // BF16 dequantisation takes the mixed-precision fma (FP32 result, BF16
    // operands): the stored pair is used as it is, with no widening step.
    // s packed as a bf16 pair (powers of two and zero convert exactly)
    __device__ static unsigned pack(float2 s)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(s.x, s.y);
        return *reinterpret_cast<const unsigned *>(&h);
    }
    // (h.x s.x + x.x, h.y s.y + x.y) with one rounding each, from the packed
    // bf16 pairs h and s: the products are exact in FP32, so this equals the
    // FP32 fma of the widened operands
    __device__ static float2 fma_packed(unsigned h, unsigned s, float2 x)
    {
        float2 r;
        asm("{\n\t.reg .b16 hl, hh, sl, sh;\n\t"
            "mov.b32 {hl, hh}, %2;\n\tmov.b32 {sl, sh}, %3;\n\t"
            "fma.rn.f32.bf16 %0, hl, sl, %4;\n\tfma.rn.f32.bf16 %1, hh, sh, %5;\n\t}"
            : "=f"(r.x), "=f"(r.y) : "r"(h), "r"(s), "f"(x.x), "f"(x.y));
        return r;
    }
    __device__ static float2 load_fma(const __nv_bfloat16 *p, float2, unsigned sb, float2 x)
    {
        return fma_packed(*reinterpret_cast<const unsigned *>(p), sb, x);
    }
    __device__ static float2 store_fma(__nv_bfloat16 *p, float2 v, float2, unsigned nswb, float2 y)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        const unsigned hb = *reinterpret_cast<const unsigned *>(&h);
        *reinterpret_cast<unsigned *>(p) = hb;
        return fma_packed(hb, nswb, y);
    }
};
template <>
struct QConv<__half> {
    static constexpr bool mixed = true;
    __device__ static float2 load2(const __half *p)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    __device__ static float2 store2(__half *p, float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b);
        *reinterpret_cast<__half2 *>(p) = h;
        return __half22float2(h);
    }
};

// Dequantising fma of the 16-bit types: y = h s + x and x = y - h sw from the
// stored pair h.  Types with a packed form (QConv::pack) take the scales as a
// packed pair as well; the others widen h and use the FP32x2 fma.
template <typename C, typename = void>
struct QFma {
    static constexpr bool packed = false;
    __device__ static unsigned pack(float2) { return 0u; }
    template <typename QT>
    __device__ static float2 load_fma(const QT *p, float2 s, unsigned, float2 x)
    {
        return __ffma2_rn(C::load2(p), s, x);
    }
    template <typename QT>
    __device__ static float2 store_fma(QT *p, float2 v, float2 nsw, unsigned, float2 y)
    {
        return __ffma2_rn(C::store2(p, v.x, v.y), nsw, y);
    }
};
template <typename C>
struct QFma<C, decltype((void)C::pack(float2{}))> {
    static constexpr bool packed = true;
    __device__ static unsigned pack(float2 s) { return C::pack(s); }
    template <typename QT>
    __device__ static float2 load_fma(const QT *p, float2 s, unsigned sb, float2 x)
    {
        return C::load_fma(p, s, sb, x);
    }
    template <typename QT>
    __device__ static float2 store_fma(QT *p, float2 v, float2 nsw, unsigned nswb, float2 y)
    {
        return C::store_fma(p, v, nsw, nswb, y);
    }
};

// Kernels are built for each side L <= 12 (compile-time L: the row loops
// unroll with fixed offsets) and once for sides 13..16 (run-time L <= 16).
__host__ __device__ constexpr int lb_of(int L) { return L <= 12 ? L : 16; }
// column pairs per consumer thread: x of an item takes 2 LB CPP registers
__host__ __device__ constexpr int cpp_of(int LB) { return LB == 2 ? 3 : 2; }
constexpr int kOutside = -(1 << 24);   // window index of a column outside the item
__host__ __device__ constexpr int vw_of(int LB) { return 2 * kNC * cpp_of(LB); }
__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }
__host__ __device__ constexpr int round128(int v) { return (v + 127) & ~127; }
// scale-plane row length of side L (windows per unit row, padded to 16 bytes)
__host__ __device__ constexpr int scale_row(int W, int L) { return ((W / L) + 3) & ~3; }

struct BItem {
    int slot, u0, nu;
};

// What the consumers need of an item, published by the producer with the
// item's x chunk (so the consumers never wait on the item tables in HBM);
// P < 0 marks the end of the CTA's items.
struct ChunkInfo {
    float *xrow;      // the item's first image row (x)
    unsigned *uflag;  // the image's window-row flags
    int P, W, nu, first;
    int u0;           // the item's first window-row
    unsigned tag;     // what its flags get once its rows are back in HBM
};

// 2^(k + shift) for the smallest k with v <= 2^k (exponent k in ex), read from
// the bits of v; 0 when v is zero, subnormal, not finite, or the power would
// leave the normal range (increments that small are stored as zero).
__device__ __forceinline__ float pow2_above(float v, int shift, int &ex)
{
    const unsigned u = __float_as_uint(v);
    const int be = (int)((u >> 23) & 0xffu);
    ex = be - 127 + ((u & 0x7fffffu) != 0u);   // v <= 2^ex
    const int r = ex + shift + 127;
    if (!(v > 0.f) || be == 0 || be == 255 || r < 1 || r > 254) return 0.f;
    return __uint_as_float((unsigned)r << 23);
}

// What the columns of a window need from the thread that took its window
// sum: the scale of the ball test (FP32 increments), or f = (1 - scale) / sw
// and the power-of-two sw (16-bit increments: q_i / sw = f y_i,
// x_i = y_i - sw h_i).
template <bool MIXED>
struct WinData;
template <>
struct WinData<false> {
    using type = float;
    __device__ static float none() { return 1.f; }
    __device__ static float scale(float d) { return d; }
    __device__ static float f(float) { return 0.f; }
    __device__ static float sw(float) { return 0.f; }
};
template <>
struct WinData<true> {
    using type = float2;
    __device__ static float2 none() { return make_float2(0.f, 0.f); }
    __device__ static float scale(float2) { return 1.f; }
    __device__ static float f(float2 d) { return d.x; }
    __device__ static float sw(float2 d) { return d.y; }
};

// Factors of one window from its sum of squares t: x = y * scale with
// scale = sqrt(cS / t) if t > cS (the projection p_s of Sec. 2.3); for 16-bit increments sw,
// a power of two with |q_i| / sw <= 2^15 from |q_i| <= (1 - scale) sqrt(t),
// and f = (1 - scale) / sw.  With `exact`, the FP64 sum t64 against cS64
// decides and gives the scale (the recheck of windows near the boundary).
template <bool MIXED>
__device__ __forceinline__ typename WinData<MIXED>::type window_factors(float t, float cS,
                                                                        float sqrt_cS, double t64,
                                                                        double cS64, bool exact)
{
    float scale = 1.f;
    if (exact) {
        if (t64 > cS64) scale = (float)sqrt(cS64 / t64);
    } else if (t > cS) {
        scale = sqrt_cS * rsqrtf(t);
    }
    if constexpr (!MIXED) {
        return scale;
    } else {
        float f = 0.f, sw = 0.f;
        const float qn = (1.f - scale) * (t * rsqrtf(t));
        int ex;
        const float s = pow2_above(qn, -14, ex);
        if (s > 0.f) {
            sw = s;
            f = (1.f - scale) * __uint_as_float((unsigned)(127 + 14 - ex) << 23);
        }
        return make_float2(f, sw);
    }
}

__device__ __forceinline__ int find_active(const int *prefix, int n_active, int item)
{
    // last active index i with prefix[i] <= item (images without items are skipped)
    int lo = 0, hi = n_active;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ BItem decode_item(const BStepArgs &A, const BGroup &G, int item)
{
    const int i = find_active(G.prefix, A.n_active, item);
    BItem it;
    it.slot = __ldg(A.active + i);
    const int k = __ldg(G.kpack + i);
    const int units = (A.imgs[it.slot].H - G.a) / A.L;
    it.u0 = (item - __ldg(G.prefix + i)) * k;
    it.nu = min(k, units - it.u0);
    return it;
}

// Bounded wait for an mbarrier phase.  On expiry (or when another CTA or
// role gave up) it records the time-out, raises the CTA's abort flag and
// returns false.
__device__ inline bool wait_phase(uint64_t *bar, unsigned parity, const BStepArgs &A,
                           volatile int *s_abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (*s_abort || ld_volatile(A.err)) break;
        if (globaltimer() - t0 > A.timeout_ns) {
            atomicCAS(A.err, 0, (int)SMRE_ETIMEOUT);
            break;
        }
    }
    *s_abort = 1;
    return false;
}

// Flag tag of group G in the cycle of an image: grows with every group run,
// so a flag at or above a group's tag says that group (or a later one) wrote
// the window-row back.
__device__ __forceinline__ unsigned group_tag(const BImage &im, const BGroup &G)
{
    return (unsigned)im.ctl->cycles * 256u + (unsigned)G.seq + 1u;
}

// Producer warp, several groups per launch: before an item's rows of x are
// loaded, the previous group's window-rows v0..v1 of the image (those that
// share rows with the item) must be back in HBM.  Lane k watches rows v0 + k,
// v0 + k + 32, ... (one round trip when they are done already).  Bounded: on
// expiry (or when another role gave up) it records the time-out, raises the
// abort flag and returns false, in every lane.
static __device__ __noinline__ bool wait_rows(const BStepArgs &A, const unsigned *uflag, int v0, int v1,
                                              unsigned tag, volatile int *s_abort)
{
    const int lane = threadIdx.x & 31;
    unsigned long long t0 = 0;
    for (int base = v0; base <= v1; base += 32) {
        const int v = base + lane;
        for (;;) {
            const bool ok = v > v1 || (int)(ld_acquire(uflag + v) - tag) >= 0;
            if (__all_sync(0xffffffffu, ok)) break;
            int give_up = 0;
            if (lane == 0) {
                const unsigned long long t = globaltimer();
                if (*s_abort || ld_volatile(A.err)) {
                    give_up = 1;
                } else if (t0 == 0) {
                    t0 = t;
                } else if (t - t0 > A.timeout_ns) {
                    atomicCAS(A.err, 0, (int)SMRE_ETIMEOUT);
                    give_up = 1;
                }
                if (give_up) *s_abort = 1;
            }
            if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
            __nanosleep(100);
        }
    }
    return true;
}

// Chunks in the ring have a fixed row stride: row i of an item's block sits at
// element i * VW of the chunk, and unit s of the item occupies columns
// s * pitch .. s * pitch + pitch - 1 of every row, so a consumer's column pair
// is at a compile-time offset in every row.  The producer and the storer move
// each (unit, row) of a block with its own bulk copy, spread over their lanes.

// Producer warp: walks the CTA's items in the consumers' order and fills the
// ring with, per item, the x block and one increment block per pass (plus the
// window scales of 16-bit increments).  In an image's first cycle the
// increments are zero: their blocks are only space for the consumers' results
// and nothing is read.  Lane 0 keeps the ring; every lane issues copies.
template <typename QT, int VW>
__device__ void produce(const BStepArgs &A, unsigned char *ring, uint64_t *full,
                        uint64_t *written, int *s_off, ChunkInfo *s_info, volatile int *s_abort)
{
    constexpr bool MIXED = QConv<QT>::mixed;
    constexpr int esz = (int)sizeof(QT);
    const int lane = threadIdx.x & 31;
    const int L = A.L;
    int head = 0, d_next = 0, d_tail = 0, n_out = 0;   // lane 0's view of the ring
    unsigned wph = 0;    // parity of the next `written` wait, per descriptor
    unsigned fiss = 0;   // toggled per issue: parity of the latest `full` phase, per descriptor
    bool dead = false;

    auto pop = [&]() -> bool {   // the oldest chunk was released
        if (!wait_phase(&written[d_tail], (wph >> d_tail) & 1u, A, s_abort)) return false;
        wph ^= 1u << d_tail;
        d_tail = d_tail + 1 == kD ? 0 : d_tail + 1;
        --n_out;
        return true;
    };
    // place n bytes in the ring: the free space runs from head to the start
    // of the oldest chunk still held, wrapping to 0 when the end is too close
    auto alloc = [&](int n, int &at) -> bool {
        for (;;) {
            if (n_out == 0) {
                at = 0;
                return true;
            }
            if (n_out < kD) {
                const int tail = s_off[d_tail];
                if (head > tail) {
                    if (head + n <= A.ring_bytes) { at = head; return true; }
                    if (n <= tail) { at = 0; return true; }
                } else if (head + n <= tail) {
                    at = head;
                    return true;
                }
            }
            if (!pop()) return false;
        }
    };
    // a chunk of n bytes whose copies will bring tx bytes (0: nothing is
    // copied); lane 0 places it and arms its barrier, all lanes learn where
    auto begin = [&](int n, unsigned tx, int &at, int &d, const ChunkInfo *info) -> bool {
        int ok = 1;
        at = 0;
        d = 0;
        if (lane == 0) {
            ok = alloc(round128(n), at) ? 1 : 0;
            if (ok) {
                s_off[d_next] = at;
                if (info) s_info[d_next] = *info;   // published by the arrive below
                if (tx) mbar_arrive_expect_tx(&full[d_next], tx);
                else mbar_arrive(&full[d_next]);
                fiss ^= 1u << d_next;
                head = at + round128(n);
                ++n_out;
                d = d_next;
                d_next = d_next + 1 == kD ? 0 : d_next + 1;
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        at = __shfl_sync(0xffffffffu, at, 0);
        d = __shfl_sync(0xffffffffu, d, 0);
        return ok != 0;
    };

    for (int g = 0; g < A.n_groups && !dead; ++g) {
        const BGroup G = A.groups[g];
        for (int item = blockIdx.x; item < G.n_items && !dead; item += gridDim.x) {
            const BItem it = decode_item(A, G, item);
            const BImage im = A.imgs[it.slot];
            if (im.ctl->stop) continue;
            const int P = im.pitch;
            const bool first = im.ctl->cycles == 0;
            const int rows = it.nu * L;   // row r = unit r / L, row r % L of it
            float *xsrc = im.x + (size_t)(G.a + L * it.u0) * P;
            const unsigned tag = group_tag(im, G);
            if (g > 0) {
                // group (L, a - 1) ran before in this launch: its window-rows
                // u0 .. u0 + nu hold this item's rows
                const int v1 = min(it.u0 + it.nu, (im.H - (G.a - 1)) / L - 1);
                if (!wait_rows(A, im.uflag, it.u0, v1, tag - 1u, s_abort)) {
                    dead = true;
                    break;
                }
                fence_proxy_async_global();   // the rows written by other CTAs, for the bulk loads
            }
            const ChunkInfo info{xsrc, im.uflag, P, im.W, it.nu, first ? 1 : 0, it.u0, tag};
            int at, d;
            if (!begin(L * VW * 4, (unsigned)(rows * P) * 4u, at, d, &info)) {
                dead = true;
                break;
            }
            for (int r = lane; r < rows; r += 32) {
                const int s = r / L, i = r - s * L;
                bulk_load(ring + at + (size_t)(i * VW + s * P) * 4, xsrc + (size_t)r * P,
                          (unsigned)P * 4u, &full[d]);
            }
            const int nwp = scale_row(im.W, L);
            const unsigned tx = first ? 0u
                                      : (unsigned)(rows * P * esz) + (MIXED ? (unsigned)(it.nu * nwp) * 4u : 0u);
            for (int b = 0; b < L; ++b) {
                if (!begin(L * VW * esz + (MIXED ? VW * 4 : 0), tx, at, d, nullptr)) {
                    dead = true;
                    break;
                }
                if (first) continue;
                const QT *qsrc = reinterpret_cast<const QT *>(im.q) + im.qoff[G.p0 + b] +
                                 (size_t)it.u0 * L * P;
                for (int r = lane; r < rows; r += 32) {
                    const int s = r / L, i = r - s * L;
                    bulk_load(ring + at + (size_t)(i * VW + s * P) * esz, qsrc + (size_t)r * P,
                              (unsigned)(P * esz), &full[d]);
                }
                if (MIXED && lane == 0)
                    bulk_load(ring + at + (size_t)L * VW * esz, im.qs + im.soff[G.p0 + b] + (size_t)it.u0 * nwp,
                              (unsigned)(it.nu * nwp) * 4u, &full[d]);
            }
        }
    }
    if (!dead) {   // the end marker: a chunk without data
        const ChunkInfo end{nullptr, nullptr, -1, 0, 0, 0, 0, 0u};
        int at, d;
        if (!begin(128, 0u, at, d, &end)) dead = true;
    }
    if (lane != 0) return;
    if (!dead) {
        while (n_out > 0)
            if (!pop()) { dead = true; break; }
    }
    if (dead) {
        // let every copy in flight land before the shared memory is released
        for (int k = 0, d = d_tail; k < n_out; ++k, d = d + 1 == kD ? 0 : d + 1) {
            const unsigned par = ((fiss >> d) & 1u) ^ 1u;
            for (unsigned it = 0; !mbar_try_wait(&full[d], par) && it < (1u << 22); ++it) {
            }
        }
    }
}

// Storer warp: once the consumers have written a pass's new increments (and
// scales) into its chunk, copies each (unit, row) of the chunk to the
// increment plane with bulk stores and releases the chunk to the producer
// when every copy has read it.
// Storer lane 0, several groups per launch: wait (bounded) until the
// consumer warps have counted `need` stored items of x in *xdone.
static __device__ __noinline__ bool wait_xdone(const BStepArgs &A, unsigned *xdone, unsigned need,
                                               volatile int *s_abort)
{
    unsigned long long t0 = 0;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(xdone)) : "memory");
        if ((int)(v - need) >= 0) return true;
        if (*s_abort || ld_volatile(A.err)) break;
        const unsigned long long t = globaltimer();
        if (t0 == 0) {
            t0 = t;
        } else if (t - t0 > A.timeout_ns) {
            atomicCAS(A.err, 0, (int)SMRE_ETIMEOUT);
            break;
        }
        __nanosleep(64);
    }
    *s_abort = 1;
    return false;
}

template <typename QT, int VW>
__device__ void store_back(const BStepArgs &A, unsigned char *ring, uint64_t *written,
                           uint64_t *ready, unsigned *xdone, const int *s_off, volatile int *s_abort)
{
    constexpr bool MIXED = QConv<QT>::mixed;
    constexpr int esz = (int)sizeof(QT);
    const int lane = threadIdx.x & 31;
    const int L = A.L;
    int ds = 0;
    unsigned rph = 0;   // parity of the next `ready` wait, per descriptor
    unsigned xneed = 0;   // consumer-warp counts in *xdone of the items published so far
    for (int g = 0; g < A.n_groups; ++g) {
        const BGroup G = A.groups[g];
        for (int item = blockIdx.x; item < G.n_items; item += gridDim.x) {
            const BItem it = decode_item(A, G, item);
            const BImage im = A.imgs[it.slot];
            if (im.ctl->stop) continue;
            const int P = im.pitch;
            const int nwp = scale_row(im.W, L);
            const int rows = it.nu * L;
            ds = ds + 1 == kD ? 0 : ds + 1;   // the x chunk: released by the consumers
            for (int b = 0; b < L; ++b) {
                int ok = 1;
                if (lane == 0) ok = wait_phase(&ready[ds], (rph >> ds) & 1u, A, s_abort) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    bulk_wait_all();
                    return;
                }
                rph ^= 1u << ds;
                const unsigned char *src = ring + s_off[ds];
                QT *qdst = reinterpret_cast<QT *>(im.q) + im.qoff[G.p0 + b] + (size_t)it.u0 * L * P;
                for (int r = lane; r < rows; r += 32) {
                    const int s = r / L, i = r - s * L;
                    bulk_store(qdst + (size_t)r * P, src + (size_t)(i * VW + s * P) * esz,
                               (unsigned)(P * esz));
                }
                if (MIXED && lane == 0)
                    bulk_store(im.qs + im.soff[G.p0 + b] + (size_t)it.u0 * nwp, src + (size_t)L * VW * esz,
                               (unsigned)(it.nu * nwp) * 4u);
                bulk_commit();
                bulk_wait_read0();
                __syncwarp();
                if (lane == 0) mbar_arrive_cnt(&written[ds], kNCW);
                ds = ds + 1 == kD ? 0 : ds + 1;
            }
            if (A.n_groups > 1) {
                // several groups in this launch: once the consumers have
                // stored the item's rows of x, its window-rows are released to
                // the next group's items (one GPU-scope fence, cumulative over
                // the consumers' stores seen through the count, then relaxed
                // flag stores; the producer that acquires a flag fences its own
                // proxy before the bulk loads)
                int ok = 1;
                xneed += kNCW;
                if (lane == 0) ok = wait_xdone(A, xdone, xneed, s_abort) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    bulk_wait_all();
                    return;
                }
                if (lane == 0) {
                    __threadfence();
                    const unsigned tag = group_tag(im, G);
                    for (int u = 0; u < it.nu; ++u) st_relaxed(im.uflag + it.u0 + u, tag);
                }
            }
        }
    }
    bulk_wait_all();
}

template <typename QT, int LB, bool EXACT>
__global__ void __launch_bounds__(kThreads, 1) bstep_kernel(const BStepArgs A)
{
    using C = QConv<QT>;
    using QF = QFma<C>;
    constexpr bool MIXED = C::mixed;
    constexpr int CPP = cpp_of(LB);
    constexpr int VW = vw_of(LB);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);   // [kD] chunk landed
    uint64_t *written = full + kD;                          // [kD] chunk free again
    uint64_t *ready = written + kD;                         // [kD] new increments in the chunk
    int *s_off = reinterpret_cast<int *>(ready + kD);       // [kD] ring offset of each chunk
    // per virtual column: the column sum of y^2, the FP64 recheck sums and,
    // at each window's first column, the window's factors (the scale of the
    // ball test; for 16-bit increments f = (1 - scale) / sw and sw instead)
    using WD = typename WinData<MIXED>::type;
    float *part = reinterpret_cast<float *>(smem + 256);            // [VW]
    double *part64 = reinterpret_cast<double *>(part + VW);         // [VW]
    WD *wdat = reinterpret_cast<WD *>(part64 + VW);                 // [VW]
    unsigned char *ring = smem + A.ring_offset;
    __shared__ volatile int s_abort;
    __shared__ ChunkInfo s_info[kD];
    __shared__ unsigned s_xdone;   // consumer warps that stored their rows of x, over all items
    unsigned *xdone = &s_xdone;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = EXACT ? LB : A.L;
    if (tid == 0) {
        for (int d = 0; d < kD; ++d) {
            mbar_init(&full[d], 1);
            mbar_init(&written[d], kNCW);
            mbar_init(&ready[d], kNCW);
            s_off[d] = 0;
        }
        *xdone = 0u;
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    if (warp == kNCW) {
        produce<QT, VW>(A, ring, full, written, s_off, s_info, &s_abort);
        return;
    }
    if (warp == kNCW + 1) {
        store_back<QT, VW>(A, ring, written, ready, xdone, s_off, &s_abort);
        return;
    }

    // ------------------------------------------------------------ consumers
    int dc = 0;          // descriptor of the next chunk
    unsigned fph = 0;    // parity of the next `full` wait, per descriptor
    const float cS = A.cS, sqrt_cS = A.sqrt_cS;
    for (;;) {
        // the next item's x chunk, with the item's description
        bool bad = !wait_phase(&full[dc], (fph >> dc) & 1u, A, &s_abort);
        fph ^= 1u << dc;
        if (named_sync_or(1, bad, kNC)) break;
        const ChunkInfo info = s_info[dc];
        if (info.P < 0) {   // no more items
            __syncwarp();
            if (lane == 0) mbar_arrive(&written[dc]);
            break;
        }
        const int P = info.P, W = info.W, nu = info.nu;
        const bool first = info.first != 0;
        const int nwp = scale_row(W, L);
        // Thread t owns the column pairs (c, c + 1), c = 2 (t + kNC j) mod P of
        // unit sj of the item.  o: row-0 offset of the pair in a chunk; po: its
        // column-sum slot; so: its unit's scale row; (vv, rr): window of column
        // c in the current pass and c's place in it, advanced each pass.
        // Columns outside the item get a window index that never lies in a pass.
        int og[CPP], so[CPP], vv[CPP], rr[CPP];
#pragma unroll
        for (int j = 0; j < CPP; ++j) {
            const int vc = 2 * (tid + kNC * j);
            const int sj = vc / P;
            const int c = vc - sj * P;
            og[j] = sj * L * P + c;   // row 0 of the pair in the image rows of the item
            so[j] = sj * nwp;
            vv[j] = sj < nu && c < W ? c / L : kOutside;
            rr[j] = c % L;
        }
        // this thread's first pair in a chunk row and in the column sums; pair j
        // and row i lie at the compile-time offset i VW + 2 kNC j from there
        const int vc0 = 2 * tid;

        // the item's rows of x into registers
        float2 x[LB][CPP];   // (column c, column c + 1); pairs use the FP32x2 arithmetic
        {
            const float *xb = reinterpret_cast<const float *>(ring + s_off[dc]) + vc0;
#pragma unroll
            for (int j = 0; j < CPP; ++j)
#pragma unroll
                for (int i = 0; i < LB; ++i) {
                    float2 v = make_float2(0.f, 0.f);
                    if (i < L && vv[j] >= 0 && !bad)
                        v = *reinterpret_cast<const float2 *>(xb + i * VW + 2 * kNC * j);
                    x[i][j] = v;
                }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&written[dc]);
        dc = dc + 1 == kD ? 0 : dc + 1;

        bool aborted = false;
        for (int b = 0; b < L; ++b) {
            const int nv = (W - b) / L;   // windows per unit row in this pass
            if (!bad) bad = !wait_phase(&full[dc], (fph >> dc) & 1u, A, &s_abort);
            fph ^= 1u << dc;
            unsigned char *chunk = ring + s_off[dc];
            QT *qc = reinterpret_cast<QT *>(chunk) + vc0;   // qc[i VW + 2 kNC j]: row i of pair j
            float *sc = reinterpret_cast<float *>(chunk + (size_t)L * VW * sizeof(QT));
            // windows of both columns of each pair
            int w1[CPP], r1[CPP];
            bool on[CPP][2];
#pragma unroll
            for (int j = 0; j < CPP; ++j) {
                r1[j] = rr[j] + 1 == L ? 0 : rr[j] + 1;
                w1[j] = rr[j] + 1 == L ? vv[j] + 1 : vv[j];
                on[j][0] = vv[j] >= 0 && vv[j] < nv;
                on[j][1] = w1[j] >= 0 && w1[j] < nv;
            }
            // y = x + q_s on the owned columns, and the column sums of y^2
#pragma unroll
            for (int j = 0; j < CPP; ++j) {
                if (!(on[j][0] || on[j][1]) || bad) continue;
                float2 s2 = make_float2(1.f, 1.f);   // dequantisation scales of the pair
                if (MIXED && !first) {
                    s2.x = on[j][0] ? sc[so[j] + vv[j]] : 0.f;
                    s2.y = on[j][1] ? sc[so[j] + w1[j]] : 0.f;
                }
                const unsigned s2b = QF::pack(s2);
                float2 sq = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < LB; ++i) {
                    if (i < L) {
                        if (!first) {
                            if constexpr (MIXED) {
                                x[i][j] = QF::load_fma(qc + i * VW + 2 * kNC * j, s2, s2b, x[i][j]);
                            } else {
                                const float2 qv = C::load2(qc + i * VW + 2 * kNC * j);
                                x[i][j] = __fadd2_rn(x[i][j], qv);
                            }
                        }
                        sq = __ffma2_rn(x[i][j], x[i][j], sq);
                    }
                }
                *reinterpret_cast<float2 *>(part + vc0 + 2 * kNC * j) = sq;
            }
            if (named_sync_or(1, bad, kNC)) {   // column sums complete (or a copy was lost)
                aborted = true;
                break;
            }

            // the consumers share out the pass's windows (nu rows of nv windows):
            // for each, sum the L column sums in column order, take the ball test
            // of the projection p_s (Sec. 2.3) and, for 16-bit increments, pick the window's
            // power-of-two scale sw with |q_i| / sw <= 2^15 (FP16 holds up to
            // 65504) from |q_i| <= |q_s|_2 = (1 - scale) sqrt(t); the factors go
            // to the window's first column, windows within the band of the test
            // are flagged for the FP64 recheck
            const int nwin = nu * nv;
            auto window_col = [&](int w) {   // virtual column of window w's first column
                const int s = nu == 1 ? 0 : w / nv;
                return s * P + b + (w - s * nv) * L;
            };
            auto window_sum = [&](int c0) {
                const float *pp = part + c0;
                float pv[LB];
#pragma unroll
                for (int m = 0; m < LB; ++m) pv[m] = m < L ? pp[m] : 0.f;
                float ts = 0.f;
#pragma unroll
                for (int m = 0; m < LB; ++m)
                    if (m < L) ts += pv[m];
                return ts;
            };
            bool near = false;
            for (int w = tid; w < nwin; w += kNC) {
                const int c0 = window_col(w);
                const float ts = window_sum(c0);
                if (fabsf(ts - cS) <= kNearBand * cS) near = true;
                wdat[c0] = window_factors<MIXED>(ts, cS, sqrt_cS, 0.0, 0.0, false);
            }
            if (named_sync_or(1, near, kNC)) {
                // rare: windows within the band get their sums again in FP64
#pragma unroll
                for (int j = 0; j < CPP; ++j)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        double s64 = 0.0;
                        if (on[j][e]) {
#pragma unroll
                            for (int i = 0; i < LB; ++i)
                                if (i < L) {
                                    const double v = e ? x[i][j].y : x[i][j].x;
                                    s64 = fma(v, v, s64);
                                }
                            part64[vc0 + 2 * kNC * j + e] = s64;
                        }
                    }
                named_sync(1, kNC);
                for (int w = tid; w < nwin; w += kNC) {
                    const int c0 = window_col(w);
                    if (fabsf(window_sum(c0) - cS) > kNearBand * cS) continue;
                    double t64 = 0.0;
                    for (int m = 0; m < L; ++m) t64 += part64[c0 + m];
                    wdat[c0] = window_factors<MIXED>((float)t64, cS, sqrt_cS, t64, A.cS64, true);
                }
                named_sync(1, kNC);
            }
            // every owned column takes its window's factors
            WD wf[CPP][2];
#pragma unroll
            for (int j = 0; j < CPP; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    wf[j][e] = on[j][e] ? wdat[vc0 + 2 * kNC * j + e - (e ? r1[j] : rr[j])]
                                        : WinData<MIXED>::none();

            // x = p_s(y), q_s = y - x; the new increments go into the chunk,
            // which the storer copies to the plane
#pragma unroll
            for (int j = 0; j < CPP; ++j) {
                if (!(on[j][0] || on[j][1])) continue;
                if (!MIXED) {
                    const float2 c2 = make_float2(WinData<MIXED>::scale(wf[j][0]),
                                                  WinData<MIXED>::scale(wf[j][1]));
#pragma unroll
                    for (int i = 0; i < LB; ++i)
                        if (i < L) {
                            const float2 y = x[i][j];
                            const float2 n = __fmul2_rn(y, c2);
                            x[i][j] = n;
                            const float2 q = __fadd2_rn(y, make_float2(-n.x, -n.y));
                            C::store2(qc + i * VW + 2 * kNC * j, q.x, q.y);
                        }
                } else {
                    // q_i / sw = y_i (1 - scale) / sw, rounded to the 16-bit type
                    const float2 f2 = make_float2(WinData<MIXED>::f(wf[j][0]), WinData<MIXED>::f(wf[j][1]));
                    const float sw0 = WinData<MIXED>::sw(wf[j][0]), sw1 = WinData<MIXED>::sw(wf[j][1]);
                    const float2 nsw = make_float2(-sw0, -sw1);
                    const unsigned nswb = QF::pack(nsw);
#pragma unroll
                    for (int i = 0; i < LB; ++i)
                        if (i < L) {
                            const float2 y = x[i][j];
                            const float2 v = __fmul2_rn(y, f2);
                            // consistent: x = y - deq(q_s)
                            x[i][j] = QF::store_fma(qc + i * VW + 2 * kNC * j, v, nsw, nswb, y);
                        }
                    if (on[j][0] && rr[j] == 0) sc[so[j] + vv[j]] = sw0;
                    if (on[j][1] && r1[j] == 0) sc[so[j] + w1[j]] = sw1;
                }
            }
            fence_proxy_async_smem();   // the chunk's new contents, for the bulk store
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[dc]);
            dc = dc + 1 == kD ? 0 : dc + 1;
#pragma unroll
            for (int j = 0; j < CPP; ++j) {   // next pass: windows start one column later
                if (--rr[j] < 0) {
                    rr[j] += L;
                    --vv[j];
                }
            }
        }
        if (aborted) break;
        // the item's rows of x back to HBM (both columns of a pair; a column
        // past the width lands in the row's padding)
        float *xg = info.xrow;
#pragma unroll
        for (int j = 0; j < CPP; ++j)
            if (vv[j] > kOutside + kBatchMaxSide) {
#pragma unroll
                for (int i = 0; i < LB; ++i)
                    if (i < L)
                        *reinterpret_cast<float2 *>(xg + og[j] + i * P) = x[i][j];
            }
        if (A.n_groups > 1) {
            // the item's rows of x are stored: count this warp (release); the
            // storer warp publishes the window-rows once every consumer warp
            // has counted the item
            __syncwarp();
            if (lane == 0)
                asm volatile("red.release.cta.shared::cta.add.u32 [%0], 1;" ::"r"(smem_u32(xdone)) : "memory");
        }
    }
}

template <typename QT, int LB, bool EXACT>
cudaError_t launch_step_t(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    if (A.n_groups > 1) {
        // items wait for items of other CTAs: every CTA must be resident
        void *args[] = {const_cast<BStepArgs *>(&A)};
        return cudaLaunchCooperativeKernel((const void *)bstep_kernel<QT, LB, EXACT>, dim3(grid),
                                           dim3(kThreads), args, smem, s);
    }
    bstep_kernel<QT, LB, EXACT><<<grid, kThreads, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename QT>
cudaError_t launch_step_q(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    switch (A.L) {
        case 1: return launch_step_t<QT, 1, true>(A, grid, smem, s);
        case 2: return launch_step_t<QT, 2, true>(A, grid, smem, s);
        case 3: return launch_step_t<QT, 3, true>(A, grid, smem, s);
        case 4: return launch_step_t<QT, 4, true>(A, grid, smem, s);
        case 5: return launch_step_t<QT, 5, true>(A, grid, smem, s);
        case 6: return launch_step_t<QT, 6, true>(A, grid, smem, s);
        case 7: return launch_step_t<QT, 7, true>(A, grid, smem, s);
        case 8: return launch_step_t<QT, 8, true>(A, grid, smem, s);
        case 9: return launch_step_t<QT, 9, true>(A, grid, smem, s);
        case 10: return launch_step_t<QT, 10, true>(A, grid, smem, s);
        case 11: return launch_step_t<QT, 11, true>(A, grid, smem, s);
        case 12: return launch_step_t<QT, 12, true>(A, grid, smem, s);
        default: return launch_step_t<QT, 16, false>(A, grid, smem, s);
    }
}

template <typename QT>
cudaError_t prepare_q(size_t smem)
{
    const void *ks[] = {
        (const void *)bstep_kernel<QT, 1, true>,  (const void *)bstep_kernel<QT, 2, true>,
        (const void *)bstep_kernel<QT, 3, true>,  (const void *)bstep_kernel<QT, 4, true>,
        (const void *)bstep_kernel<QT, 5, true>,  (const void *)bstep_kernel<QT, 6, true>,
        (const void *)bstep_kernel<QT, 7, true>,  (const void *)bstep_kernel<QT, 8, true>,
        (const void *)bstep_kernel<QT, 9, true>,  (const void *)bstep_kernel<QT, 10, true>,
        (const void *)bstep_kernel<QT, 11, true>, (const void *)bstep_kernel<QT, 12, true>,
        (const void *)bstep_kernel<QT, 16, false>};
    for (const void *k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace batch

}  // namespace smre

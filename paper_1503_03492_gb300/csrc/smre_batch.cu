// Batched standard Dykstra path on sm_103a: the images of a batch (any mix of
// sizes up to 2048 columns) share every launch.
//
// Paper: Sec. 2.3 (Algorithm 2, projection Eq. dykstra:if) with the increment
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
// asynchronous copies (TMA engine), as far ahead as the ring allows.  The 480
// consumer threads keep the item's x in registers (thread t owns columns
// t + 480 j), form y = x + q, the column sums of y^2 and, through shared
// memory, the window sums in a fixed column order (the same order as the
// single-image kernels, so FP32 results agree bit for bit), take the ball
// test and write x (at the item's end) and the new increments straight to
// HBM.
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "smre_internal.h"
#include "smre_ptx.cuh"

namespace smre {

namespace {

constexpr float kNearBand = 1e-6f;   // FP64 recheck band of the ball test, relative to cS
constexpr int kNC = kBatchConsumers;
constexpr int kD = kBatchDescs;
constexpr int kThreads = kNC + 32;
constexpr int kNormThreads = 256;

template <typename QT>
struct QConv;
template <>
struct QConv<float> {
    static constexpr bool mixed = false;
    __device__ static float to(float v) { return v; }
    __device__ static float from(float v) { return v; }
};
template <>
struct QConv<__nv_bfloat16> {
    static constexpr bool mixed = true;
    __device__ static __nv_bfloat16 to(float v) { return __float2bfloat16_rn(v); }
    __device__ static float from(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <>
struct QConv<__half> {
    static constexpr bool mixed = true;
    __device__ static __half to(float v) { return __float2half_rn(v); }
    __device__ static float from(__half v) { return __half2float(v); }
};

__host__ __device__ constexpr int lb_of(int L)
{
    return L <= 1 ? 1 : L <= 2 ? 2 : L <= 4 ? 4 : L <= 8 ? 8 : L <= 12 ? 12 : 16;
}
// columns per consumer thread: x of an item takes LB * CPT registers
__host__ __device__ constexpr int cpt_of(int LB) { return LB == 1 ? 16 : LB == 2 ? 8 : 5; }
__host__ __device__ constexpr int vw_of(int LB) { return kNC * cpt_of(LB); }
__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }
__host__ __device__ constexpr int round128(int v) { return (v + 127) & ~127; }
// scale-plane row length of side L (windows per unit row, padded to 16 bytes)
__host__ __device__ constexpr int scale_row(int W, int L) { return ((W / L) + 3) & ~3; }

struct BItem {
    int slot, u0, nu;
};

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

__device__ __forceinline__ BItem decode_item(const BStepArgs &A, int item)
{
    const int i = find_active(A.prefix, A.n_active, item);
    BItem it;
    it.slot = __ldg(A.active + i);
    const int k = __ldg(A.kpack + i);
    const int units = (A.imgs[it.slot].H - A.a) / A.L;
    it.u0 = (item - __ldg(A.prefix + i)) * k;
    it.nu = min(k, units - it.u0);
    return it;
}

// Bounded wait for an mbarrier phase.  On expiry (or when another CTA or
// role gave up) it records the time-out, raises the CTA's abort flag and
// returns false.
__device__ bool wait_phase(uint64_t *bar, unsigned parity, const BStepArgs &A,
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

// Producer: walks the CTA's items in the consumers' order and fills the ring.
template <typename QT>
__device__ void produce(const BStepArgs &A, unsigned char *ring, uint64_t *full,
                        uint64_t *written, int *s_off, volatile int *s_abort)
{
    constexpr bool MIXED = QConv<QT>::mixed;
    const int L = A.L;
    int head = 0, d_next = 0, d_tail = 0, n_out = 0;
    unsigned wph = 0;    // parity of the next `written` wait, per descriptor
    unsigned fiss = 0;   // toggled per issue: parity of the latest `full` phase, per descriptor
    bool dead = false;

    auto pop = [&]() -> bool {   // the consumers released the oldest chunk
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
    auto issue = [&](const void *src0, unsigned b0, const void *src1, unsigned b1) -> bool {
        const int n = round128(round16((int)b0) + (int)b1);
        int at;
        if (!alloc(n, at)) return false;
        s_off[d_next] = at;
        mbar_arrive_expect_tx(&full[d_next], b0 + b1);
        bulk_load(ring + at, src0, b0, &full[d_next]);
        if (b1) bulk_load(ring + at + round16((int)b0), src1, b1, &full[d_next]);
        fiss ^= 1u << d_next;
        head = at + n;
        ++n_out;
        d_next = d_next + 1 == kD ? 0 : d_next + 1;
        return true;
    };

    for (int item = blockIdx.x; item < A.n_items && !dead; item += gridDim.x) {
        const BItem it = decode_item(A, item);
        const BImage &im = A.imgs[it.slot];
        if (im.ctl->stop) continue;
        const int P = im.pitch;
        const bool first = im.ctl->cycles == 0;
        const unsigned xbytes = (unsigned)(it.nu * L * P) * 4u;
        if (!issue(im.x + (size_t)(A.a + L * it.u0) * P, xbytes, nullptr, 0)) {
            dead = true;
            break;
        }
        if (first) continue;   // q = 0 in an image's first cycle: nothing to read
        const unsigned qbytes = (unsigned)(it.nu * L * P) * (unsigned)sizeof(QT);
        const int nwp = scale_row(im.W, L);
        const unsigned sbytes = MIXED ? (unsigned)(it.nu * nwp) * 4u : 0u;
        for (int b = 0; b < L; ++b) {
            const QT *qsrc = reinterpret_cast<const QT *>(im.q) + im.qoff[A.p0 + b] +
                             (size_t)it.u0 * L * P;
            const float *ssrc = MIXED ? im.qs + im.soff[A.p0 + b] + (size_t)it.u0 * nwp : nullptr;
            if (!issue(qsrc, qbytes, ssrc, sbytes)) {
                dead = true;
                break;
            }
        }
    }
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

template <typename QT, int LB>
__global__ void __launch_bounds__(kThreads, 1) bstep_kernel(const BStepArgs A)
{
    using C = QConv<QT>;
    constexpr bool MIXED = C::mixed;
    constexpr int CPT = cpt_of(LB);
    constexpr int VW = vw_of(LB);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);   // [kD]
    uint64_t *written = full + kD;                          // [kD]
    int *s_off = reinterpret_cast<int *>(written + kD);     // [kD] ring offset of each chunk
    float *part = reinterpret_cast<float *>(smem + 256);    // [VW] column sums (LB > 1)
    double *part64 = reinterpret_cast<double *>(smem + 256 + (size_t)VW * 4);   // [VW]
    unsigned char *ring = smem + A.ring_offset;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = A.L;
    if (tid == 0) {
        for (int d = 0; d < kD; ++d) {
            mbar_init(&full[d], 1);
            mbar_init(&written[d], kNC / 32);
            s_off[d] = 0;
        }
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    if (warp == kNC / 32) {
        if (lane == 0) produce<QT>(A, ring, full, written, s_off, &s_abort);
        return;
    }

    // ------------------------------------------------------------ consumers
    int dc = 0;          // descriptor of the next chunk
    unsigned fph = 0;    // parity of the next `full` wait, per descriptor
    const float cS = A.cS, sqrt_cS = A.sqrt_cS;
    for (int item = blockIdx.x; item < A.n_items; item += gridDim.x) {
        const BItem it = decode_item(A, item);
        const BImage &im = A.imgs[it.slot];
        if (im.ctl->stop) continue;
        const int P = im.pitch, W = im.W;
        const bool first = im.ctl->cycles == 0;
        const int nwp = scale_row(W, L);
        int sj[CPT], cj[CPT];
        bool vj[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int vc = tid + j * kNC;   // virtual column: unit vc / P, column vc % P
            sj[j] = vc / P;
            cj[j] = vc - sj[j] * P;
            vj[j] = sj[j] < it.nu && cj[j] < W;
        }

        // the item's rows of x into registers
        float x[LB][CPT];
        bool bad = !wait_phase(&full[dc], (fph >> dc) & 1u, A, &s_abort);
        fph ^= 1u << dc;
        {
            const float *xb = reinterpret_cast<const float *>(ring + s_off[dc]);
#pragma unroll
            for (int j = 0; j < CPT; ++j)
#pragma unroll
                for (int i = 0; i < LB; ++i)
                    x[i][j] = (i < L && vj[j] && !bad) ? xb[(sj[j] * L + i) * P + cj[j]] : 0.f;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&written[dc]);
        dc = dc + 1 == kD ? 0 : dc + 1;

        bool aborted = false;
        for (int b = 0; b < L; ++b) {
            const int cend = b + ((W - b) / L) * L;   // columns b .. cend-1 lie in windows
            const QT *qb = nullptr;
            const float *sb = nullptr;
            if (!first) {
                if (!bad) bad = !wait_phase(&full[dc], (fph >> dc) & 1u, A, &s_abort);
                fph ^= 1u << dc;
                const int off = s_off[dc];
                qb = reinterpret_cast<const QT *>(ring + off);
                sb = reinterpret_cast<const float *>(ring + off +
                                                     round16(it.nu * L * P * (int)sizeof(QT)));
            }
            // y = x + q_s on the owned columns, and the column sums of y^2
            bool on[CPT];
            int v[CPT];
            float sq[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                on[j] = vj[j] && cj[j] >= b && cj[j] < cend;
                v[j] = on[j] ? (cj[j] - b) / L : 0;
                sq[j] = 0.f;
                if (on[j] && !bad) {
                    float qsc = 1.f;
                    if (MIXED && !first) qsc = sb[sj[j] * nwp + v[j]];
#pragma unroll
                    for (int i = 0; i < LB; ++i) {
                        if (i < L) {
                            float qv = 0.f;
                            if (!first) {
                                qv = C::from(qb[(sj[j] * L + i) * P + cj[j] - b]);
                                if (MIXED) qv *= qsc;
                            }
                            const float y = x[i][j] + qv;
                            x[i][j] = y;
                            sq[j] = fmaf(y, y, sq[j]);
                        }
                    }
                    if (LB > 1) part[sj[j] * P + cj[j]] = sq[j];
                }
            }
            if (!first) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&written[dc]);   // chunk read: the ring slot is free
                dc = dc + 1 == kD ? 0 : dc + 1;
            }
            if (named_sync_or(1, bad, kNC)) {   // column sums complete (or a copy was lost)
                aborted = true;
                break;
            }

            // window sums in column order and the ball test of Eq. (dykstra:if)
            float scale[CPT], tsv[CPT];
            bool near = false;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                scale[j] = 1.f;
                tsv[j] = 0.f;
                if (on[j]) {
                    float ts;
                    if (LB == 1) {
                        ts = sq[j];
                    } else {
                        const float *pp = part + sj[j] * P + b + v[j] * L;
                        ts = 0.f;
                        for (int m = 0; m < L; ++m) ts += pp[m];
                    }
                    tsv[j] = ts;
                    if (fabsf(ts - cS) <= kNearBand * cS) near = true;
                    if (ts > cS) scale[j] = sqrt_cS * rsqrtf(ts);
                }
            }
            if (named_sync_or(1, near, kNC)) {
                // rare: windows within the band get their sums again in FP64
                double s64[CPT];
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    s64[j] = 0.0;
                    if (on[j]) {
#pragma unroll
                        for (int i = 0; i < LB; ++i)
                            if (i < L) s64[j] = fma((double)x[i][j], (double)x[i][j], s64[j]);
                        if (LB > 1) part64[sj[j] * P + cj[j]] = s64[j];
                    }
                }
                named_sync(1, kNC);
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    if (!on[j] || fabsf(tsv[j] - cS) > kNearBand * cS) continue;
                    double t64 = s64[j];
                    if (LB > 1) {
                        const double *pp = part64 + sj[j] * P + b + v[j] * L;
                        t64 = 0.0;
                        for (int m = 0; m < L; ++m) t64 += pp[m];
                    }
                    scale[j] = t64 > A.cS64 ? (float)sqrt(A.cS64 / t64) : 1.f;
                    tsv[j] = (float)t64;
                }
            }

            // x = p_s(y), q_s = y - x, increments straight to HBM
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                if (!on[j]) continue;
                QT *qg = reinterpret_cast<QT *>(im.q) + im.qoff[A.p0 + b] +
                         (size_t)(it.u0 + sj[j]) * L * P + (cj[j] - b);
                if (!MIXED) {
#pragma unroll
                    for (int i = 0; i < LB; ++i)
                        if (i < L) {
                            const float y = x[i][j];
                            const float xn = y * scale[j];
                            x[i][j] = xn;
                            __stcs(reinterpret_cast<float *>(qg) + (size_t)i * P, y - xn);
                        }
                } else {
                    // window scale: a power of two >= 2^-14 |q_s|_2 >= 2^-14 max |q_i|
                    const float qn = (1.f - scale[j]) * sqrtf(tsv[j]);
                    float sw = 0.f, inv = 0.f;
                    if (qn > 0.f) {
                        int e;
                        frexpf(qn, &e);
                        sw = ldexpf(1.f, e - 14);
                        inv = ldexpf(1.f, 14 - e);
                    }
#pragma unroll
                    for (int i = 0; i < LB; ++i)
                        if (i < L) {
                            const float y = x[i][j];
                            const float xn = y * scale[j];
                            const QT h = C::to((y - xn) * inv);
                            x[i][j] = y - C::from(h) * sw;   // consistent: x = y - deq(q_s)
                            qg[(size_t)i * P] = h;
                        }
                    if (cj[j] == b + v[j] * L)
                        im.qs[im.soff[A.p0 + b] + (size_t)(it.u0 + sj[j]) * nwp + v[j]] = sw;
                }
            }
        }
        if (aborted) break;
        // the item's rows of x back to HBM
        const int row0 = A.a + L * it.u0;
#pragma unroll
        for (int j = 0; j < CPT; ++j)
            if (vj[j]) {
#pragma unroll
                for (int i = 0; i < LB; ++i)
                    if (i < L) im.x[(size_t)(row0 + sj[j] * L + i) * P + cj[j]] = x[i][j];
            }
    }
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < kNormThreads / 32; ++i) s += sh[i];   // fixed order
    return s;
}

// Cycle norm of Algorithm 2 per image: d^2 = |x - x_prev|^2, n^2 = |x_prev|^2
// over fixed chunks of kBatchNormRows rows (FP32 within a row and thread,
// FP64 across), then x_prev <- x.  The chunking and the order depend on the
// image alone, not on the batch it is in.
__global__ void __launch_bounds__(kNormThreads) bnorm_kernel(const BNormArgs A)
{
    __shared__ double sh[kNormThreads / 32];
    for (int ch = blockIdx.x; ch < A.n_chunks; ch += gridDim.x) {
        const int i = find_active(A.prefix, A.n_active, ch);
        const BImage &im = A.imgs[__ldg(A.active + i)];
        if (im.ctl->stop) continue;
        const int c0 = ch - __ldg(A.prefix + i);
        const int r0 = c0 * kBatchNormRows, r1 = min(im.H, r0 + kBatchNormRows);
        double D = 0.0, N = 0.0;
        for (int r = r0; r < r1; ++r) {
            const float *xr = im.x + (size_t)r * im.pitch;
            float *pr = im.xprev + (size_t)r * im.pitch;
            float dd = 0.f, nn = 0.f;
            for (int c = threadIdx.x; c < im.W; c += kNormThreads) {
                const float xv = xr[c], pv = pr[c];
                const float d = xv - pv;
                dd = fmaf(d, d, dd);
                nn = fmaf(pv, pv, nn);
                pr[c] = xv;
            }
            D += (double)dd;
            N += (double)nn;
        }
        D = block_sum(D, sh);
        N = block_sum(N, sh);
        if (threadIdx.x == 0) {
            im.part[2 * c0] = D;
            im.part[2 * c0 + 1] = N;
        }
    }
}

// Stopping test of Algorithm 2 per image (one block per active image).
__global__ void __launch_bounds__(kNormThreads) bdecide_kernel(const BDecideArgs A)
{
    __shared__ double sh[kNormThreads / 32];
    const BImage &im = A.imgs[A.active[blockIdx.x]];
    Control *ctl = im.ctl;
    if (ctl->stop) return;
    double d = 0.0, n = 0.0;
    for (int i = threadIdx.x; i < im.nchunks; i += kNormThreads) {
        d += im.part[2 * i];
        n += im.part[2 * i + 1];
    }
    d = block_sum(d, sh);
    n = block_sum(n, sh);
    if (threadIdx.x == 0) {
        const double step = sqrt(d), prev = sqrt(n);
        const int cyc = ctl->cycles;
        if (cyc < im.hist_cap) {
            im.hist[2 * cyc] = step;
            im.hist[2 * cyc + 1] = prev;
        }
        ctl->cycles = cyc + 1;
        ctl->step = step;
        ctl->prev_norm = prev;
        const bool conv = A.tol >= 0.0 && (A.tol_relative ? step <= A.tol * prev : step <= A.tol);
        const bool cap = cyc + 1 >= A.max_cycles;
        ctl->status = conv || A.tol < 0.0 ? (int)SMRE_OK : (int)SMRE_ENOTCONVERGED;
        ctl->stop = (conv || cap) ? 1 : 0;
    }
}

template <typename QT, int LB>
cudaError_t launch_step_t(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    bstep_kernel<QT, LB><<<grid, kThreads, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename QT>
cudaError_t launch_step_q(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    switch (lb_of(A.L)) {
        case 1: return launch_step_t<QT, 1>(A, grid, smem, s);
        case 2: return launch_step_t<QT, 2>(A, grid, smem, s);
        case 4: return launch_step_t<QT, 4>(A, grid, smem, s);
        case 8: return launch_step_t<QT, 8>(A, grid, smem, s);
        case 12: return launch_step_t<QT, 12>(A, grid, smem, s);
        default: return launch_step_t<QT, 16>(A, grid, smem, s);
    }
}

template <typename QT>
cudaError_t prepare_q(size_t smem)
{
    const void *ks[] = {(const void *)bstep_kernel<QT, 1>, (const void *)bstep_kernel<QT, 2>,
                        (const void *)bstep_kernel<QT, 4>, (const void *)bstep_kernel<QT, 8>,
                        (const void *)bstep_kernel<QT, 12>, (const void *)bstep_kernel<QT, 16>};
    for (const void *k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

int batch_lb(int L) { return lb_of(L); }
int batch_virtual_width(int L) { return vw_of(lb_of(L)); }
size_t batch_part_bytes(int L) { return lb_of(L) > 1 ? (size_t)vw_of(lb_of(L)) * 12 : 0; }
int batch_threads() { return kThreads; }

cudaError_t batch_prepare(int qtype, size_t smem_max)
{
    if (qtype == 1) return prepare_q<__nv_bfloat16>(smem_max);
    if (qtype == 2) return prepare_q<__half>(smem_max);
    return prepare_q<float>(smem_max);
}

cudaError_t launch_batch_step(int qtype, const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    if (A.n_items <= 0 || grid <= 0) return cudaSuccess;
    if (qtype == 1) return launch_step_q<__nv_bfloat16>(A, grid, smem, s);
    if (qtype == 2) return launch_step_q<__half>(A, grid, smem, s);
    return launch_step_q<float>(A, grid, smem, s);
}

cudaError_t launch_batch_norm(const BNormArgs &A, int grid, cudaStream_t s)
{
    if (A.n_chunks <= 0 || grid <= 0) return cudaSuccess;
    bnorm_kernel<<<grid, kNormThreads, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_batch_decide(const BDecideArgs &A, cudaStream_t s)
{
    if (A.n_active <= 0) return cudaSuccess;
    bdecide_kernel<<<A.n_active, kNormThreads, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace smre

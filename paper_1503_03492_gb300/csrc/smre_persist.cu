// Persistent cooperative kernel of the standard Dykstra path on sm_103a.
//
// One launch runs the whole projection (Sec. 2.3, Algorithm 2): every cycle
// visits the groups (L, a) in the set order (sides descending, a ascending);
// inside a group the L tilings (L, a, b), b = 0..L-1, only move windows
// sideways, so a CTA that holds a band of window-rows ("units") of the group
// runs all L passes on it with block barriers alone.
//
// Side-resident bands: for each side L a CTA owns units [u0, u1) for all
// offsets a.  Its band of x rows (rows a + L u0 .. a + L u1 - 1) stays in
// shared memory for the whole side; from offset a to a + 1 the band slides
// down one row: the top row is published (stored to HBM, then a release flag)
// and the lower neighbour's published top row is taken in at the bottom
// (acquire).  At a side change the band is stored and the next side's band
// loaded after the flags of the CTAs that last wrote those rows.  One grid
// barrier per cycle gathers the FP64 norms of the stopping test.
//
// Data movement:
//  - increments q_s (the HBM stream, sum_L L^2 H W floats) come in through a
//    ring of shared-memory stages filled by bulk async copies (TMA engine)
//    that a producer warp keeps up to 16 passes ahead of the consumers; the
//    consumers write the updated increments straight back to HBM with
//    streaming stores (immediate row offsets when the pitch equals the
//    shared-memory row stride);
//  - x lives in shared memory, in the bands; it goes through L2 only as the
//    published rows;
//  - the cycle norm |x - x_prev|^2, |x_prev|^2 (FP64) is fused into the
//    publication that makes each row final in a cycle.
//
// Every wait (dependency flags, grid barrier, copy completion) has a time
// limit; on expiry the kernel records SMRE_ETIMEOUT, lets its copies in
// flight finish, and returns, so the context stays usable.
#include <cuda_runtime.h>

#include <cstdint>

#include "smre_internal.h"
#include "smre_ptx.cuh"

namespace smre {

namespace {

constexpr float kNearBand = 1e-6f;

// Record a time-out once and raise the abort word every CTA polls.
__device__ void raise_timeout(const PersistArgs &A)
{
    atomicCAS(&A.ctl->status, (int)SMRE_OK, (int)SMRE_ETIMEOUT);
    atomicExch(A.abort_word, 1);
}

// Thread 0: wait until *p >= target (acquire), or time out / see an abort.
// Returns false when the CTA must abandon the projection.
__device__ bool wait_geq(const PersistArgs &A, const unsigned *p, unsigned target)
{
    if (ld_acquire(p) >= target) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 0;; ++it) {
        if (ld_acquire(p) >= target) return true;
        if (it >= 4) __nanosleep(40);
        if ((it & 31) == 31) {
            if (ld_volatile(A.abort_word)) return false;
            if (globaltimer() - t0 > A.timeout_ns) {
                raise_timeout(A);
                return false;
            }
        }
    }
}

// Wait on an mbarrier phase with a time limit (every wait of the kernel is
// bounded).  Returns false on time-out or when another CTA aborted.
__device__ bool mbar_wait_timed(const PersistArgs &A, uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (ld_volatile(A.abort_word)) return false;
        if (globaltimer() - t0 > A.timeout_ns) {
            raise_timeout(A);
            return false;
        }
    }
}

// named barrier 1 among the consumer warps; returns the OR of pred over them
__device__ __forceinline__ bool consumers_sync_or(bool pred, int nthreads)
{
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)pred), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void consumers_sync(int nthreads)
{
    asm volatile("barrier.sync 1, %0;" ::"r"(nthreads) : "memory");
}

__device__ __forceinline__ void cta_sync_all() { asm volatile("barrier.sync 0;" ::: "memory"); }

// named barrier 2 among the warps that hold windows in the current task,
// returning the OR of pred over them
__device__ __forceinline__ bool workers_sync_or(bool pred, int nthreads)
{
    if (nthreads == 32) {
        __syncwarp();
        return __any_sync(0xffffffffu, pred);
    }
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, 2, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)pred), "r"(nthreads)
        : "memory");
    return r != 0;
}

// One offset a of a side task as the passes see it.
struct PassTask {
    int L, U;          // side, units present at this offset (band rows 0 .. U*L-1)
    int pass0;         // q offset entry of pass b = 0
    float cS, sqrt_cS;
    double cS64;
};

// Everything a consumer warp needs to run the passes of one task.
struct PassCtx {
    const PersistArgs *A;
    uint64_t *full, *written;
    float *stage0, *xs;
    const long long *pass_qoff; // q offset of each pass of this CTA's cycle
    int S, NCW, NC, warp, lane, pitch;
};

// The L passes b = 0..L-1 of one task, side L known at compile time.  Returns
// true when the launch must be abandoned (a copy did not arrive in time).
template <int L, int SP, bool PEQ>
__device__ __forceinline__ bool run_passes(const PassCtx &cx, const PassTask &ts, int &s_cur,
                                           unsigned &fph)
{
    // SP: row stride of x and of the stages in shared memory (compile time,
    // so every shared-memory access of a pass uses an immediate offset);
    // PEQ: the image pitch equals SP, so the increment stores in HBM use
    // immediate row offsets too
    constexpr int wpw = 32 / L;                     // windows per warp
    constexpr int MI = max_items_for_side(L);       // items per warp and task
    const int lane = cx.lane, warp = cx.warp, pitch = PEQ ? SP : cx.pitch;
    const int wl = lane / L, col = lane - wl * L;   // window of the lane, column in it
    const int base = wl * L;
    const bool lane_on = lane < wpw * L;
    const int W = cx.A->W, U = ts.U;
    const int nv0 = W / L, rem0 = W - nv0 * L;      // pass b has nv0 - (b > rem0) windows
    const int nwc = (nv0 + wpw - 1) / wpw;          // warp chunks per unit
    // this warp's (unit, chunk) items, fixed for the task's passes
    int it_q[MI], it_g[MI], it_v[MI];
    int nit = 0;
#pragma unroll
    for (int n = 0; n < MI; ++n) {
        const int item = warp + n * cx.NCW;
        it_q[n] = it_g[n] = 0;
        it_v[n] = 1 << 30;
        if (item < U * nwc) {
            const int j = item / nwc, k = item - j * nwc;
            it_v[n] = k * wpw + wl;
            it_q[n] = j * L * SP + it_v[n] * L + col;      // shared memory (pass-relative column)
            it_g[n] = j * L * pitch + it_v[n] * L + col;   // the same column in HBM
            nit = n + 1;
        }
    }
    const int nwork = U * nwc < cx.NCW ? U * nwc : cx.NCW;   // warps holding items
    if (nit == 0) {
        // no window of this task in this warp: follow the stages (the wait
        // suspends the warp) and release each one untouched
        bool bad = false;
        for (int b = 0; b < L; ++b) {
            if (!bad) bad = !mbar_wait_timed(*cx.A, &cx.full[s_cur], (fph >> s_cur) & 1u);
            fph ^= 1u << s_cur;
            __syncwarp();
            if (lane == 0) mbar_arrive(&cx.written[s_cur]);
            s_cur = s_cur + 1 == cx.S ? 0 : s_cur + 1;
        }
        return bad;
    }
    const float cS = ts.cS, sqrt_cS = ts.sqrt_cS;
    for (int b = 0; b < L; ++b) {
        const int s = s_cur;
        const bool bad = !mbar_wait_timed(*cx.A, &cx.full[s], (fph >> s) & 1u);
        fph ^= 1u << s;
        float *stg = cx.stage0 + (size_t)s * cx.A->stage_floats;
        float *qg = cx.A->q + cx.pass_qoff[ts.pass0 + b];   // this pass's increments in HBM
        const int nv = b <= rem0 ? nv0 : nv0 - 1;
#pragma unroll
        for (int n = 0; n < MI; ++n) {
            if (n >= nit) break;
            const bool on = lane_on && it_v[n] < nv;
            float *xr = cx.xs + it_q[n] + b;
            const float *qr = stg + it_q[n];
            float *qw = qg + it_g[n];
            float y[L];
            float sq = 0.f;
            if (on) {
#pragma unroll
                for (int i = 0; i + 1 < L; i += 2) {   // FP32x2: rows i, i + 1
                    const float2 s2 = __fadd2_rn(make_float2(xr[i * SP], xr[(i + 1) * SP]),
                                                 make_float2(qr[i * SP], qr[(i + 1) * SP]));
                    y[i] = s2.x;
                    y[i + 1] = s2.y;
                }
                if (L & 1) y[L - 1] = xr[(L - 1) * SP] + qr[(L - 1) * SP];
#pragma unroll
                for (int i = 0; i < L; ++i) sq = fmaf(y[i], y[i], sq);
            }
            // window sum over its L lanes, in column order
            float t = 0.f;
#pragma unroll
            for (int m = 0; m < L; ++m) t += __shfl_sync(0xffffffffu, sq, (base + m) & 31);
            float scale = 1.f;
            const bool near = on && fabsf(t - cS) <= kNearBand * cS;
            if (on && t > cS) scale = sqrt_cS * rsqrtf(t);
            if (__any_sync(0xffffffffu, near)) {
                // rare: redo the sums of windows near the boundary in FP64
                double sq64 = 0.0;
                if (on) {
#pragma unroll
                    for (int i = 0; i < L; ++i) sq64 = fma((double)y[i], (double)y[i], sq64);
                }
                double t64 = 0.0;
#pragma unroll
                for (int m = 0; m < L; ++m) t64 += __shfl_sync(0xffffffffu, sq64, (base + m) & 31);
                if (near) scale = t64 > ts.cS64 ? (float)sqrt(ts.cS64 / t64) : 1.f;
            }
            if (on) {
                // x = y * scale, q = y - x (FP32x2 on row pairs; streaming stores:
                // the increments are read again only next cycle)
                const float2 sc2 = make_float2(scale, scale);
#pragma unroll
                for (int i = 0; i + 1 < L; i += 2) {
                    const float2 y2 = make_float2(y[i], y[i + 1]);
                    const float2 n2 = __fmul2_rn(y2, sc2);
                    const float2 q2 = __fadd2_rn(y2, make_float2(-n2.x, -n2.y));
                    xr[i * SP] = n2.x;
                    xr[(i + 1) * SP] = n2.y;
                    __stcs(qw + i * pitch, q2.x);
                    __stcs(qw + (i + 1) * pitch, q2.y);
                }
                if (L & 1) {
                    const float xn = y[L - 1] * scale;
                    xr[(L - 1) * SP] = xn;
                    __stcs(qw + (L - 1) * pitch, y[L - 1] - xn);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&cx.written[s]);   // this warp is done reading the stage
        s_cur = s + 1 == cx.S ? 0 : s + 1;
        // orders xs between passes; a copy lost anywhere abandons the launch
        if (workers_sync_or(bad, nwork * 32)) return true;
    }
    return false;
}

template <int SP, bool PEQ>
__device__ __forceinline__ bool run_task_passes(const PassCtx &cx, const PassTask &ts, int &s_cur,
                                                unsigned &fph)
{
    switch (ts.L) {
#define RP(l) case l: return run_passes<l, SP, PEQ>(cx, ts, s_cur, fph);
        RP(1) RP(2) RP(3) RP(4) RP(5) RP(6) RP(7) RP(8)
        RP(9) RP(10) RP(11) RP(12) RP(13) RP(14) RP(15) RP(16)
#undef RP
        default: return true;
    }
}

// Rows r_first .. r_first + n - 1 of the image (those inside it) into shared
// memory rows k0 .. k0 + n - 1 (row stride SP), by the consumer threads.
template <int SP>
__device__ __forceinline__ void load_rows(const PersistArgs &A, float *xs, int k0, int r_first,
                                          int n, int tid, int NC)
{
    const int q4 = A.pitch / 4;
    const int rows = min(n, A.H - r_first);
    if (rows <= 0) return;
    const float4 *src = reinterpret_cast<const float4 *>(A.x + (size_t)r_first * A.pitch);
    float4 *dst = reinterpret_cast<float4 *>(xs + (size_t)k0 * SP);
    const int n4 = rows * q4;
    for (int i = tid; i < n4; i += NC) {
        const int rr = i / q4, c4 = i - rr * q4;
        dst[rr * (SP / 4) + c4] = __ldcg(src + i);
    }
}

// Shared-memory rows 0 .. n-1 back to image rows r_first .. (inside the image);
// rows whose bit is set in `fin` are final in the cycle: add their step and
// previous norm (FP64) and keep them as the next cycle's x_prev.
template <int SP>
__device__ __forceinline__ void store_rows(const PersistArgs &A, const float *xs, int r_first,
                                           int n, unsigned long long fin, int tid, int NC,
                                           double &d2, double &n2)
{
    const int q4 = A.pitch / 4;
    const int rows = min(n, A.H - r_first);
    if (rows <= 0) return;
    float4 *dst = reinterpret_cast<float4 *>(A.x + (size_t)r_first * A.pitch);
    const float4 *src = reinterpret_cast<const float4 *>(xs);
    const int n4 = rows * q4;
    for (int i = tid; i < n4; i += NC) {
        const int rr = i / q4, c4i = i - rr * q4;
        const float4 v = src[rr * (SP / 4) + c4i];
        dst[i] = v;
        const int c4 = c4i * 4;
        if (((fin >> rr) & 1ull) && c4 < A.W) {
            float4 *pp = reinterpret_cast<float4 *>(A.xprev + (size_t)(r_first + rr) * A.pitch) + c4i;
            const float4 pv = __ldcg(pp);
            const float xv[4] = {v.x, v.y, v.z, v.w};
            const float pw[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c4 + e < A.W) {
                    const double dd = (double)xv[e] - (double)pw[e];
                    d2 = fma(dd, dd, d2);
                    n2 = fma((double)pw[e], (double)pw[e], n2);
                }
            *pp = v;
        }
    }
}

// Shared-memory rows 1 .. n-1 move to 0 .. n-2.  Each thread owns whole
// float4 columns and walks them top-down, so no other thread's data is read.
template <int SP>
__device__ __forceinline__ void shift_rows_up(const PersistArgs &A, float *xs, int n, int tid,
                                              int NC)
{
    const int q4 = A.pitch / 4;
    float4 *x4 = reinterpret_cast<float4 *>(xs);
    for (int c = tid; c < q4; c += NC)
        for (int k = 0; k + 1 < n; ++k) x4[k * (SP / 4) + c] = x4[(k + 1) * (SP / 4) + c];
}

enum { kGo = 0, kStop = 1, kAbort = 2 };

// ------------------------------------------------------------------ kernel
//
// Warps 0 .. NCW-1 consume: they run the projections of each pass.  Warp NCW
// produces: its lane 0 streams the increments through the stage ring.
//   full[s]    completes when stage s holds the increments of its next pass
//              (bulk load; in the first cycle q = 0 and a plain arrive only
//              hands the empty stage over)
//   written[s] completes when every consumer warp is done reading stage s
//              (the new increments go straight to HBM with ordinary stores),
//              so the producer can refill the stage S passes ahead.
// In pass b of a task the consumer lanes map onto windows: with
// wpw = floor(32 / L) windows per warp, lane l takes column l % L of window
// k * wpw + l / L of its warp's chunk k; a window's column sums meet by
// shuffles in a fixed order, so every lane of a window sees the same sum.
// x of the task's rows lives in shared memory for the task's L passes.
template <int SP, bool PEQ>
__global__ void __launch_bounds__(kPersistThreads, 1) persist_kernel(const PersistArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = A.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);              // [S]
    uint64_t *written = full + kMaxStages;                            // [S]
    int *s_prov = reinterpret_cast<int *>(written + kMaxStages);      // [S] provides per stage
    unsigned char *tbl = smem + 512;                                  // schedule
    float *stage0 = reinterpret_cast<float *>(smem + A.stage_offset); // [S][stage_floats]
    float *xs = stage0 + (size_t)S * A.stage_floats;                  // [rows][SP]
    __shared__ int s_dec;
    __shared__ double s_red[2][32];

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int NCW = A.consumer_warps, NC = NCW * 32;
    const int cta = blockIdx.x, G = gridDim.x;
    const int pitch = A.pitch;

    // this CTA's schedule into shared memory
    {
        const int *hdr = reinterpret_cast<const int *>(A.sched + A.cta_off[cta]);
        const int nsd = hdr[0], ngr = hdr[1], npa = hdr[2], nde = hdr[3];
        const int n16 = (int)((16 + sizeof(SideS) * nsd + sizeof(GrpS) * ngr +
                               sizeof(long long) * npa + sizeof(int) * nde + 15) / 16);
        const int4 *src = reinterpret_cast<const int4 *>(hdr);
        int4 *dst = reinterpret_cast<int4 *>(tbl);
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int nside = reinterpret_cast<const int *>(tbl)[0];
    const int ngrp = reinterpret_cast<const int *>(tbl)[1];
    const int npass_tab = reinterpret_cast<const int *>(tbl)[2];
    const SideS *sides_s = reinterpret_cast<const SideS *>(tbl + 16);
    const GrpS *grps_s = reinterpret_cast<const GrpS *>(sides_s + nside);
    const long long *pass_qoff = reinterpret_cast<const long long *>(grps_s + ngrp);
    const int *deps_s = reinterpret_cast<const int *>(pass_qoff + npass_tab);
    // passes per cycle that carry increments (offsets with units present)
    int npass = 0;
    for (int si = 0; si < nside; ++si)
        for (int a = 0; a < sides_s[si].L; ++a)
            if (grps_s[sides_s[si].grp0 + a].U > 0) npass += sides_s[si].L;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&written[s], (unsigned)NCW);
            s_prov[s] = 0;
        }
        fence_mbar_init();
        s_dec = kGo;
    }
    __syncthreads();

    if (warp == NCW) {
        // ===================================================== producer warp
        bool dead = false;
        int s_head = 0;        // stage of the next pass to store
        unsigned wph = 0;      // parity of the next `written` wait, per stage
        for (int cyc = 0;; ++cyc) {
            const bool first = cyc == 0;
            if (lane == 0 && npass > 0 && !dead) {
                // cursor over the passes of the cycle: (side, offset, pass)
                struct Cur { int si, a, b; };
                auto advance = [&](Cur &c) {
                    if (++c.b < sides_s[c.si].L) return;
                    c.b = 0;
                    for (;;) {
                        if (++c.a >= sides_s[c.si].L) { c.a = 0; if (++c.si >= nside) return; }
                        if (grps_s[sides_s[c.si].grp0 + c.a].U > 0) return;
                    }
                };
                auto provide = [&](const Cur &c, int stg) {
                    s_prov[stg] += 1;
                    const SideS &sd = sides_s[c.si];
                    const int L = sd.L, U = grps_s[sd.grp0 + c.a].U;
                    const unsigned row_bytes = (unsigned)(pitch * sizeof(float));
                    mbar_arrive_expect_tx(&full[stg], row_bytes * L * U);
                    // the first cycle starts from q = 0: copy from a zeroed block
                    const float *src = first ? A.zeros : A.q + pass_qoff[sd.pass0 + c.a * L + c.b];
                    float *dst = stage0 + (size_t)stg * A.stage_floats;
                    if (pitch == SP) {         // one contiguous block per unit
                        for (int j = 0; j < U; ++j)
                            bulk_load(dst + (size_t)j * L * SP,
                                      first ? src : src + (size_t)j * L * pitch, row_bytes * L,
                                      &full[stg]);
                    } else {                   // row by row into SP-strided rows
                        for (int r = 0; r < L * U; ++r)
                            bulk_load(dst + (size_t)r * SP, first ? src : src + (size_t)r * pitch,
                                      row_bytes, &full[stg]);
                    }
                };
                Cur rc{0, 0, 0};               // refill cursor: first offset with units
                while (rc.si < nside && grps_s[sides_s[rc.si].grp0 + rc.a].U == 0) {
                    if (++rc.a >= sides_s[rc.si].L) { rc.a = 0; ++rc.si; }
                }
                int rs = s_head;
                const int pre = npass < S ? npass : S;
                for (int k = 0; k < pre; ++k) {
                    provide(rc, rs);
                    advance(rc);
                    rs = rs + 1 == S ? 0 : rs + 1;
                }
                for (int p = 0; p < npass; ++p) {
                    // consumers have read the stage of pass p: refill it S passes ahead
                    if (!mbar_wait_timed(A, &written[s_head], (wph >> s_head) & 1u)) {
                        dead = true;
                        break;
                    }
                    wph ^= 1u << s_head;
                    if (p + S < npass) {
                        provide(rc, s_head);
                        advance(rc);
                    }
                    s_head = s_head + 1 == S ? 0 : s_head + 1;
                }
            }
            __syncwarp();
            cta_sync_all();                    // consumers publish the decision
            const int dec = s_dec;
            cta_sync_all();
            if (dec != kGo || dead) break;
            // the consumers stored this cycle's increments with ordinary stores;
            // order them before the bulk (async-proxy) loads of the next cycle
            fence_proxy_async_global();
        }
        if (lane == 0) {
            // let every load in flight land before the shared memory is released
            for (int s = 0; s < S; ++s) {
                if (s_prov[s] == 0) continue;
                const unsigned par = (unsigned)((s_prov[s] - 1) & 1);
                for (unsigned it = 0; !mbar_try_wait(&full[s], par) && it < (1u << 22); ++it) {
                }
            }
            bulk_wait_all();
        }
        return;
    }

    // ======================================================== consumer warps
    const PassCtx cx{&A, full, written, stage0, xs, pass_qoff, S, NCW, NC, warp, lane, pitch};
    int s_cur = 0;
    unsigned fph = 0;            // parity of the next `full` wait, per stage
    double d2 = 0.0, n2 = 0.0;   // this thread's share of the cycle norm
    bool aborted = false;

    for (int cyc = 0;; ++cyc) {
        for (int si = 0; si < nside && !aborted; ++si) {
            const SideS sd = sides_s[si];
            const int L = sd.L, band = sd.U * L;

            // side start: wait for the last publishers (other CTAs) of the rows
            // this side may read, then bring the band in
            bool lost = false;
            if (tid == 0) {
                bool ok = true;
                if (A.selftest_timeout && cta == 0 && si == 0)
                    ok = wait_geq(A, A.selftest_flag, 1u);   // a flag nothing sets
                for (int k = 0; k < sd.dep_count && ok; ++k)
                    ok = wait_geq(A, A.flags + deps_s[sd.dep_begin + k], (unsigned)(cyc + 1));
                lost = !ok;
            }
            if (consumers_sync_or(lost, NC)) { aborted = true; break; }
            load_rows<SP>(A, xs, 0, sd.r0, band, tid, NC);
            consumers_sync(NC);

            for (int a = 0; a < L; ++a) {
                const GrpS gp = grps_s[sd.grp0 + a];
                if (a > 0) {
                    // the band slides down one row: drop the (published) top row,
                    // take the lower neighbour's published top row at the bottom
                    shift_rows_up<SP>(A, xs, band, tid, NC);
                    bool lost = false;
                    if (tid == 0)
                        lost = !(gp.nb_flag < 0 || wait_geq(A, A.flags + gp.nb_flag, (unsigned)(cyc + 1)));
                    if (consumers_sync_or(lost, NC)) { aborted = true; break; }
                    load_rows<SP>(A, xs, band - 1, sd.r0 + a - 1 + band, 1, tid, NC);
                    consumers_sync(NC);
                }
                if (gp.U > 0) {
                    const PassTask pt{L, gp.U, sd.pass0 + a * L, sd.cS, sd.sqrt_cS, sd.cS64};
                    const bool ab = run_task_passes<SP, PEQ>(cx, pt, s_cur, fph);
                    if (consumers_sync_or(ab, NC)) { aborted = true; break; }
                }
                // publish: the top row (dropped next), or the whole band at the end
                const int nrows = a < L - 1 ? 1 : band;
                const unsigned long long fin = a < L - 1 ? (unsigned long long)((sd.top_final >> a) & 1u)
                                                         : sd.end_final;
                store_rows<SP>(A, xs, sd.r0 + a, nrows, fin, tid, NC, d2, n2);
                consumers_sync(NC);
                if (tid == 0)   // release: the rows stored above (ordered by the barrier)
                    st_release(A.flags + sd.flag0 + a, (unsigned)(cyc + 1));
            }
        }

        // ---- end of cycle: publish norms, grid barrier, same decision everywhere
        int dec = kGo;
        double step = 0.0, prev = 0.0;
        if (aborted) {
            dec = kAbort;
        } else {
            double *slot = A.partials + (size_t)(cyc & 1) * 2 * G;   // double-buffered
            double a = d2, bb = n2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                bb += __shfl_xor_sync(0xffffffffu, bb, o);
            }
            if (lane == 0) {
                s_red[0][warp] = a;
                s_red[1][warp] = bb;
            }
            consumers_sync(NC);
            bool late = false;
            if (tid == 0) {
                double D = 0.0, N = 0.0;
                for (int w = 0; w < NCW; ++w) {
                    D += s_red[0][w];
                    N += s_red[1][w];
                }
                slot[2 * (size_t)cta] = D;
                slot[2 * (size_t)cta + 1] = N;
                __threadfence();
                atomicAdd(A.barrier, 1u);
                late = !wait_geq(A, A.barrier, (unsigned)G * (unsigned)(cyc + 1));
            }
            late = consumers_sync_or(late, NC);
            d2 = 0.0;
            n2 = 0.0;
            if (late) {
                dec = kAbort;
            } else {
                // every CTA sums the partials in the same fixed tree, in parallel:
                // thread i loads partial i, warps reduce by xor butterfly, then
                // the warp sums are added in warp order
                double a = 0.0, bq = 0.0;
                for (int i = tid; i < G; i += NC) {
                    a += __ldcg(slot + 2 * (size_t)i);
                    bq += __ldcg(slot + 2 * (size_t)i + 1);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    bq += __shfl_xor_sync(0xffffffffu, bq, o);
                }
                if (lane == 0) {
                    s_red[0][warp] = a;
                    s_red[1][warp] = bq;
                }
                consumers_sync(NC);
                double D = 0.0, N = 0.0;
                for (int w = 0; w < NCW; ++w) {
                    D += s_red[0][w];
                    N += s_red[1][w];
                }
                step = sqrt(D);
                prev = sqrt(N);
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
        fence_proxy_async_global();   // this cycle's increment stores before next cycle's bulk loads
        if (tid == 0) s_dec = dec;
        cta_sync_all();
        cta_sync_all();
        if (dec != kGo) break;
    }
}

template <int SP, bool PEQ>
cudaError_t launch_persist_t(const PersistArgs &A, int grid, int threads, size_t smem,
                             cudaStream_t s)
{
    auto k = persist_kernel<SP, PEQ>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<PersistArgs *>(&A)};
    return cudaLaunchCooperativeKernel((const void *)k, dim3(grid), dim3(threads), args, smem, s);
}

const void *kernel_for(int sp, bool peq)
{
    switch (sp) {
        case 128: return peq ? (const void *)persist_kernel<128, true> : (const void *)persist_kernel<128, false>;
        case 256: return peq ? (const void *)persist_kernel<256, true> : (const void *)persist_kernel<256, false>;
        case 512: return peq ? (const void *)persist_kernel<512, true> : (const void *)persist_kernel<512, false>;
        case 1024: return peq ? (const void *)persist_kernel<1024, true> : (const void *)persist_kernel<1024, false>;
        default: return nullptr;
    }
}

}  // namespace

int persist_smem_pitch(int pitch)
{
    int sp = 128;
    while (sp < pitch) sp *= 2;
    return sp <= 1024 ? sp : 0;
}

bool persist_supported(int max_side) { return max_side >= 1 && max_side <= 16; }

cudaError_t persist_occupancy(int sp, int pitch, int threads, size_t smem, int *blocks_per_sm)
{
    const void *k = kernel_for(sp, pitch == sp);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

cudaError_t launch_persist(const PersistArgs &A, int sp, int grid, int threads, size_t smem,
                           cudaStream_t s)
{
    const bool peq = A.pitch == sp;
    switch (sp) {
        case 128: return peq ? launch_persist_t<128, true>(A, grid, threads, smem, s)
                             : launch_persist_t<128, false>(A, grid, threads, smem, s);
        case 256: return peq ? launch_persist_t<256, true>(A, grid, threads, smem, s)
                             : launch_persist_t<256, false>(A, grid, threads, smem, s);
        case 512: return peq ? launch_persist_t<512, true>(A, grid, threads, smem, s)
                             : launch_persist_t<512, false>(A, grid, threads, smem, s);
        case 1024: return peq ? launch_persist_t<1024, true>(A, grid, threads, smem, s)
                              : launch_persist_t<1024, false>(A, grid, threads, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smre

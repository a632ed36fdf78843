// Standard (exact) Dykstra path on sm_103a: the group kernel, the fused
// cycle-norm reduction, the device-side stopping decision and the optional
// constraint-violation check.
//
// Paper: Sec. 2.3 (Algorithm 2 with the projection p_s of Sec. 2.3), with the
// increment update of the Sec. 3.2 listing applied to every set in turn.
//
// One cycle visits the tilings (L, a, b) in the order sides descending,
// a outer, b inner.  The L tilings of one group (L, a) share their window-rows
// ("units": rows a + L u .. a + L u + L - 1), and consecutive tilings of a
// group only move the windows sideways, so one CTA owns a whole unit and runs
// the L passes b = 0..L-1 on it with block-local barriers only.  Units of the
// same group are disjoint, hence independent CTAs; groups follow each other
// in stream order.
//
// Thread mapping: thread t owns the columns c = t + j*blockDim (j < CPT) of
// its unit for all L passes, keeping the unit's L x CPT pixels in registers.
// In pass b the column belongs to window v = (c - b) / L; a thread sums the
// squares of its column, the L column sums of a window are added from shared
// memory in a fixed order, so every thread of the window sees the same sum.
#include <cuda_runtime.h>

#include <mutex>

#include <cstdint>

#include "smre_internal.h"

namespace smre {

namespace {

// Near-boundary band of the ball test, relative to cS.  Inside it the sum of
// squares is recomputed in FP64 before the test t > cS is taken.
constexpr float kNearBand = 1e-6f;

template <int LB, int CPT>
__global__ void __launch_bounds__(1024, 1) group_kernel(const GroupArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_part = reinterpret_cast<float *>(smem_raw);                 // [2][pitch]
    double *s_part64 = reinterpret_cast<double *>(s_part + 2 * A.pitch); // [pitch]

    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int u = blockIdx.x;
    const int L = A.L;
    const int r0 = A.a + L * u;
    const int pitch = A.pitch;

    float xr[LB][CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        const int c = t + j * T;
#pragma unroll
        for (int i = 0; i < LB; ++i)
            if (i < L) xr[i][j] = (c < A.W) ? A.x[(size_t)(r0 + i) * pitch + c] : 0.f;
    }

    for (int b = 0; b < L; ++b) {
        const int nv = (A.W - b) / L;
        const int cend = b + nv * L;
        float *qb = A.q + A.q_off[b] + (size_t)u * L * pitch;
        float *part = s_part + (b & 1) * pitch;

        // y = x + q_s on this thread's columns, and the column sums of y^2
        bool inw[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = t + j * T;
            inw[j] = (c >= b) && (c < cend);
            float s = 0.f;
            if (inw[j]) {
#pragma unroll
                for (int i = 0; i < LB; ++i)
                    if (i < L) {
                        const float qv = A.first ? 0.f : qb[(size_t)i * pitch + (c - b)];
                        const float y = xr[i][j] + qv;
                        xr[i][j] = y;
                        s = fmaf(y, y, s);
                    }
            }
            if (c < pitch) part[c] = s;
        }
        __syncthreads();

        // window sums (fixed order) and the ball test of the projection p_s (Sec. 2.3)
        float scale[CPT];
        int v0[CPT];
        bool near = false;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = t + j * T;
            scale[j] = 1.f;
            v0[j] = 0;
            if (inw[j]) {
                v0[j] = b + ((c - b) / L) * L;
                float ts = 0.f;
                for (int jj = 0; jj < L; ++jj) ts += part[v0[j] + jj];
                if (fabsf(ts - A.cS) <= kNearBand * A.cS) near = true;
                if (ts > A.cS) scale[j] = A.sqrt_cS * rsqrtf(ts);
            }
        }
        if (__syncthreads_or(near)) {
            // rare: some window of this unit lies within the band; redo the
            // sums of squares of those windows in FP64 and take the test there
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int c = t + j * T;
                double s64 = 0.0;
                if (inw[j]) {
#pragma unroll
                    for (int i = 0; i < LB; ++i)
                        if (i < L) s64 = fma((double)xr[i][j], (double)xr[i][j], s64);
                }
                if (c < pitch) s_part64[c] = s64;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                if (!inw[j]) continue;
                float ts = 0.f;
                for (int jj = 0; jj < L; ++jj) ts += part[v0[j] + jj];
                if (fabsf(ts - A.cS) <= kNearBand * A.cS) {
                    double t64 = 0.0;
                    for (int jj = 0; jj < L; ++jj) t64 += s_part64[v0[j] + jj];
                    scale[j] = t64 > A.cS64 ? (float)sqrt(A.cS64 / t64) : 1.f;
                }
            }
        }

        // x = p_s(y), q_s = y - x
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            if (!inw[j]) continue;
            const int c = t + j * T;
#pragma unroll
            for (int i = 0; i < LB; ++i)
                if (i < L) {
                    const float y = xr[i][j];
                    const float xn = y * scale[j];
                    xr[i][j] = xn;
                    qb[(size_t)i * pitch + (c - b)] = y - xn;
                }
        }
    }

#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        const int c = t + j * T;
        if (c < A.W) {
#pragma unroll
            for (int i = 0; i < LB; ++i)
                if (i < L) A.x[(size_t)(r0 + i) * pitch + c] = xr[i][j];
        }
    }
}

template <int LB, int CPT>
cudaError_t launch_group_t(const GroupArgs &A, int threads, cudaStream_t s)
{
    const size_t smem = (size_t)A.pitch * (2 * sizeof(float) + sizeof(double));
    auto k = group_kernel<LB, CPT>;
    // the shared-memory opt-in is a per-device setting of the function: once
    // per device, under a lock (several threads may launch on several devices)
    constexpr int kDevs = 64;
    static std::mutex mu;
    static bool attr_set[kDevs] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev]) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kMaxWidth * (2 * sizeof(float) + sizeof(double))));
            if (e != cudaSuccess) return e;
            attr_set[dev] = true;
        }
    }
    k<<<A.n_units, threads, smem, s>>>(A);
    return cudaGetLastError();
}

constexpr int kNormThreads = 256;
constexpr int kNormBlocks = 512;   // fixed: the reduction order does not depend on the device

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cycle-end norm of Algorithm 2: d^2 = |x - x_prev|^2 and n^2 = |x_prev|^2 in
// FP64, then x_prev <- x.  Rows are strided over blocks, columns over threads.
__global__ void __launch_bounds__(kNormThreads) cycle_norm_kernel(const float *__restrict__ x,
                                                                  float *__restrict__ xp, int H,
                                                                  int W, int pitch,
                                                                  double *__restrict__ partials)
{
    double d = 0.0, n = 0.0;
    for (int r = blockIdx.x; r < H; r += gridDim.x) {
        const float *xr = x + (size_t)r * pitch;
        float *pr = xp + (size_t)r * pitch;
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            const float xv = xr[c], pv = pr[c];
            const double dd = (double)xv - (double)pv;
            d = fma(dd, dd, d);
            n = fma((double)pv, (double)pv, n);
            pr[c] = xv;
        }
    }
    __shared__ double sd[kNormThreads / 32], sn[kNormThreads / 32];
    d = warp_sum(d);
    n = warp_sum(n);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sd[w] = d; sn[w] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double D = 0.0, N = 0.0;
        for (int i = 0; i < kNormThreads / 32; ++i) { D += sd[i]; N += sn[i]; }
        partials[2 * blockIdx.x] = D;
        partials[2 * blockIdx.x + 1] = N;
    }
}

// Stopping test of Algorithm 2 (unsquared L2 change, absolute or relative),
// taken on the device so the host never has to look at the norms.
__global__ void __launch_bounds__(256) decide_kernel(const double *__restrict__ partials,
                                                     int n_blocks, Control *ctl, double *hist,
                                                     int max_cycles, double tol, int tol_relative)
{
    __shared__ double sd[256], sn[256];
    double d = 0.0, n = 0.0;
    for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) {
        d += partials[2 * i];
        n += partials[2 * i + 1];
    }
    sd[threadIdx.x] = d;
    sn[threadIdx.x] = n;
    __syncthreads();
    for (int m = blockDim.x / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m) {
            sd[threadIdx.x] += sd[threadIdx.x + m];
            sn[threadIdx.x] += sn[threadIdx.x + m];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double step = sqrt(sd[0]), prev = sqrt(sn[0]);
        const int cyc = ctl->cycles;
        if (cyc < max_cycles) {
            hist[2 * cyc] = step;
            hist[2 * cyc + 1] = prev;
        }
        ctl->cycles = cyc + 1;
        ctl->step = step;
        ctl->prev_norm = prev;
        // a NaN or Inf in x0 shows in the first cycle's norms (|x_prev| is
        // |x0| there); any non-finite norm ends the run with EINVAL
        const bool bad_in = !isfinite(step) || !isfinite(prev);
        const bool conv = !bad_in && tol >= 0.0 && (tol_relative ? step <= tol * prev : step <= tol);
        const bool cap = cyc + 1 >= max_cycles;
        ctl->stop = (conv || cap || bad_in) ? 1 : 0;
        ctl->status = bad_in ? (int)SMRE_EINVAL
                             : (conv || tol < 0.0 ? (int)SMRE_OK : (int)SMRE_ENOTCONVERGED);
    }
}

// Largest relative violation (t_s - cS) / cS over every window of every side,
// one thread per top-left position; per-block maxima go to partials.
__global__ void __launch_bounds__(256) violation_kernel(const ViolationArgs A,
                                                        double *__restrict__ partials)
{
    double worst = -1e300;
    const long long npx = (long long)A.H * A.W;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
         p += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(p / A.W), c = (int)(p % A.W);
        for (int si = 0; si < A.n_sides; ++si) {
            const int L = A.sides[si];
            if (r + L > A.H || c + L > A.W) continue;
            double t = 0.0;
            for (int i = 0; i < L; ++i) {
                const float *row = A.x + (size_t)(r + i) * A.pitch + c;
                float ts = 0.f;
                for (int j = 0; j < L; ++j) ts = fmaf(row[j], row[j], ts);
                t += ts;
            }
            worst = fmax(worst, (t - A.cS[si]) / A.cS[si]);
        }
    }
    __shared__ double sw[256];
    sw[threadIdx.x] = worst;
    __syncthreads();
    for (int m = blockDim.x / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m) sw[threadIdx.x] = fmax(sw[threadIdx.x], sw[threadIdx.x + m]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sw[0];
}

__global__ void max_reduce_kernel(const double *__restrict__ partials, int n, double *out)
{
    __shared__ double sw[256];
    double w = -1e300;
    for (int i = threadIdx.x; i < n; i += blockDim.x) w = fmax(w, partials[i]);
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int m = blockDim.x / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m) sw[threadIdx.x] = fmax(sw[threadIdx.x], sw[threadIdx.x + m]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sw[0];
}

}  // namespace

int norm_blocks() { return kNormBlocks; }

cudaError_t launch_group(const GroupArgs &A, cudaStream_t s)
{
    if (A.n_units <= 0) return cudaSuccess;
    int cpt = (A.pitch + 1023) / 1024;
    if (cpt > 4) return cudaErrorInvalidValue;
    if (cpt == 3) cpt = 4;
    const int threads = ((A.pitch / cpt) + 31) / 32 * 32;
    if (A.L <= 4) {
        if (cpt == 1) return launch_group_t<4, 1>(A, threads, s);
        if (cpt == 2) return launch_group_t<4, 2>(A, threads, s);
        return launch_group_t<4, 4>(A, threads, s);
    }
    if (A.L <= 8) {
        if (cpt == 1) return launch_group_t<8, 1>(A, threads, s);
        if (cpt == 2) return launch_group_t<8, 2>(A, threads, s);
        return launch_group_t<8, 4>(A, threads, s);
    }
    if (A.L <= 16) {
        if (cpt == 1) return launch_group_t<16, 1>(A, threads, s);
        if (cpt == 2) return launch_group_t<16, 2>(A, threads, s);
        return launch_group_t<16, 4>(A, threads, s);
    }
    if (cpt == 1) return launch_group_t<32, 1>(A, threads, s);
    if (cpt == 2) return launch_group_t<32, 2>(A, threads, s);
    return launch_group_t<32, 4>(A, threads, s);
}

cudaError_t launch_cycle_norm(const float *x, float *xprev, int H, int W, int pitch,
                              double *partials, int n_blocks, cudaStream_t s)
{
    cycle_norm_kernel<<<n_blocks, kNormThreads, 0, s>>>(x, xprev, H, W, pitch, partials);
    return cudaGetLastError();
}

cudaError_t launch_decide(const double *partials, int n_blocks, Control *ctl, double *hist,
                          int max_cycles, double tol, int tol_relative, cudaStream_t s)
{
    decide_kernel<<<1, 256, 0, s>>>(partials, n_blocks, ctl, hist, max_cycles, tol, tol_relative);
    return cudaGetLastError();
}

cudaError_t launch_violation(const ViolationArgs &a, double *partials, int n_blocks,
                             double *out, cudaStream_t s)
{
    violation_kernel<<<n_blocks, 256, 0, s>>>(a, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    max_reduce_kernel<<<1, 256, 0, s>>>(partials, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace smre

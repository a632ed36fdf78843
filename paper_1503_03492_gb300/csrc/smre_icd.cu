// Incomplete Dykstra (Sec. 3.2) on sm_103a.
//
// Pass i covers the image with B x B tiles (B = 2^K) at origins
// (1 << i) mod B + B t, tiles fully inside.  Inside a tile the sets of
// Omega^i are the non-overlapping 2^k x 2^k squares for k = K down to i.  A
// tile runs Dykstra sweeps over these levels until the L1 change of a sweep
// is <= tol * B^2 (at least one sweep, at most max_sweeps); its increments
// start at zero for every pass.
//
// Layout: the B^2 pixels of a tile are numbered in Morton (Z) order, so that
// every aligned 2^k x 2^k square is a contiguous run of 4^k numbers.  Thread
// t of a tile holds the P consecutive pixels tP .. tP + P - 1 together with
// their increments of every level, all in registers; nothing of a tile
// touches shared memory except the cross-warp partial sums of the K = 5
// top level.  A level-k window therefore spans 4^k / P aligned lanes and its
// sum is an xor-butterfly over them (identical in every lane).  Tiles are
// independent and converge at their own pace.
#include <cuda_runtime.h>

#include "smre_internal.h"

namespace smre {

namespace {

constexpr float kNearBand = 1e-6f;

template <int K>
struct IcdShape {
    static constexpr int B = 1 << K;
    static constexpr int NPX = B * B;
    // pixels per thread: K = 3 (8 x 8 tiles) takes 4 -- two tiles a warp, one
    // shuffle step less per level-2 window and per sweep reduction than with
    // 2 (512^2, K 3, tol 1e-3: 185 -> 177 us per call; 8 a thread, 222 us)
    static constexpr int P = K <= 0 ? 1 : (K < 3 ? 2 : K == 3 ? 4 : 8);
    static constexpr int TPT = NPX / P;                               // threads per tile
    static constexpr int TPC = TPT >= 128 ? 1 : 128 / TPT;            // tiles per CTA
    static constexpr int THREADS = TPT * TPC;
    static constexpr int WARPS_PER_TILE = TPT > 32 ? TPT / 32 : 1;
};

// de-interleave the even (column) / odd (row) bits of a Morton number
__device__ __forceinline__ int morton_col(int m)
{
    int c = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) c |= ((m >> (2 * b)) & 1) << b;
    return c;
}
__device__ __forceinline__ int morton_row(int m)
{
    int r = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) r |= ((m >> (2 * b + 1)) & 1) << b;
    return r;
}

// Sum over an aligned group of G lanes (G a power of two <= 32) by xor
// butterfly; every lane of the group ends with the bitwise-same value.
template <typename T>
__device__ __forceinline__ T group_sum(T v, int G, unsigned mask)
{
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int K>
__global__ void __launch_bounds__(IcdShape<K>::THREADS) icd_pass_kernel(const IcdArgs A)
{
    using S = IcdShape<K>;
    constexpr int P = S::P, TPT = S::TPT, B = S::B;
    __shared__ float s_red[S::TPC][S::WARPS_PER_TILE];
    __shared__ double s_red64[S::TPC][S::WARPS_PER_TILE];

    const int tile_in_cta = threadIdx.x / TPT;
    const int tt = threadIdx.x % TPT;                     // thread within tile
    const int tile = blockIdx.x * S::TPC + tile_in_cta;
    const int n_tiles = A.n_ti * A.n_tj;
    if (tile >= n_tiles) return;                          // whole tile leaves together

    const int lane = threadIdx.x & 31;
    // lanes of this tile inside its warp (all 32 when the tile spans warps)
    const unsigned tile_mask =
        TPT >= 32 ? 0xffffffffu : (((1u << TPT) - 1u) << (lane & ~(TPT - 1) & 31));
    const int warp_in_tile = tt >> 5;

    const int ti = tile / A.n_tj, tj = tile % A.n_tj;
    const int r0 = A.off + B * ti, c0 = A.off + B * tj;

    float x[P];
    float q[K + 1][P];
    int gofs[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int m = tt * P + p;
        gofs[p] = (r0 + morton_row(m)) * A.pitch + (c0 + morton_col(m));
        x[p] = A.x[gofs[p]];
#pragma unroll
        for (int k = 0; k <= K; ++k) q[k][p] = 0.f;
    }

    // tiles within one warp: the level-K window is the whole tile, so the next
    // sweep's level-K sum is formed while this sweep's change is reduced over
    // the same lanes (two independent butterflies, each with the operations
    // and order it has on its own)
    constexpr bool kAheadK = TPT <= 32;
    float tK = 0.f;
    bool have_tK = false;
    int sweeps = 0;
    bool done = false;
    while (!done) {
        float delta = 0.f;
#pragma unroll
        for (int k = K; k >= 0; --k) {
            if (k < A.pass) break;
            const int wpx = 1 << (2 * k);                 // pixels of a level-k window
            float y[P];
#pragma unroll
            for (int p = 0; p < P; ++p) y[p] = x[p] + q[k][p];

            // window sums of y^2
            float tsum[P];
            if (kAheadK && k == K && have_tK) {
#pragma unroll
                for (int p = 0; p < P; ++p) tsum[p] = tK;
            } else if (wpx <= P) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const int w0 = (p / wpx) * wpx;
                    float s = 0.f;
                    for (int e = 0; e < wpx; ++e) s = fmaf(y[w0 + e], y[w0 + e], s);
                    tsum[p] = s;
                }
            } else {
                float s = 0.f;
#pragma unroll
                for (int p = 0; p < P; ++p) s = fmaf(y[p], y[p], s);
                const int lanes = wpx / P;
                if (lanes <= 32) {
                    const unsigned gmask = lanes >= 32 ? 0xffffffffu
                                                       : (((1u << lanes) - 1u) << (lane & ~(lanes - 1) & 31));
                    s = group_sum(s, lanes, gmask);
                } else {
                    s = group_sum(s, 32, 0xffffffffu);
                    if (lane == 0) s_red[tile_in_cta][warp_in_tile] = s;
                    __syncthreads();
                    float tot = 0.f;
                    for (int w = 0; w < S::WARPS_PER_TILE; ++w) tot += s_red[tile_in_cta][w];
                    __syncthreads();
                    s = tot;
                }
#pragma unroll
                for (int p = 0; p < P; ++p) tsum[p] = s;
            }

            // ball test, scale sqrt(cS) rsqrt(t) as in the standard kernels (a
            // tile's sweeps are one dependent chain, and an IEEE division plus
            // square root per level doubled its length); FP64 recheck of
            // windows whose sum lies near cS
            const float c = A.cS[k];
            float scale[P];
            bool near_any = false;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                scale[p] = tsum[p] > c ? A.sqrt_cS[k] * rsqrtf(tsum[p]) : 1.f;
                near_any |= fabsf(tsum[p] - c) <= kNearBand * c;
            }
            if (wpx <= P) {
                if (near_any) {
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (fabsf(tsum[p] - c) > kNearBand * c) continue;
                        const int w0 = (p / wpx) * wpx;
                        double s = 0.0;
                        for (int e = 0; e < wpx; ++e) s = fma((double)y[w0 + e], (double)y[w0 + e], s);
                        scale[p] = s > A.cS64[k] ? (float)sqrt(A.cS64[k] / s) : 1.f;
                    }
                }
            } else {
                const int lanes = wpx / P;
                // near_any is uniform over the window's lanes (same sum)
                if (lanes <= 32) {
                    if (near_any) {
                        const unsigned gmask = lanes >= 32 ? 0xffffffffu
                                                           : (((1u << lanes) - 1u) << (lane & ~(lanes - 1) & 31));
                        double s = 0.0;
#pragma unroll
                        for (int p = 0; p < P; ++p) s = fma((double)y[p], (double)y[p], s);
                        s = group_sum(s, lanes, gmask);
                        const float sc = s > A.cS64[k] ? (float)sqrt(A.cS64[k] / s) : 1.f;
#pragma unroll
                        for (int p = 0; p < P; ++p) scale[p] = sc;
                    }
                } else {
                    // the window is the whole multi-warp tile: near_any is tile-uniform
                    if (near_any) {
                        double s = 0.0;
#pragma unroll
                        for (int p = 0; p < P; ++p) s = fma((double)y[p], (double)y[p], s);
                        s = group_sum(s, 32, 0xffffffffu);
                        if (lane == 0) s_red64[tile_in_cta][warp_in_tile] = s;
                        __syncthreads();
                        double tot = 0.0;
                        for (int w = 0; w < S::WARPS_PER_TILE; ++w) tot += s_red64[tile_in_cta][w];
                        __syncthreads();
                        const float sc = tot > A.cS64[k] ? (float)sqrt(A.cS64[k] / tot) : 1.f;
#pragma unroll
                        for (int p = 0; p < P; ++p) scale[p] = sc;
                    }
                }
            }

            // x = p_s(y), q_s = y - x, delta += |x_old - x_new|
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float xn = y[p] * scale[p];
                delta += fabsf(x[p] - xn);
                q[k][p] = y[p] - xn;
                x[p] = xn;
            }
        }
        ++sweeps;

        // tile-wide L1 change of the sweep
        float dtile;
        if (kAheadK) {
            float s = 0.f;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float yk = x[p] + q[K][p];
                s = fmaf(yk, yk, s);
            }
            float d = delta;
            for (int o = TPT >> 1; o > 0; o >>= 1) {
                d += __shfl_xor_sync(tile_mask, d, o);
                s += __shfl_xor_sync(tile_mask, s, o);
            }
            dtile = d;
            tK = s;
            have_tK = true;
        } else {
            float s = group_sum(delta, 32, 0xffffffffu);
            if (lane == 0) s_red[tile_in_cta][warp_in_tile] = s;
            __syncthreads();
            dtile = 0.f;
            for (int w = 0; w < S::WARPS_PER_TILE; ++w) dtile += s_red[tile_in_cta][w];
            __syncthreads();
        }
        done = !(dtile > A.tol_b2) || sweeps >= A.max_sweeps;
    }

#pragma unroll
    for (int p = 0; p < P; ++p) A.x[gofs[p]] = x[p];
    if (tt == 0) A.sweeps[tile] = sweeps;
}

template <int K>
cudaError_t launch_icd_t(const IcdArgs &A, cudaStream_t s)
{
    using S = IcdShape<K>;
    const int n_tiles = A.n_ti * A.n_tj;
    if (n_tiles <= 0) return cudaSuccess;
    const int blocks = (n_tiles + S::TPC - 1) / S::TPC;
    icd_pass_kernel<K><<<blocks, S::THREADS, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_icd_pass(const IcdArgs &A, cudaStream_t s)
{
    switch (A.K) {
        case 0: return launch_icd_t<0>(A, s);
        case 1: return launch_icd_t<1>(A, s);
        case 2: return launch_icd_t<2>(A, s);
        case 3: return launch_icd_t<3>(A, s);
        case 4: return launch_icd_t<4>(A, s);
        case 5: return launch_icd_t<5>(A, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smre

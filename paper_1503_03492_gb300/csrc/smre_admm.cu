// ADMM outer loop of the multi-resolution estimator (smre_admm_* of
// include/smre.h; Sec. 2.2, Algorithm 1 on the split problem of Eq. 3).
//
// One iteration is five kinds of launch on the handle's stream:
//   xstep  : A(rho1 (I - A x - eps) + Y1) by a 32 x 32 tile with its halo in
//            shared memory (the blurred argument is formed while the tile is
//            loaded), then the x-step in the epilogue, and the block's share
//            of |x_new - x|^2 (FP64);
//   blur   : A x_new (tile + halo), kept for the next iteration's x-step, and
//            the projection's input s = I - A x_new + Y1 / rho1;
//   the eps-step: smre_dykstra_project(s -> eps) on the owned projection handle
//            (or its incomplete variant, smre_dykstra_project_incomplete);
//   tv     : up to four projected-gradient steps on the dual of the TV prox
//            per launch (tile with a four-pixel halo of p and f = x + Y2 / rho2
//            in shared memory), ping-pong buffers between launches;
//   final  : z = f - D^T p / rho2, the multiplier steps and the block's share
//            of |I - A x - eps|^2 (FP64).
// The block partial sums are added on the host in block order, so the norms
// (and the stopping decision) do not depend on scheduling.  Every pass over
// an image is a bandwidth-bound stencil (a few flops per byte); the images
// of a 512 x 512 problem (1 MB each) stay in L2 between the launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "smre_internal.h"

namespace smre {
namespace {

constexpr int kTile = 32;            // output tile (pixels per side)
constexpr int kRows = 8;             // threads per tile column (block 32 x 8)
constexpr int kMaxR = 16;            // largest PSF radius
constexpr int kSpan = kTile + 2 * kMaxR;
constexpr int kTvSteps = 4;          // TV dual steps per launch (halo of the tile)

struct AdmmArgs {
    const float *I;
    float *x, *z, *eps, *Y1, *Y2, *Ax, *s;
    const float *p1, *p2;            // TV dual, read
    float *p1n, *p2n;                // TV dual, written (tv step)
    double *part;                    // one partial sum per block
    int H, W, r;
    int tv_steps;                    // steps of this tv launch (1..kTvSteps)
    float rho1, rho2, inv_rho1, inv_rho2, inv_gamma, tau;
    float w[2 * kMaxR + 1];          // PSF weights per axis, k = -r..r
};

// Sum of a double over the block, written by thread 0 to part[block].
__device__ void block_partial(double v, double *part)
{
    __shared__ double red[kRows];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[threadIdx.y] = v;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double t = 0.0;
        for (int k = 0; k < kRows; ++k) t += red[k];
        part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// The separable blur of the (32 + 2r)^2 input tile `tin` into out[kTile/kRows]
// (this thread's pixels (ty + kRows k, tx)): rows first, then columns, taps in
// the order k = -r..r.
__device__ void blur_tile(const AdmmArgs &A, float (*tin)[kSpan + 1], float (*trow)[kTile + 1],
                          float out[kTile / kRows])
{
    const int tx = threadIdx.x, ty = threadIdx.y, r = A.r, span = kTile + 2 * r;
    for (int ii = ty; ii < span; ii += kRows) {
        float acc = 0.f;
        for (int t = 0; t <= 2 * r; ++t) acc = fmaf(A.w[t], tin[ii][tx + t], acc);
        trow[ii][tx] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTile / kRows; ++k) {
        const int i = ty + kRows * k;
        float acc = 0.f;
        for (int t = 0; t <= 2 * r; ++t) acc = fmaf(A.w[t], trow[i + t][tx], acc);
        out[k] = acc;
    }
}

// x <- x - (1/gamma) [ -A(rho1 (I - A x - eps) + Y1) + rho2 (x - z) + Y2 ]
__global__ void __launch_bounds__(kTile * kRows) xstep_kernel(const AdmmArgs A)
{
    __shared__ float tin[kSpan][kSpan + 1];
    __shared__ float trow[kSpan][kTile + 1];
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile, r = A.r, span = kTile + 2 * r;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    for (int e = tid; e < span * span; e += kTile * kRows) {
        const int ii = e / span, jj = e - ii * span;
        const int gi = i0 - r + ii, gj = j0 - r + jj;
        float v = 0.f;   // the blurred argument is zero outside the image
        if (gi >= 0 && gi < A.H && gj >= 0 && gj < A.W) {
            const size_t g = (size_t)gi * A.W + gj;
            v = fmaf(A.rho1, (A.I[g] - A.Ax[g]) - A.eps[g], A.Y1[g]);
        }
        tin[ii][jj] = v;
    }
    __syncthreads();
    float v[kTile / kRows];
    blur_tile(A, tin, trow, v);
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < kTile / kRows; ++k) {
        const int gi = i0 + threadIdx.y + kRows * k, gj = j0 + threadIdx.x;
        if (gi < A.H && gj < A.W) {
            const size_t g = (size_t)gi * A.W + gj;
            const float xo = A.x[g];
            const float grad = fmaf(A.rho2, xo - A.z[g], A.Y2[g]) - v[k];
            const float xn = xo - grad * A.inv_gamma;
            A.x[g] = xn;
            const double d = (double)xn - (double)xo;
            d2 = fma(d, d, d2);
        }
    }
    block_partial(d2, A.part);
}

// Ax <- A x;  s <- I - A x + Y1 / rho1
__global__ void __launch_bounds__(kTile * kRows) blur_kernel(const AdmmArgs A)
{
    __shared__ float tin[kSpan][kSpan + 1];
    __shared__ float trow[kSpan][kTile + 1];
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile, r = A.r, span = kTile + 2 * r;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    for (int e = tid; e < span * span; e += kTile * kRows) {
        const int ii = e / span, jj = e - ii * span;
        const int gi = i0 - r + ii, gj = j0 - r + jj;
        tin[ii][jj] = gi >= 0 && gi < A.H && gj >= 0 && gj < A.W ? A.x[(size_t)gi * A.W + gj] : 0.f;
    }
    __syncthreads();
    float v[kTile / kRows];
    blur_tile(A, tin, trow, v);
#pragma unroll
    for (int k = 0; k < kTile / kRows; ++k) {
        const int gi = i0 + threadIdx.y + kRows * k, gj = j0 + threadIdx.x;
        if (gi < A.H && gj < A.W) {
            const size_t g = (size_t)gi * A.W + gj;
            A.Ax[g] = v[k];
            A.s[g] = fmaf(A.Y1[g], A.inv_rho1, A.I[g] - v[k]);
        }
    }
}

// (D^T p) at (i, j) from a tile of p with a one-pixel halo above / left
__device__ __forceinline__ float dtp(float a_up, float a, float b_left, float b, int i, int j, int H, int W)
{
    float o = 0.f;
    if (i <= H - 2) o -= a;
    if (i >= 1) o += a_up;
    if (j <= W - 2) o -= b;
    if (j >= 1) o += b_left;
    return o;
}

// tv_steps (1..kTvSteps) steps of p <- clip(p + tau D(f - D^T p / rho2), -1, 1),
// f = x + Y2 / rho2, in one launch: the block loads p and f on its tile with a
// kTvSteps-pixel halo and runs the steps in shared memory; each step needs
// the previous one's p within one pixel, so the region still exact shrinks by
// one pixel a side per step and the tile itself stays exact.  Every value is
// computed with the same operations as by one launch per step.
__global__ void __launch_bounds__(kTile * kRows) tv_kernel(const AdmmArgs A)
{
    constexpr int R = kTile + 2 * kTvSteps;
    __shared__ float P1[2][R][R + 1], P2[2][R][R + 1];
    __shared__ float F[R][R + 1], T[R][R + 1];
    const int i0 = blockIdx.y * kTile - kTvSteps, j0 = blockIdx.x * kTile - kTvSteps;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    const int H = A.H, W = A.W;
    for (int e = tid; e < R * R; e += kTile * kRows) {
        const int u = e / R, v = e - u * R;
        const int gi = i0 + u, gj = j0 + v;
        const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
        const size_t g = in ? (size_t)gi * W + gj : 0;
        P1[0][u][v] = in ? A.p1[g] : 0.f;   // p is zero outside the image
        P2[0][u][v] = in ? A.p2[g] : 0.f;
        F[u][v] = in ? fmaf(A.Y2[g], A.inv_rho2, A.x[g]) : 0.f;
    }
    __syncthreads();
    int c = 0;
    for (int st = 1; st <= A.tv_steps; ++st) {
        // p is exact on [st - 1, R - st + 1); t = f - D^T p / rho2 on [st, R - st + 1)
        const int lo = st, hi = R - st + 1, n = hi - lo;
        for (int e = tid; e < n * n; e += kTile * kRows) {
            const int u = lo + e / n, v = lo + e % n;
            const int gi = i0 + u, gj = j0 + v;
            float t = 0.f;
            if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
                const float d = dtp(P1[c][u - 1][v], P1[c][u][v], P2[c][u][v - 1], P2[c][u][v], gi, gj, H, W);
                t = F[u][v] - d * A.inv_rho2;
            }
            T[u][v] = t;
        }
        __syncthreads();
        // the new p on [st, R - st)
        const int m = n - 1;
        for (int e = tid; e < m * m; e += kTile * kRows) {
            const int u = lo + e / m, v = lo + e % m;
            const int gi = i0 + u, gj = j0 + v;
            float a = 0.f, b = 0.f;
            if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
                const float tc = T[u][v];
                const float g1 = gi <= H - 2 ? T[u + 1][v] - tc : 0.f;
                const float g2 = gj <= W - 2 ? T[u][v + 1] - tc : 0.f;
                a = fminf(1.f, fmaxf(-1.f, fmaf(A.tau, g1, P1[c][u][v])));
                b = fminf(1.f, fmaxf(-1.f, fmaf(A.tau, g2, P2[c][u][v])));
            }
            P1[c ^ 1][u][v] = a;
            P2[c ^ 1][u][v] = b;
        }
        __syncthreads();
        c ^= 1;
    }
#pragma unroll
    for (int k = 0; k < kTile / kRows; ++k) {
        const int u = kTvSteps + threadIdx.y + kRows * k, v = kTvSteps + threadIdx.x;
        const int gi = i0 + u, gj = j0 + v;
        if (gi < H && gj < W) {
            const size_t g = (size_t)gi * W + gj;
            A.p1n[g] = P1[c][u][v];
            A.p2n[g] = P2[c][u][v];
        }
    }
}

// z <- f - D^T p / rho2;  Y1 += rho1 (I - A x - eps);  Y2 += rho2 (x - z)
__global__ void __launch_bounds__(kTile * kRows) final_kernel(const AdmmArgs A)
{
    const int H = A.H, W = A.W;
    double r2 = 0.0;
#pragma unroll
    for (int k = 0; k < kTile / kRows; ++k) {
        const int gi = blockIdx.y * kTile + threadIdx.y + kRows * k, gj = blockIdx.x * kTile + threadIdx.x;
        if (gi < H && gj < W) {
            const size_t g = (size_t)gi * W + gj;
            const float a_up = gi >= 1 ? A.p1[g - W] : 0.f;
            const float b_left = gj >= 1 ? A.p2[g - 1] : 0.f;
            const float x = A.x[g], y2 = A.Y2[g];
            const float f = fmaf(y2, A.inv_rho2, x);
            const float z = f - dtp(a_up, A.p1[g], b_left, A.p2[g], gi, gj, H, W) * A.inv_rho2;
            const float res = (A.I[g] - A.Ax[g]) - A.eps[g];
            A.z[g] = z;
            A.Y1[g] = fmaf(A.rho1, res, A.Y1[g]);
            A.Y2[g] = fmaf(A.rho2, x - z, y2);
            r2 = fma((double)res, (double)res, r2);
        }
    }
    block_partial(r2, A.part);
}

thread_local std::string g_admm_err;

}  // namespace
}  // namespace smre

using namespace smre;

struct smre_admm {
    int H = 0, W = 0;
    smre_dykstra *proj = nullptr;
    cudaStream_t stream = nullptr;
    smre_admm_params ap{};
    AdmmArgs base{};
    float *buf = nullptr;            // the solver's planes
    float *x = nullptr, *z = nullptr, *eps = nullptr, *Y1 = nullptr, *Y2 = nullptr;
    float *Ax = nullptr, *s = nullptr, *p1[2] = {nullptr, nullptr}, *p2[2] = {nullptr, nullptr};
    double *d_part = nullptr;        // [2][blocks]: |dx|^2 and residual^2 partials
    double *h_part = nullptr;        // pinned copy
    int blocks = 0;
    long long launches = 0;
    std::string err;
};

namespace {

smre_status afail(smre_admm *a, smre_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    (a ? a->err : g_admm_err) = buf;
    return s;
}

#define ACK(a, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return afail((a), e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA,     \
                         "%s: %s", #call, cudaGetErrorString(e_));                            \
    } while (0)

// The solver's kernels read and write its images directly: each must be
// device (or managed) memory, checked on the host so that a host pointer is
// an EINVAL and not a fault.
bool device_image(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void release(smre_admm *a)
{
    if (!a) return;
    if (a->stream) cudaStreamSynchronize(a->stream);
    cudaFree(a->buf);
    cudaFree(a->d_part);
    cudaFreeHost(a->h_part);
    smre_dykstra_destroy(a->proj);
    delete a;
}

}  // namespace

extern "C" {

smre_status smre_admm_create(const smre_params *proj, const smre_admm_params *ap, void *cuda_stream,
                             smre_admm **out)
{
    const AllocScope scope;
    if (!out || !proj || !ap) return afail(nullptr, SMRE_EINVAL, "proj / ap / out is NULL");
    *out = nullptr;
    if (!(ap->sigma > 0.0) || !std::isfinite(ap->sigma))
        return afail(nullptr, SMRE_EINVAL, "sigma must be > 0");
    const int r = ap->radius > 0 ? ap->radius : (int)std::ceil(3.0 * ap->sigma);
    if (r < 1 || r > kMaxR) return afail(nullptr, SMRE_EINVAL, "PSF radius %d outside 1..%d", r, kMaxR);
    if (!(ap->rho1 > 0.0) || !(ap->rho2 > 0.0) || !std::isfinite(ap->rho1) || !std::isfinite(ap->rho2))
        return afail(nullptr, SMRE_EINVAL, "rho1 and rho2 must be > 0");
    if (ap->tv_iters < 0) return afail(nullptr, SMRE_EINVAL, "tv_iters must be >= 0");
    if (ap->max_iters < 1) return afail(nullptr, SMRE_EINVAL, "max_iters must be >= 1");
    if (std::isnan(ap->delta) || std::isnan(ap->gamma)) return afail(nullptr, SMRE_EINVAL, "delta / gamma is NaN");
    if (ap->eps_incomplete && !(ap->icd_tol >= 0.0))
        return afail(nullptr, SMRE_EINVAL, "icd_tol must be >= 0");
    const double gamma = ap->gamma > 0.0 ? ap->gamma : 1.01 * (ap->rho1 + ap->rho2);
    if (gamma < ap->rho1 + ap->rho2)
        return afail(nullptr, SMRE_EINVAL, "gamma %g below rho1 + rho2 = %g (the x-step would not converge)",
                     gamma, ap->rho1 + ap->rho2);

    smre_admm *a = new (std::nothrow) smre_admm;
    if (!a) return afail(nullptr, SMRE_ENOMEM, "out of host memory");
    a->stream = (cudaStream_t)cuda_stream;
    a->ap = *ap;
    a->ap.radius = r;
    a->ap.gamma = gamma;
    smre_status st = smre_dykstra_create(proj, cuda_stream, &a->proj);
    if (st != SMRE_OK) {
        afail(nullptr, st, "projection handle: %s", smre_last_error(nullptr));
        release(a);
        return st;
    }
    a->H = proj->height;
    a->W = proj->width;
    const size_t n = (size_t)a->H * a->W;
    const int gx = (a->W + kTile - 1) / kTile, gy = (a->H + kTile - 1) / kTile;
    a->blocks = gx * gy;
    cudaError_t e = dev_malloc(&a->buf, sizeof(float) * n * 11);
    if (e == cudaSuccess) e = dev_malloc(&a->d_part, sizeof(double) * 2 * a->blocks);
    if (e == cudaSuccess) e = host_malloc(&a->h_part, sizeof(double) * 2 * a->blocks);
    if (e != cudaSuccess) {
        afail(nullptr, e == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA, "allocation: %s",
              cudaGetErrorString(e));
        release(a);
        return e == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA;
    }
    float *p = a->buf;
    for (float **q : {&a->x, &a->z, &a->eps, &a->Y1, &a->Y2, &a->Ax, &a->s, &a->p1[0], &a->p1[1],
                      &a->p2[0], &a->p2[1]}) {
        *q = p;
        p += n;
    }
    // PSF weights (FP64, normalised), rounded once to FP32
    std::vector<double> w(2 * r + 1);
    double sum = 0.0;
    for (int k = -r; k <= r; ++k) sum += (w[k + r] = std::exp(-(double)k * k / (2.0 * ap->sigma * ap->sigma)));
    AdmmArgs &B = a->base;
    B.H = a->H;
    B.W = a->W;
    B.r = r;
    for (int t = 0; t <= 2 * r; ++t) B.w[t] = (float)(w[t] / sum);
    B.rho1 = (float)ap->rho1;
    B.rho2 = (float)ap->rho2;
    B.inv_rho1 = (float)(1.0 / ap->rho1);
    B.inv_rho2 = (float)(1.0 / ap->rho2);
    B.inv_gamma = (float)(1.0 / gamma);
    B.tau = (float)(ap->rho2 / 8.0);
    *out = a;
    return SMRE_OK;
}

smre_status smre_admm_solve(smre_admm *a, const float *I, float *x, float *z, float *eps,
                            smre_admm_result *res)
{
    if (!a) return afail(nullptr, SMRE_EINVAL, "solver is NULL");
    if (!I || !x) return afail(a, SMRE_EINVAL, "I / x is NULL");
    if (!device_image(I) || !device_image(x) || (z && !device_image(z)) || (eps && !device_image(eps)))
        return afail(a, SMRE_EINVAL, "I, x, z and eps must be device images");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t n = (size_t)a->H * a->W;
    ACK(a, cudaMemsetAsync(a->buf, 0, sizeof(float) * n * 11, a->stream));
    const dim3 grid((a->W + kTile - 1) / kTile, (a->H + kTile - 1) / kTile), block(kTile, kRows);
    AdmmArgs A = a->base;
    A.I = I;
    A.x = a->x;
    A.z = a->z;
    A.eps = a->eps;
    A.Y1 = a->Y1;
    A.Y2 = a->Y2;
    A.Ax = a->Ax;
    A.s = a->s;
    int cur = 0;             // TV dual buffer holding the current p
    int it = 0;
    double dx = 0.0, rr = 0.0, proj_s = 0.0;
    long long cycles = 0;
    smre_status status = SMRE_OK;
    while (it < a->ap.max_iters) {
        A.part = a->d_part;
        xstep_kernel<<<grid, block, 0, a->stream>>>(A);
        blur_kernel<<<grid, block, 0, a->stream>>>(A);
        ACK(a, cudaGetLastError());
        a->launches += 2;
        smre_result pr{};
        const smre_status ps = a->ap.eps_incomplete
                                   ? smre_dykstra_project_incomplete(a->proj, a->s, a->eps, a->ap.icd_K,
                                                                     a->ap.icd_tol, &pr)
                                   : smre_dykstra_project(a->proj, a->s, a->eps, &pr);
        if (ps != SMRE_OK && ps != SMRE_ENOTCONVERGED)
            return afail(a, ps, "eps-step (projection): %s", smre_last_error(a->proj));
        cycles += pr.cycles;
        proj_s += pr.seconds;
        int tv_launches = 0;
        for (int k = 0; k < a->ap.tv_iters; k += kTvSteps) {
            A.tv_steps = std::min(kTvSteps, a->ap.tv_iters - k);
            A.p1 = a->p1[cur];
            A.p2 = a->p2[cur];
            A.p1n = a->p1[cur ^ 1];
            A.p2n = a->p2[cur ^ 1];
            tv_kernel<<<grid, block, 0, a->stream>>>(A);
            cur ^= 1;
            ++tv_launches;
        }
        A.p1 = a->p1[cur];
        A.p2 = a->p2[cur];
        A.part = a->d_part + a->blocks;
        final_kernel<<<grid, block, 0, a->stream>>>(A);
        ACK(a, cudaGetLastError());
        a->launches += tv_launches + 1;
        ++it;
        // the norms are needed every iteration only for the stopping test;
        // with a fixed count they are read once, after the last iteration
        if (a->ap.delta >= 0.0 || it == a->ap.max_iters) {
            ACK(a, cudaMemcpyAsync(a->h_part, a->d_part, sizeof(double) * 2 * a->blocks,
                                   cudaMemcpyDeviceToHost, a->stream));
            ACK(a, cudaStreamSynchronize(a->stream));
            double d2 = 0.0, r2 = 0.0;
            for (int b = 0; b < a->blocks; ++b) {
                d2 += a->h_part[b];
                r2 += a->h_part[a->blocks + b];
            }
            dx = std::sqrt(d2);
            rr = std::sqrt(r2);
            if (a->ap.delta >= 0.0 && dx <= a->ap.delta && rr <= a->ap.delta) break;
        }
    }
    if (a->ap.delta >= 0.0 && !(dx <= a->ap.delta && rr <= a->ap.delta)) status = SMRE_ENOTCONVERGED;
    ACK(a, cudaMemcpyAsync(x, a->x, sizeof(float) * n, cudaMemcpyDeviceToDevice, a->stream));
    if (z) ACK(a, cudaMemcpyAsync(z, a->z, sizeof(float) * n, cudaMemcpyDeviceToDevice, a->stream));
    if (eps) ACK(a, cudaMemcpyAsync(eps, a->eps, sizeof(float) * n, cudaMemcpyDeviceToDevice, a->stream));
    ACK(a, cudaStreamSynchronize(a->stream));
    if (res) {
        res->iters = it;
        res->status = status;
        res->dx = dx;
        res->residual = rr;
        res->dykstra_cycles = cycles;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        res->projection_seconds = proj_s;
    }
    return status;
}

long long smre_admm_kernel_launches(const smre_admm *a) { return a ? a->launches : 0; }

smre_dykstra *smre_admm_projector(smre_admm *a) { return a ? a->proj : nullptr; }

void smre_admm_destroy(smre_admm *a) { release(a); }

const char *smre_admm_last_error(const smre_admm *a) { return a ? a->err.c_str() : g_admm_err.c_str(); }

}  // extern "C"

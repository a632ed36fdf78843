// Norm and stopping-test kernels of the batched path, and the dispatch of the
// step kernel (built once per increment type in smre_batch_f32.cu,
// smre_batch_bf16.cu and smre_batch_f16.cu from smre_batch_kernel.cuh).
#include <cuda_runtime.h>

#include "smre_batch_kernel.cuh"

namespace smre {

namespace {

using batch::kNormThreads;
using batch::find_active;

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
        // a NaN or Inf in x0 shows in the first cycle's norms (|x_prev| is
        // |x0| there); any non-finite norm ends the image's run with EINVAL
        const bool bad_in = !isfinite(step) || !isfinite(prev);
        const bool conv = !bad_in && A.tol >= 0.0 &&
                          (A.tol_relative ? step <= A.tol * prev : step <= A.tol);
        const bool cap = cyc + 1 >= A.max_cycles;
        ctl->status = bad_in ? (int)SMRE_EINVAL
                             : (conv || A.tol < 0.0 ? (int)SMRE_OK : (int)SMRE_ENOTCONVERGED);
        ctl->stop = (conv || cap || bad_in) ? 1 : 0;
    }
}

}  // namespace

int batch_lb(int L) { return batch::lb_of(L); }
int batch_virtual_width(int L) { return batch::vw_of(batch::lb_of(L)); }
// column sums, the FP64 recheck and the window factors: 16 bytes a virtual
// column with FP32 increments, 20 with 16-bit ones
size_t batch_part_bytes(int L, int qtype)
{
    return (size_t)batch::vw_of(batch::lb_of(L)) * (qtype == 0 ? 16 : 20);
}
int batch_threads() { return batch::kThreads; }

cudaError_t batch_prepare(int qtype, size_t smem_max)
{
    if (qtype == 1) return batch_prepare_bf16(smem_max);
    if (qtype == 2) return batch_prepare_f16(smem_max);
    return batch_prepare_f32(smem_max);
}

cudaError_t launch_batch_step(int qtype, const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    if (A.max_items <= 0 || grid <= 0) return cudaSuccess;
    if (qtype == 1) return launch_batch_step_bf16(A, grid, smem, s);
    if (qtype == 2) return launch_batch_step_f16(A, grid, smem, s);
    return launch_batch_step_f32(A, grid, smem, s);
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

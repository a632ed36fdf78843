// Step kernels of the batched path with __nv_bfloat16 increments (one translation
// unit per increment type, so the three sets compile in parallel).
#include "smre_batch_kernel.cuh"

namespace smre {

cudaError_t launch_batch_step_bf16(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    return batch::launch_step_q<__nv_bfloat16>(A, grid, smem, s);
}

cudaError_t batch_prepare_bf16(size_t smem)
{
    return batch::prepare_q<__nv_bfloat16>(smem);
}

}  // namespace smre

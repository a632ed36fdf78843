// Step kernels of the batched path with __half increments (one translation
// unit per increment type, so the three sets compile in parallel).
#include "smre_batch_kernel.cuh"

namespace smre {

cudaError_t launch_batch_step_f16(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    return batch::launch_step_q<__half>(A, grid, smem, s);
}

cudaError_t batch_prepare_f16(size_t smem)
{
    return batch::prepare_q<__half>(smem);
}

}  // namespace smre

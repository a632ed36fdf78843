// Step kernels of the batched path with float increments (one translation
// unit per increment type, so the three sets compile in parallel).
#include "smre_batch_kernel.cuh"

namespace smre {

cudaError_t launch_batch_step_f32(const BStepArgs &A, int grid, size_t smem, cudaStream_t s)
{
    return batch::launch_step_q<float>(A, grid, smem, s);
}

cudaError_t batch_prepare_f32(size_t smem)
{
    return batch::prepare_q<float>(smem);
}

}  // namespace smre

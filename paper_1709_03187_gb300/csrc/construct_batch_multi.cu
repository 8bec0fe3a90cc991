// construct_batch_multi.cu -- the batched construction schedules with several ants (warps) per
// block (the one-ant schedules are in construct_batch.cu).
#include "construct_dev.cuh"

cudaError_t launch_construct_batch_multi(const BatchMap& B, int config, int blocks, size_t smem, cudaStream_t s) {
    switch (config) {
        case 4: return launch_batch_schedule<2, 8>(B, blocks, smem, s);
        case 5: return launch_batch_schedule<2, 16>(B, blocks, smem, s);
        case 6: return launch_batch_schedule<4, 4>(B, blocks, smem, s);
        case 7: return launch_batch_schedule<4, 8>(B, blocks, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

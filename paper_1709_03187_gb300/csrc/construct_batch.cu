// construct_batch.cu -- batched colonies: one construction launch over every colony's ants
// (device code in construct_dev.cuh).  Schedules of one ant per block are instantiated here, those
// of several ants per block in construct_batch_multi.cu, and the persistent launch is in
// construct_persist.cu, so that the units compile in parallel.
#include "construct_dev.cuh"

// Batched launch schedules: (ants per block, minimum resident blocks per SM).  The second
// number caps the registers per thread (65536 / (32 * ants * blocks)), trading register spills
// for more concurrent ant chains.
extern const int kBatchConfigs[ACO_BATCH_CONFIGS][2] = {{1, 8}, {1, 16}, {1, 24}, {1, 32}, {2, 8}, {2, 16}, {4, 4}, {4, 8}};

cudaError_t launch_construct_batch_multi(const BatchMap& B, int config, int blocks, size_t smem, cudaStream_t s);

cudaError_t launch_construct_batch(const LbestArgs* args, const int2* slot, const int* iteration, int slots,
                                   int smem_per_ant, int config, cudaStream_t s) {
    if (config < 0 || config >= ACO_BATCH_CONFIGS) return cudaErrorInvalidValue;
    BatchMap B{args, slot, iteration, slots, smem_per_ant};
    const int warps = kBatchConfigs[config][0];
    const size_t smem = (size_t)smem_per_ant * warps;
    const int blocks = (slots + warps - 1) / warps;
    switch (config) {
        case 0: return launch_batch_schedule<1, 8>(B, blocks, smem, s);
        case 1: return launch_batch_schedule<1, 16>(B, blocks, smem, s);
        case 2: return launch_batch_schedule<1, 24>(B, blocks, smem, s);
        case 3: return launch_batch_schedule<1, 32>(B, blocks, smem, s);
        default: return launch_construct_batch_multi(B, config, blocks, smem, s);
    }
}

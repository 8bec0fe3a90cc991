// construct_persist.cu -- batched colonies: the persistent launch of whole iterations (device
// code of the construction in construct_dev.cuh).
#include "construct_dev.cuh"

// ------------------------------------------------------------------ persistent batched kernel
// Every iteration of a batch in one launch: the resident warps pull (instance, ant) slots from a
// device work queue and construct them, then -- after a grid-wide barrier -- pull slots again to
// commit, then update every colony's C_gbest and weights, then pull chunks of cities (whole
// blocks) for the pheromone rebuild, and after a last barrier start the next iteration.  The
// launch is cooperative, so every block is resident and the barriers can complete.  Every
// barrier wait is bounded by wait_ns: a block that waits longer sets bit 0 of *status and
// leaves, and so does every block that passes a barrier after that, so the launch always ends;
// the host then reports ACO_ERR_TIMEOUT.  Each ant's work is the same deterministic function of
// the colony state as in the four-launch iteration, so the schedule changes no result.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait; false when this block or another one gave up.
__device__ bool grid_barrier(const PersistArgs& P) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = P.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(P.bar, 1u) == gridDim.x - 1) {
            atomicExch(P.bar, 0u);
            __threadfence();
            atomicAdd(P.bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > P.wait_ns) {
                    atomicOr(P.status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        if (*reinterpret_cast<volatile int*>(P.status) & 1) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// The integer pheromone of city i's candidate edges from its rank row (lane-private histogram
// columns, then lane r sums rank r), and the row's weights.
__device__ __forceinline__ void rebuild_city(const RebuildArgs& R, int i, const unsigned long long* qs,
                                             unsigned long long* hist, int lane) {
    const int m = R.use_ants ? R.m : 0, k = R.k;
    for (int r = 0; r < k; ++r) hist[r * 32 + lane] = 0ull;
    const uint8_t* row = R.nbrank + (size_t)i * R.m * 2;
    for (int b = lane; b < 2 * m; b += 32) {
        const uint32_t r = row[b];
        if (r < (uint32_t)k) hist[r * 32 + lane] += qs[b >> 1];
    }
    __syncwarp();
    unsigned long long Q = 0;
    if (lane < k) {
        const unsigned long long* h = hist + lane * 32;
        for (int l = 0; l < 32; ++l) Q += h[(l + lane) & 31];
    }
    __syncwarp();
    const double eta = lane < k ? R.etab[(size_t)i * k + lane] : 0.0;
    finish_row(R, i, Q, eta, lane);
}

template <int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) persistent_batch_kernel(const __grid_constant__ PersistArgs P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int item_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* my_smem = smem_raw + (size_t)warp * P.smem_per_ant;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    for (int t = 0; t < P.iterations; ++t) {
        const int iteration = *reinterpret_cast<volatile int*>(P.iteration);
        // 1. construction: each warp pulls `pull` ant slots at a time
        if (leader) P.queue[2] = 0u;  // the rebuild counter of the previous iteration is free again
        for (;;) {
            int base = 0;
            if (lane == 0) base = (int)atomicAdd(&P.queue[0], (unsigned)P.pull);
            base = __shfl_sync(FULL, base, 0);
            if (base >= P.slots) break;
            const int end = min(base + P.pull, P.slots);
            for (int j = base; j < end; ++j) {
                const int2 sa = P.slot[j];
                construct_ant<true, STAGE_K>(P.largs[sa.x], sa.y, iteration, my_smem, lane);
            }
        }
        if (!grid_barrier(P)) return;
        // 2. Algorithm 1's replacement, one slot per pull
        if (leader) P.queue[0] = 0u;
        for (;;) {
            int j = 0;
            if (lane == 0) j = (int)atomicAdd(&P.queue[1], 1u);
            j = __shfl_sync(FULL, j, 0);
            if (j >= P.slots) break;
            const int2 sa = P.slot[j];
            commit_ant(P.cargs[sa.x], sa.y, lane);
        }
        if (!grid_barrier(P)) return;
        // 3. C_gbest and the deposit weights, one warp per colony
        if (leader) P.queue[1] = 0u;
        for (int i = blockIdx.x * WARPS + warp; i < P.count; i += gridDim.x * WARPS) gbest_warp(P.gargs[i], lane);
        if (!grid_barrier(P)) return;
        // 4. pheromone rebuild: whole blocks pull chunks of one colony's cities
        unsigned long long* qs = reinterpret_cast<unsigned long long*>(smem_raw);
        unsigned long long* hist = qs + P.m_cap + (size_t)warp * P.k * 32;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) item_s = (int)atomicAdd(&P.queue[2], 1u);
            __syncthreads();
            const int item = item_s;
            if (item >= P.ritems) break;
            const int4 bm = P.rmap[item];
            const RebuildArgs& R = P.rargs[bm.x];
            for (int a = threadIdx.x; a < R.m; a += blockDim.x) qs[a] = R.q[a];
            __syncthreads();
            for (int i = bm.y + warp; i < bm.z; i += WARPS) rebuild_city(R, i, qs, hist, lane);
        }
        if (leader) *P.iteration = iteration + 1;
        if (!grid_barrier(P)) return;
    }
}

// Persistent schedules: (warps per block, minimum resident blocks per SM, slots per pull).
extern const int kPersistConfigs[ACO_PERSIST_CONFIGS][3] = {{1, 32, 1}, {2, 16, 1}, {4, 8, 1}, {4, 4, 1}};

size_t persistent_smem_bytes(int smem_per_ant, int warps, int m_cap, int k) {
    const size_t c = (size_t)smem_per_ant * warps;
    const size_t r = sizeof(unsigned long long) * ((size_t)m_cap + (size_t)warps * k * 32);
    return c > r ? c : r;
}

// One cooperative launch of P.iterations iterations with persistent schedule `config`: as many
// blocks as fit on the device at once.
cudaError_t launch_persistent_batch(PersistArgs P, int config, int num_sms, cudaStream_t s, int* grid_out) {
    const int warps = kPersistConfigs[config][0];
    P.pull = kPersistConfigs[config][2];
    const size_t smem = persistent_smem_bytes(P.smem_per_ant, warps, P.m_cap, P.k);
    void (*kern)(PersistArgs) = nullptr;
    switch (config) {
        case 0: kern = persistent_batch_kernel<1, 32>; break;
        case 1: kern = persistent_batch_kernel<2, 16>; break;
        case 2: kern = persistent_batch_kernel<4, 8>; break;
        case 3: kern = persistent_batch_kernel<4, 4>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * num_sms;
    if (grid_out) *grid_out = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P);
}

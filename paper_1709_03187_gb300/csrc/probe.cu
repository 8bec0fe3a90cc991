// probe.cu -- STREAM-style bandwidth probe: the denominator of the construction kernel's roofline.
//
// The construction kernel's working set (candidate rows, pheromone weights, the per-ant lists) is
// a few tens of MB, far inside the L2 cache, so its memory roofline is the L2 bandwidth, which the
// chip's data sheet does not give.  This probe measures it on the caller's buffer: every launch
// streams the buffer through 16-byte loads that bypass L1 (ld.global.cg), so a buffer well inside
// L2 is served by L2 after the first pass.  A copy mode (first half to second half, 16-byte
// loads and stores cached in L2 only) measures read + write traffic.  Nothing here changes a
// clock or any other setting of the device.
#include "common.cuh"

__device__ __forceinline__ int4 ld_cg(const int4* p) {
    int4 v;
    asm volatile("ld.global.cg.v4.s32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_cg(int4* p, int4 v) {
    asm volatile("st.global.cg.v4.s32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// Every thread XORs four independent 16-byte loads per round into its own accumulator; the
// accumulator is stored only if it equals a value no buffer of zeros produces, so the loads
// cannot be dropped and nothing is written.
__global__ void __launch_bounds__(512) probe_read_kernel(const int4* __restrict__ buf, long long n16, int passes,
                                                         int4* __restrict__ sink) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    int4 acc = make_int4(0, 0, 0, 0);
    for (int pass = 0; pass < passes; ++pass) {
        long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const int4 a = ld_cg(buf + i), b = ld_cg(buf + i + stride), c = ld_cg(buf + i + 2 * stride),
                       d = ld_cg(buf + i + 3 * stride);
            acc.x ^= a.x ^ b.x ^ c.x ^ d.x;
            acc.y ^= a.y ^ b.y ^ c.y ^ d.y;
            acc.z ^= a.z ^ b.z ^ c.z ^ d.z;
            acc.w ^= a.w ^ b.w ^ c.w ^ d.w;
        }
        for (; i < n16; i += stride) {
            const int4 a = ld_cg(buf + i);
            acc.x ^= a.x; acc.y ^= a.y; acc.z ^= a.z; acc.w ^= a.w;
        }
    }
    if (acc.x == 0x5EED1234 && acc.y == 0x0BADF00D && acc.z == 0x12345678 && acc.w == 0x7FFFFFFE) *sink = acc;
}

__global__ void __launch_bounds__(512) probe_copy_kernel(const int4* __restrict__ src, int4* __restrict__ dst,
                                                         long long n16, int passes) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int pass = 0; pass < passes; ++pass) {
        long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + stride < n16; i += 2 * stride) {
            const int4 a = ld_cg(src + i), b = ld_cg(src + i + stride);
            st_cg(dst + i, a);
            st_cg(dst + i + stride, b);
        }
        for (; i < n16; i += stride) st_cg(dst + i, ld_cg(src + i));
    }
}

extern "C" aco_status aco_probe_bandwidth(void* buf_dev, int64_t bytes, int32_t mode, int32_t reps, void* stream,
                                          float* ms_out) {
    ACO_RANGE("aco_probe_bandwidth");
    if (!buf_dev || !ms_out || reps < 1 || (mode != 0 && mode != 1)) return ACO_ERR_INVALID_ARG;
    if (bytes < 4096 || (bytes & 31) || (reinterpret_cast<uintptr_t>(buf_dev) & 15)) return ACO_ERR_INVALID_ARG;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return ACO_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int4* buf = static_cast<int4*>(buf_dev);
    // the read mode keeps 16 bytes at the start as its (never written) sink
    const long long n16 = bytes / 16;
    const int blocks = sms * 4;  // 4 blocks of 512 threads per SM: 64 warps, the SM's full occupancy
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return ACO_ERR_CUDA;
    }
    // every launch makes `passes` passes over the buffer, so that launch overheads do not count
    auto launch = [&](int passes) {
        if (mode == 0) probe_read_kernel<<<blocks, 512, 0, s>>>(buf + 1, n16 - 1, passes, buf);
        else probe_copy_kernel<<<blocks, 512, 0, s>>>(buf, buf + n16 / 2, n16 / 2, passes);
    };
    launch(1);  // brings the buffer into L2 (when it fits)
    cudaEventRecord(e0, s);
    launch(reps);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return ACO_ERR_CUDA;
    *ms_out = ms;
    return ACO_OK;
}

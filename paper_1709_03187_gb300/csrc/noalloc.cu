// noalloc.cu -- candidate lists for callers that cannot allocate device memory.
//
// aco_build_candidates_noalloc runs the same grid-bucketed exact k-nearest-neighbour build as
// aco_build_candidates, but its working memory (the city grid and its counting sort) is a fixed
// file-scope __device__ array instead of buffers from cudaMalloc.  Some callers cannot call
// cudaMalloc at the point where they need candidate lists: a host process whose device memory is
// owned by another allocator or memory pool, or code that must not allocate once it has started
// (for latency or certification reasons).  They pass their own input and output buffers and get
// the lists without any allocation by this library.
//
// Limits and sharing: at most ACO_NOALLOC_MAX_N cities.  Every GPU that loads the library holds
// the array (1,966,080 bytes, 1.875 MiB) until the process exits.  All calls on a device share it
// and it keeps the contents of the last call; each call clears what must start at zero.  Calls
// whose work overlaps on the GPU (different streams, or different host threads) race on the
// array and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

#define ACO_NOALLOC_MAX_N 65536
#define ACO_NOALLOC_MAX_DEVICES 64

size_t knn_scratch_bytes(int max_n);
cudaError_t launch_knn_on_scratch(const double* xy, int n, int k, int32_t* cand, unsigned char* scratch,
                                  int num_sms, cudaStream_t s);

// knn_scratch_bytes(ACO_NOALLOC_MAX_N) = 1,835,232 bytes, rounded up; checked on every call.
#define ACO_NOALLOC_SCRATCH_BYTES (1920u * 1024u)

static __device__ __align__(256) unsigned char g_noalloc_scratch[ACO_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array per device, looked up with that device current.  In host
// code the array's name is only a host-side stand-in, never a device address.  The address
// belongs to the context the module was loaded into: if the caller resets the device (or the
// primary context is destroyed and created again), the module is loaded again and the array may
// move, so the cache is keyed by the context's unique id and the lookup repeats when it changes.
typedef int (*CtxGetCurrentFn)(void**);                       // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void*, unsigned long long*);        // cuCtxGetId
static CtxGetCurrentFn g_ctx_current;
static CtxGetIdFn g_ctx_id;
static bool g_driver_looked_up;
static void* g_scratch_ptr[ACO_NOALLOC_MAX_DEVICES];
static unsigned long long g_scratch_ctx[ACO_NOALLOC_MAX_DEVICES];
static int g_num_sms[ACO_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mutex;

// Unique id of the current context (0 if none is current or the driver entry points are missing).
static unsigned long long current_context_id() {
    if (!g_driver_looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            f1 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            f2 = nullptr;
        cudaGetLastError();
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
        g_driver_looked_up = true;
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

static aco_status scratch_for_current_device(void** ptr, int* num_sms, int* device) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ACO_NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return ACO_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    const unsigned long long ctx = current_context_id();
    // without a context id (no driver entry point) the address is looked up on every call
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            g_scratch_ptr[dev] = nullptr;
            return ACO_ERR_CUDA;
        }
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms[dev] = sms > 0 ? sms : 1;
        g_scratch_ptr[dev] = p;
        // the symbol lookup makes the primary context current if none was
        g_scratch_ctx[dev] = ctx ? ctx : current_context_id();
    }
    *ptr = g_scratch_ptr[dev];
    *num_sms = g_num_sms[dev];
    *device = dev;
    return ACO_OK;
}

extern "C" aco_status aco_build_candidates_noalloc(const double* xy_dev, int32_t n, int32_t k, int32_t* cand_out_dev,
                                                   void* stream) {
    ACO_RANGE("aco_build_candidates_noalloc");
    if (!xy_dev || !cand_out_dev) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(xy_dev, 8) || aco_misaligned(cand_out_dev, 4)) return ACO_ERR_INVALID_ARG;
    if (n < 2 || n > ACO_NOALLOC_MAX_N) return ACO_ERR_INVALID_ARG;  // beyond the fixed scratch
    if (k < 1 || k > ACO_MAX_K || k > n - 1) return ACO_ERR_INVALID_ARG;
    if (knn_scratch_bytes(n) > ACO_NOALLOC_SCRATCH_BYTES) return ACO_ERR_INVALID_ARG;
    // the call reads its error flag back and synchronises: it cannot be part of a captured graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return ACO_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return ACO_ERR_INVALID_ARG;
    void* scratch = nullptr;
    int sms = 1, dev = 0;
    aco_status st = scratch_for_current_device(&scratch, &sms, &dev);
    if (st != ACO_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_knn_on_scratch(xy_dev, n, k, cand_out_dev, static_cast<unsigned char*>(scratch), sms, s);
    if (e != cudaSuccess) return ACO_ERR_CUDA;
    // the device error flags sit right after the grid descriptor in the scratch
    int flag = 0;
    const size_t flag_off = (sizeof(GridDesc) + 15) & ~(size_t)15;
    e = cudaMemcpyAsync(&flag, static_cast<unsigned char*>(scratch) + flag_off, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ACO_ERR_CUDA;
    }
    if (flag & (DEVERR_DUPLICATE | DEVERR_NONFINITE)) return ACO_ERR_INVALID_ARG;
    return flag ? ACO_ERR_CUDA : ACO_OK;
}

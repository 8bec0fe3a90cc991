// localsearch.cu -- windowed 2-opt on constructed tours (Section 3.2 local search; Section 5
// restricts it to edges within W tour positions of each other).
//
// After the construction kernel, each ant (index order, at most ACO_LS_MAX_ANTS per iteration)
// whose Philox draw (0, ant, iteration, 5) gives u < p applies 2-opt to its new tour:
//   ls_select_kernel       the selected ants, in index order;
//   ls_materialize_kernel  each selected ant's whole new tour in l_best layout (the preserved
//                          positions from l_best, the rebuilt ones from the segment);
//   ls_pass_kernel         one pass: positions split into blocks at 0, off, off + 2W, ..., n
//                          (off = 0 on even passes, W on odd ones), one warp per block and ant;
//                          every position i (ascending) scans j = i + 2 .. min(i + W, end - 2)
//                          (ascending, 32 at a time), takes the first move with FP64 gain
//                          (d(a,b) + d(c,d)) - (d(a,c) + d(b,d)) > 0, reverses T[i+1..j] and
//                          carries on with the next j.  Gains are screened in FP32 on coordinates
//                          relative to the block's first city; a gain within the screen's error
//                          bound of zero is decided in FP64.  A pass is skipped once the two
//                          passes before it made no move (at most ACO_LS_MAX_PASSES);
//   ls_finalize_kernel     the exact fixed-point length, and the tour handed to the commit as a
//                          whole tour (committed if strictly shorter than l_best).
#include <float.h>
#include <math.h>

#include "common.cuh"

#define FULL 0xffffffffu

struct LsArgs {
    int n, m, W, iteration;
    double p;
    unsigned long long seed;
    const double* __restrict__ xy;
    const int* __restrict__ lbest;
    int* __restrict__ seg;
    AntIter* __restrict__ antit;
    int* __restrict__ buf;   // ACO_LS_MAX_ANTS * n working tours
    int* __restrict__ sel;   // ACO_LS_MAX_ANTS selected ants, then the count
    int* __restrict__ imp;   // ACO_LS_MAX_ANTS * ACO_LS_MAX_PASSES: a move in that pass
    unsigned long long* __restrict__ moves;
    int* __restrict__ errflag;
};

// The first ACO_LS_MAX_ANTS ants (index order) whose local-search draw is below p.
__global__ void ls_select_kernel(const __grid_constant__ LsArgs L) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) base = 0;
    for (int e = tid; e < ACO_LS_MAX_ANTS * ACO_LS_MAX_PASSES; e += blockDim.x) L.imp[e] = 0;
    __syncthreads();
    for (int a0 = 0; a0 < L.m; a0 += blockDim.x) {
        const int a = a0 + tid;
        bool s = false;
        if (a < L.m) {
            const Draw4 d = aco_draw(L.seed, 0, (uint32_t)a, (uint32_t)L.iteration, PURPOSE_LS);
            s = unit53(d.x0, d.x1) < L.p;
        }
        const unsigned b = __ballot_sync(FULL, s);
        if (lane == 0) wsum[w] = __popc(b);
        __syncthreads();
        int before = base;
        for (int v = 0; v < w; ++v) before += wsum[v];
        const int pos = before + __popc(b & ((1u << lane) - 1u));
        if (s && pos < ACO_LS_MAX_ANTS) L.sel[pos] = a;
        __syncthreads();
        if (tid == 0)
            for (int v = 0; v < nw; ++v) base += wsum[v];
        __syncthreads();
    }
    if (tid == 0) L.sel[ACO_LS_MAX_ANTS] = base < ACO_LS_MAX_ANTS ? base : ACO_LS_MAX_ANTS;
}

__global__ void ls_materialize_kernel(const __grid_constant__ LsArgs L) {
    const int slot = blockIdx.y;
    if (slot >= L.sel[ACO_LS_MAX_ANTS]) return;
    const int a = L.sel[slot], n = L.n;
    const AntIter it = L.antit[a];
    const int* S = L.seg + (size_t)a * n;
    const int* Lb = L.lbest + (size_t)a * n;
    int* T = L.buf + (size_t)slot * n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        if (it.s < 0) {
            T[p] = S[p];
        } else {
            int q = p - (it.s + it.P);
            q = ((q % n) + n) % n;
            T[p] = q < it.M ? S[q] : Lb[p];
        }
    }
}

__device__ __forceinline__ float len32(float2 p, float2 q) {
    const float dx = __fsub_rn(p.x, q.x), dy = __fsub_rn(p.y, q.y);
    return __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
}

__device__ __forceinline__ double len64(const double* __restrict__ xy, int i, int j) {
    return __dsqrt_rn(dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1]));
}

// One pass over one block of one ant's tour (one warp).  Dynamic shared memory: the block's
// city ids (2W + 2) and FP32 coordinates relative to its first city (2W + 2).
__global__ void __launch_bounds__(32) ls_pass_kernel(const __grid_constant__ LsArgs L, int pass) {
    extern __shared__ __align__(16) unsigned char ls_smem[];
    const int slot = blockIdx.y, lane = threadIdx.x;
    if (slot >= L.sel[ACO_LS_MAX_ANTS]) return;
    const int* imp = L.imp + slot * ACO_LS_MAX_PASSES;
    if (pass >= 2 && !imp[pass - 1] && !imp[pass - 2]) return;  // converged
    const int n = L.n, W = L.W, b = blockIdx.x;
    const int off = (pass & 1) ? W : 0;
    long long b0, b1;
    if (off == 0) {
        b0 = 2LL * W * b;
        b1 = b0 + 2LL * W;
    } else {
        b0 = b == 0 ? 0 : W + 2LL * W * (b - 1);
        b1 = b == 0 ? W : b0 + 2LL * W;
    }
    if (b0 >= n) return;
    if (b1 > n) b1 = n;
    const int len = (int)(b1 - b0);
    if (len < 4) return;
    float2* rel = reinterpret_cast<float2*>(ls_smem);
    int* ids = reinterpret_cast<int*>(ls_smem + sizeof(float2) * (size_t)(2 * W + 2));
    int* T = L.buf + (size_t)slot * n + b0;
    const double xr = L.xy[2 * T[0]], yr = L.xy[2 * T[0] + 1];
    float S = 0.f;
    for (int p = lane; p < len; p += 32) {
        const int c = T[p];
        ids[p] = c;
        const float2 r = make_float2(__double2float_rn(__dsub_rn(L.xy[2 * c], xr)),
                                     __double2float_rn(__dsub_rn(L.xy[2 * c + 1], yr)));
        rel[p] = r;
        S = fmaxf(S, fmaxf(fabsf(r.x), fabsf(r.y)));
    }
    for (int o = 16; o; o >>= 1) S = fmaxf(S, __shfl_xor_sync(FULL, S, o));
    __syncwarp();
    int moved = 0;
    for (int i = 0; i + 3 < len; ++i) {
        const int jmax = min(i + W, len - 2);
        int j0 = i + 2;
        while (j0 <= jmax) {
            const int j = j0 + lane;
            const bool valid = j <= jmax;
            const float2 pa = rel[i], pb = rel[i + 1];
            const float dab = len32(pa, pb);
            int state = 0;  // 1 = improving, -1 = not, 2 = undecided
            if (valid) {
                const float2 pc = rel[j], pd = rel[j + 1];
                const float dcd = len32(pc, pd), dac = len32(pa, pc), dbd = len32(pb, pd);
                const float g = __fsub_rn(__fadd_rn(dab, dcd), __fadd_rn(dac, dbd));
                // FP32 error bound: coordinates rounded relative to the block (<= 2^-24 S each),
                // four lengths and three sums (<= 2^-24 (12 S + 6 D)); 2^-20 (S + D) covers both
                const float D = __fadd_rn(__fadd_rn(dab, dcd), __fadd_rn(dac, dbd));
                const float B = __fmul_rn(0x1.0p-20f, __fadd_rn(S, D));
                state = g > B ? 1 : (g < -B ? -1 : 2);
            }
            const unsigned im = __ballot_sync(FULL, state == 1);
            unsigned un = __ballot_sync(FULL, state == 2);
            const int first_im = im ? __ffs(im) - 1 : 32;
            un &= first_im < 32 ? ((1u << first_im) - 1u) : FULL;  // only undecided lanes before it
            unsigned ex = 0;
            if (un) {
                bool e = false;
                if ((un >> lane) & 1u) {
                    const int a = ids[i], bb = ids[i + 1], c = ids[j], d = ids[j + 1];
                    const double g64 = __dsub_rn(__dadd_rn(len64(L.xy, a, bb), len64(L.xy, c, d)),
                                                 __dadd_rn(len64(L.xy, a, c), len64(L.xy, bb, d)));
                    e = g64 > 0.0;
                }
                ex = __ballot_sync(FULL, e);
            }
            const unsigned take = im | ex;
            if (!take) {
                j0 += 32;
                continue;
            }
            const int js = j0 + __ffs(take) - 1;
            // reverse positions i+1 .. js
            const int cnt = (js - i) >> 1;
            for (int q = lane; q < cnt; q += 32) {
                const int l = i + 1 + q, r = js - q;
                const int ti = ids[l];
                ids[l] = ids[r];
                ids[r] = ti;
                const float2 tr = rel[l];
                rel[l] = rel[r];
                rel[r] = tr;
            }
            __syncwarp();
            ++moved;
            j0 = js + 1;
        }
    }
    if (moved) {
        for (int p = lane; p < len; p += 32) T[p] = ids[p];
        if (lane == 0) {
            atomicOr(&L.imp[slot * ACO_LS_MAX_PASSES + pass], 1);
            atomicAdd(L.moves, (unsigned long long)moved);
        }
    }
}

// Exact length of each improved tour; the tour becomes the ant's whole new tour.
__global__ void ls_finalize_kernel(const __grid_constant__ LsArgs L) {
    __shared__ unsigned long long part[64];
    const int slot = blockIdx.x;
    if (slot >= L.sel[ACO_LS_MAX_ANTS]) return;
    const int a = L.sel[slot], n = L.n, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int* T = L.buf + (size_t)slot * n;
    int* S = L.seg + (size_t)a * n;
    u128 acc = 0;
    for (int p = tid; p < n; p += blockDim.x) {
        const int c = T[p], d = T[p + 1 == n ? 0 : p + 1];
        acc += len_to_fix(__dsqrt_rn(dist2(L.xy[2 * c], L.xy[2 * c + 1], L.xy[2 * d], L.xy[2 * d + 1])));
        S[p] = c;
    }
    acc = warp_sum_u128(acc);
    if (lane == 0) {
        part[2 * w] = (unsigned long long)acc;
        part[2 * w + 1] = (unsigned long long)(acc >> 64);
    }
    __syncthreads();
    if (tid == 0) {
        u128 total = 0;
        for (int v = 0; v < (int)(blockDim.x >> 5); ++v) total += ((u128)part[2 * v + 1] << 64) | part[2 * v];
        AntIter it;
        it.s = -1;
        it.P = 0;
        it.M = n - 1;
        it.start = T[0];
        it.newlen = fix_to_len(total);
        it.fix_lo = (unsigned long long)total;
        it.fix_hi = (unsigned long long)(total >> 64);
        L.antit[a] = it;
    }
}

static size_t ls_smem_bytes(int W) { return (sizeof(float2) + sizeof(int)) * (size_t)(2 * W + 2); }

aco_status launch_local_search(aco_instance* inst, int32_t iteration) {
    const aco_params& p = inst->p;
    LsArgs L;
    L.n = p.n; L.m = p.m; L.W = inst->ls_window; L.iteration = iteration; L.p = inst->ls_p; L.seed = p.seed;
    L.xy = inst->xy; L.lbest = inst->lbest; L.seg = inst->seg; L.antit = inst->antit; L.buf = inst->ls_buf;
    L.sel = inst->ls_sel; L.imp = inst->ls_imp; L.moves = inst->counters + CNT_LS_MOVES; L.errflag = inst->errflag;
    cudaStream_t s = inst->stream;
    ls_select_kernel<<<1, 1024, 0, s>>>(L);
    ls_materialize_kernel<<<dim3(ceil_div(p.n, 1024), ACO_LS_MAX_ANTS), 1024, 0, s>>>(L);
    const size_t smem = ls_smem_bytes(inst->ls_window);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(ls_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int nblk = ceil_div(p.n, 2 * inst->ls_window) + 1;
    for (int pass = 0; pass < ACO_LS_MAX_PASSES; ++pass)
        ls_pass_kernel<<<dim3(nblk, ACO_LS_MAX_ANTS), 32, smem, s>>>(L, pass);
    ls_finalize_kernel<<<ACO_LS_MAX_ANTS, 256, 0, s>>>(L);
    return check_launch(inst, "local search kernels");
}

extern "C" aco_status aco_set_local_search(aco_instance* inst, double p, int32_t window) {
    ACO_RANGE("aco_set_local_search");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "set_local_search: LBEST mode only");
    if (inst->constructed) return set_err(inst, ACO_ERR_STATE, "set_local_search: tours constructed, update pending");
    if (!(p >= 0.0 && p <= 1.0)) return set_err(inst, ACO_ERR_INVALID_ARG, "set_local_search: p in [0, 1]");
    if (window < 2 || window > 4096) return set_err(inst, ACO_ERR_INVALID_ARG, "set_local_search: window in [2, 4096]");
    if (p > 0.0 && inst->async_share)
        return set_err(inst, ACO_ERR_STATE, "set_local_search: asynchronous sharing is on (the two exclude each other)");
    if (p > 0.0 && (inst->ant0 != 0 || inst->ant1 != inst->p.m))
        return set_err(inst, ACO_ERR_STATE, "set_local_search: the colony is split over ranks");
    if (p > 0.0 && !inst->ls_buf) {
        bool ok = cudaMalloc(&inst->ls_buf, sizeof(int) * (size_t)ACO_LS_MAX_ANTS * inst->p.n) == cudaSuccess;
        ok = ok && cudaMalloc(&inst->ls_sel, sizeof(int) * (ACO_LS_MAX_ANTS + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(&inst->ls_imp, sizeof(int) * ACO_LS_MAX_ANTS * ACO_LS_MAX_PASSES) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return set_err(inst, ACO_ERR_OOM, "set_local_search: scratch allocation failed");
        }
    }
    inst->ls_p = p;
    inst->ls_window = window;
    return ACO_OK;
}

// mlp.cu -- learned edge proposal: a 3-layer MLP that scores candidate edges in place of
// eta^beta, with its training on the GPU.
//
// Network (per candidate edge, row-major rows of 16 BF16 inputs):
//   h1 = relu(W1 x)      W1: 64 x 16   (input 5 is the constant 1: column 5 of W1 is the bias)
//   h1[63] = 1           (constant unit: column 63 of W2 is the layer-2 bias)
//   h2 = relu(W2 h1)     W2: 64 x 64
//   h2[63] = 1           (constant unit: w3[63] is the output bias)
//   z  = w3 . h2         score = exp(z)
// BF16 weights and activations, FP32 accumulation on the fifth-generation tensor cores (tcgen05
// MMAs with accumulators in tensor memory, umma.cuh), the hidden activations rounded to BF16
// between layers.
//
// Training objective: for every city, the softmax of z over its k candidate edges against the
// best tour's edges among them (cross-entropy; each of the city's best-tour neighbours that is a
// candidate carries equal target mass).  Gradients:
//   dz = softmax(z) - y;  dh2 = dz w3 * [h2 > 0];  dh1 = dh2 W2 * [h1 > 0]  (constant units 0)
//   dW2 = dh2^T h1;  dW1 = dh1^T x;  dw3 = dz^T h2
// The weight gradients are split over blocks of MLP_RPB rows with per-block partial sums and a
// fixed-order reduction, so a training step is deterministic.  Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "common.cuh"
#include "umma.cuh"

#define FULL 0xffffffffu
#define MLP_IN 16
#define MLP_H 64
#define MLP_NW (MLP_H * MLP_IN + MLP_H * MLP_H + MLP_H)  // W1 | W2 | w3
#define MLP_RPB 256  // rows per block of the weight gradients (summed in FP32, then the blocks in order)

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct MlpWeights {  // BF16 copies used by the kernels
    const bf16* W1;  // [64][16]
    const bf16* W2;  // [64][64]
    const bf16* w3;  // [64]
};

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// ---------------------------------------------------------------- forward on the tensor cores
// One CTA of 128 threads works through 128-row tiles; thread t owns row t of the tile.  Layer 1 is
// one tcgen05 MMA (M 128, N 64, K 16) of the feature rows by W1; layer 2 four MMAs (K = 64 in steps
// of 16) of the BF16 h1 tile by W2.  The FP32 accumulators live in tensor memory (columns 0..63
// layer 1, 64..127 layer 2) and come back to registers one row per thread for the epilogues: ReLU,
// the constant unit, BF16 rounding and z = w3 . h2 summed in FP32 in unit order.
#define TC_COLS 128u               // tensor-memory columns per CTA
#define TC_SMEM (64 * 1024)        // dynamic shared memory per CTA; also keeps 3 CTAs at most on an SM
#define TC_MAX_CTAS_PER_SM 4       // 512 tensor-memory columns / TC_COLS: more would wait in tcgen05.alloc
#define TC_WAIT_NS 2000000000ull   // a wait for an MMA gives up after 2 s
// shared-memory map (byte offsets; the base is 1024-byte aligned)
#define TC_A1 0          // feature tile, 128 x 16 BF16
#define TC_A2 4096       // h1 tile, 128 x 64 BF16
#define TC_W1 20480      // W1, 64 x 16
#define TC_W2 22528      // W2, 64 x 64
#define TC_W3 30720      // w3 as FP32
#define TC_BAR 30976     // mbarrier of the MMA completions
#define TC_SLOT 30984    // tensor-memory base address written by tcgen05.alloc

// Byte offset of 16-byte chunk `kg` of row `row` in a K-major tile of `kgroups` chunks per row.
__device__ __forceinline__ uint32_t kmajor_off(int row, int kg, int kgroups) {
    return (uint32_t)((row >> 3) * (128 * kgroups) + kg * 128 + (row & 7) * 16);
}

// z and/or score = exp(beta z) (beta z clamped to [-60, 60]), optionally h1 and h2 (BF16), for R
// rows.  A wait that gives up sets *status and writes NaN to the z and score rows this CTA has
// not finished.
__global__ void __launch_bounds__(128, 1)
    mlp_forward_tc_kernel(MlpWeights w, const bf16* __restrict__ X, long long R, float* __restrict__ z,
                          float* __restrict__ score, float beta, bf16* __restrict__ h1out, bf16* __restrict__ h2out,
                          int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tc_smem + TC_BAR);
    uint32_t* slot = reinterpret_cast<uint32_t*>(tc_smem + TC_SLOT);
    float* w3s = reinterpret_cast<float*>(tc_smem + TC_W3);
    // weights into the K-major operand layout (16-byte chunks of rows)
    for (int c = tid; c < MLP_H * 2; c += 128)
        *reinterpret_cast<uint4*>(tc_smem + TC_W1 + kmajor_off(c >> 1, c & 1, 2)) =
            *reinterpret_cast<const uint4*>(w.W1 + (size_t)(c >> 1) * MLP_IN + 8 * (c & 1));
    for (int c = tid; c < MLP_H * 8; c += 128)
        *reinterpret_cast<uint4*>(tc_smem + TC_W2 + kmajor_off(c >> 3, c & 7, 8)) =
            *reinterpret_cast<const uint4*>(w.W2 + (size_t)(c >> 3) * MLP_H + 8 * (c & 7));
    if (tid < MLP_H) w3s[tid] = __bfloat162float(w.w3[tid]);
    if (tid == 0) umma::mbar_init(bar, 1);
    if (warp == 0) umma::tmem_alloc(slot, TC_COLS);
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;  // this warp's quarter of the lanes
    constexpr uint32_t idesc = umma::IdescBf16<128, MLP_H>::value;
    const uint32_t a1 = umma::smem_addr(tc_smem + TC_A1), a2 = umma::smem_addr(tc_smem + TC_A2);
    const uint32_t b1 = umma::smem_addr(tc_smem + TC_W1), b2 = umma::smem_addr(tc_smem + TC_W2);
    uint32_t phase = 0;
    bool failed = false;
    const long long tiles = (R + 127) / 128;
    long long tile = blockIdx.x;
    for (; tile < tiles; tile += gridDim.x) {
        const long long row = tile * 128 + tid;
        uint32_t xv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) xv[i] = row < R ? ld32(X + (size_t)row * MLP_IN + 2 * i) : 0u;
        *reinterpret_cast<uint4*>(tc_smem + TC_A1 + kmajor_off(tid, 0, 2)) = make_uint4(xv[0], xv[1], xv[2], xv[3]);
        *reinterpret_cast<uint4*>(tc_smem + TC_A1 + kmajor_off(tid, 1, 2)) = make_uint4(xv[4], xv[5], xv[6], xv[7]);
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            umma::mma_bf16(tmem, umma::smem_desc(a1, 128, 256), umma::smem_desc(b1, 128, 256), idesc, 0u);
            umma::commit(bar);
        }
        bool ok = umma::mbar_wait(bar, phase, TC_WAIT_NS);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        umma::fence_after_sync();
        // layer-1 epilogue: h1 = bf16(relu(.)), unit 63 = 1, into the h1 tile (and out)
        uint32_t hp[32];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float acc[32];
            umma::tmem_ld32(tmem + lanes + 32u * half, acc);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = 32 * half + 2 * i;
                const float v0 = fmaxf(acc[2 * i], 0.f);
                const float v1 = c + 1 == MLP_H - 1 ? 1.f : fmaxf(acc[2 * i + 1], 0.f);
                hp[16 * half + i] = pack_bf16(v0, v1);
            }
        }
#pragma unroll
        for (int kg = 0; kg < 8; ++kg) {
            const uint4 v = make_uint4(hp[4 * kg], hp[4 * kg + 1], hp[4 * kg + 2], hp[4 * kg + 3]);
            *reinterpret_cast<uint4*>(tc_smem + TC_A2 + kmajor_off(tid, kg, 8)) = v;
            if (h1out && row < R) *reinterpret_cast<uint4*>(h1out + (size_t)row * MLP_H + 8 * kg) = v;
        }
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
#pragma unroll
            for (int s = 0; s < 4; ++s)
                umma::mma_bf16(tmem + MLP_H, umma::smem_desc(a2 + 256u * s, 128, 1024),
                               umma::smem_desc(b2 + 256u * s, 128, 1024), idesc, s > 0 ? 1u : 0u);
            umma::commit(bar);
        }
        ok = umma::mbar_wait(bar, phase, TC_WAIT_NS);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        umma::fence_after_sync();
        // layer-2 epilogue and layer 3
        float zr = 0.f;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float acc[32];
            umma::tmem_ld32(tmem + lanes + MLP_H + 32u * half, acc);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int c = 32 * half + i;
                acc[i] = c == MLP_H - 1 ? 1.f : bf16_round(fmaxf(acc[i], 0.f));
                zr = __fmaf_rn(acc[i], w3s[c], zr);
            }
            if (h2out && row < R) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4*>(h2out + (size_t)row * MLP_H + 32 * half + 8 * q) =
                        make_uint4(pack_bf16(acc[8 * q], acc[8 * q + 1]), pack_bf16(acc[8 * q + 2], acc[8 * q + 3]),
                                   pack_bf16(acc[8 * q + 4], acc[8 * q + 5]), pack_bf16(acc[8 * q + 6], acc[8 * q + 7]));
            }
        }
        if (row < R) {
            if (z) z[row] = zr;
            if (score) score[row] = __expf(fminf(fmaxf(beta * zr, -60.f), 60.f));
        }
    }
    if (failed) {
        if (tid == 0) atomicExch(status, 1);
        for (; tile < tiles; tile += gridDim.x) {
            const long long row = tile * 128 + tid;
            if (row < R) {
                if (z) z[row] = __int_as_float(0x7fc00000);
                if (score) score[row] = __int_as_float(0x7fc00000);
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, TC_COLS);
    }
}

// ---------------------------------------------------------------- backward on the tensor cores
// One CTA per block of MLP_RPB = 256 rows: two 128-row sub-tiles, thread t owning row t of each.
// Per sub-tile: dh2 = dz w3 [h2 > 0] in registers; dh1 = dh2 W2 [h1 > 0] by four tcgen05 MMAs
// (M 128, N 64, K 16; B = W2 transposed, K-major); then a chain of eight MMAs over the sub-tile's
// rows accumulates
//     D[128 x 144] += [dh2 | dh1]^T [h1 | x | h2]
// with both operands MN-major (the rows are the contraction index): D[u][0..63] = dW2 row u,
// D[64 + u][64..79] = dW1 row u, and because unit 63 of dh2 is always zero (the constant unit) that
// row of the A operand carries dz instead, so that D[63][80..143] = dw3.  The block's gradient goes
// out as one partial vector in the layout W1 | W2 | w3, reduced over the blocks in order by
// mlp_reduce_kernel.
#define TCB_COLS 256u               // tensor-memory columns per CTA: dh1 (64) and D (144)
#define TCB_SMEM (96 * 1024)        // dynamic shared memory per CTA; also keeps 2 CTAs at most on an SM
#define TCB_MAX_CTAS_PER_SM 2       // 512 tensor-memory columns / TCB_COLS
#define TCB_N 144                   // columns of D: h1 | x | h2
#define TCB_W2T 0                   // W2 transposed, 64 x 64 K-major (8 KB)
#define TCB_AH 8192                 // dh2 tile, 128 x 64 K-major (16 KB)
#define TCB_AW 24576                // [dh2 | dh1], 16 unit groups x 16 row groups, MN-major (32 KB)
#define TCB_BW 57344                // [h1 | x | h2], 18 column groups x 16 row groups, MN-major (36 KB)
#define TCB_W3 94208                // w3 as FP32
#define TCB_BAR 94464
#define TCB_SLOT 94472

// Byte offset of the 16-byte chunk of M/N group g (8 values) in row r (along K) of an MN-major
// tile of 128 rows: 16 K groups of 128 bytes per M/N group.
__device__ __forceinline__ uint32_t mnmajor_off(int r, int g) {
    return (uint32_t)(g * 2048 + (r >> 3) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ uint32_t word_of(const uint4& v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Per block of MLP_RPB rows the gradient of sum(scale * loss) into partial[block][MLP_NW];
// dz: softmax - y per row (unscaled); h1, h2: the forward's BF16 activations.  A wait that gives
// up sets *status and writes NaN into the block's partial vector.
__global__ void __launch_bounds__(128, 1)
    mlp_backward_tc_kernel(MlpWeights w, const bf16* __restrict__ X, const float* __restrict__ dz, float scale, int R,
                           const bf16* __restrict__ h1, const bf16* __restrict__ h2, float* __restrict__ partial,
                           int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t tcb_smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tcb_smem + TCB_BAR);
    uint32_t* slot = reinterpret_cast<uint32_t*>(tcb_smem + TCB_SLOT);
    float* w3s = reinterpret_cast<float*>(tcb_smem + TCB_W3);
    // B of dh1 = dh2 W2: B[n][k] = W2[k][n] (n an h1 unit, k an h2 unit), K-major
    for (int e = tid; e < MLP_H * MLP_H; e += 128) {
        const int k = e >> 6, n = e & 63;
        *reinterpret_cast<bf16*>(tcb_smem + TCB_W2T + kmajor_off(n, k >> 3, 8) + (k & 7) * 2) = w.W2[e];
    }
    if (tid < MLP_H) w3s[tid] = __bfloat162float(w.w3[tid]);
    if (tid == 0) umma::mbar_init(bar, 1);
    if (warp == 0) umma::tmem_alloc(slot, TCB_COLS);
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t dh = tmem, dd = tmem + MLP_H;         // dh1 accumulator, gradient accumulator
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    constexpr uint32_t idesc_h = umma::IdescBf16<128, MLP_H>::value;
    constexpr uint32_t idesc_w = umma::IdescBf16<128, TCB_N, true, true>::value;
    const uint32_t ah = umma::smem_addr(tcb_smem + TCB_AH), w2t = umma::smem_addr(tcb_smem + TCB_W2T);
    const uint32_t aw = umma::smem_addr(tcb_smem + TCB_AW), bw = umma::smem_addr(tcb_smem + TCB_BW);
    uint32_t phase = 0;
    bool failed = false;
    const long long rbeg = (long long)blockIdx.x * MLP_RPB;
    for (int sub = 0; sub < 2 && !failed; ++sub) {
        const long long row = rbeg + 128 * sub + tid;
        const bool live = row < R;
        const float d = live ? dz[row] * scale : 0.f;
        uint4 h1v[8], h2v[8], xv[2];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            h1v[q] = live ? *reinterpret_cast<const uint4*>(h1 + (size_t)row * MLP_H + 8 * q) : make_uint4(0, 0, 0, 0);
            h2v[q] = live ? *reinterpret_cast<const uint4*>(h2 + (size_t)row * MLP_H + 8 * q) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            uint32_t x4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x4[i] = live ? ld32(X + (size_t)row * MLP_IN + 8 * q + 2 * i) : 0u;
            xv[q] = make_uint4(x4[0], x4[1], x4[2], x4[3]);
        }
        // dh2 = dz w3 where h2 > 0 (the constant unit 63 gets 0), BF16 pairs
        uint32_t dp[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const uint32_t hw = word_of(h2v[i >> 2], i & 3);
            const int c = 2 * i;
            const float a = bf16_lo(hw) > 0.f ? d * w3s[c] : 0.f;
            const float b = (c + 1 != MLP_H - 1 && bf16_hi(hw) > 0.f) ? d * w3s[c + 1] : 0.f;
            dp[i] = pack_bf16(a, b);
        }
        const uint32_t dzb = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(d));
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const uint4 v = make_uint4(dp[4 * g], dp[4 * g + 1], dp[4 * g + 2], dp[4 * g + 3]);
            *reinterpret_cast<uint4*>(tcb_smem + TCB_AH + kmajor_off(tid, g, 8)) = v;
            // the A operand of the gradient: unit 63 carries dz
            const uint4 u = g == 7 ? make_uint4(v.x, v.y, v.z, (v.w & 0xffffu) | (dzb << 16)) : v;
            *reinterpret_cast<uint4*>(tcb_smem + TCB_AW + mnmajor_off(tid, g)) = u;
            *reinterpret_cast<uint4*>(tcb_smem + TCB_BW + mnmajor_off(tid, g)) = h1v[g];
            *reinterpret_cast<uint4*>(tcb_smem + TCB_BW + mnmajor_off(tid, 10 + g)) = h2v[g];
        }
        *reinterpret_cast<uint4*>(tcb_smem + TCB_BW + mnmajor_off(tid, 8)) = xv[0];
        *reinterpret_cast<uint4*>(tcb_smem + TCB_BW + mnmajor_off(tid, 9)) = xv[1];
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
#pragma unroll
            for (int s = 0; s < 4; ++s)
                umma::mma_bf16(dh, umma::smem_desc(ah + 256u * s, 128, 1024), umma::smem_desc(w2t + 256u * s, 128, 1024),
                               idesc_h, s > 0 ? 1u : 0u);
            umma::commit(bar);
        }
        bool ok = umma::mbar_wait(bar, phase, TC_WAIT_NS);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        umma::fence_after_sync();
        // dh1 = (dh2 W2) where h1 > 0 (unit 63 gets 0), BF16, into units 64..127 of the A operand
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float acc[32];
            umma::tmem_ld32(dh + lanes + 32u * half, acc);
            uint32_t hp[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = 32 * half + 2 * i;
                const uint32_t hw = word_of(h1v[c >> 3], (c >> 1) & 3);
                const float a = bf16_lo(hw) > 0.f ? acc[2 * i] : 0.f;
                const float b = (c + 1 != MLP_H - 1 && bf16_hi(hw) > 0.f) ? acc[2 * i + 1] : 0.f;
                hp[i] = pack_bf16(a, b);
            }
#pragma unroll
            for (int g = 0; g < 4; ++g)
                *reinterpret_cast<uint4*>(tcb_smem + TCB_AW + mnmajor_off(tid, 8 + 4 * half + g)) =
                    make_uint4(hp[4 * g], hp[4 * g + 1], hp[4 * g + 2], hp[4 * g + 3]);
        }
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
#pragma unroll
            for (int s = 0; s < 8; ++s)
                umma::mma_bf16(dd, umma::smem_desc(aw + 256u * s, 128, 2048), umma::smem_desc(bw + 256u * s, 128, 2048),
                               idesc_w, (sub > 0 || s > 0) ? 1u : 0u);
            umma::commit(bar);
        }
        ok = umma::mbar_wait(bar, phase, TC_WAIT_NS);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        umma::fence_after_sync();
    }
    float* out = partial + (size_t)blockIdx.x * MLP_NW;
    if (!failed) {
        // thread t holds row t of D
        if (warp < 2) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float acc[32];
                umma::tmem_ld32(dd + lanes + 32u * half, acc);
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    out[MLP_H * MLP_IN + tid * MLP_H + 32 * half + i] = tid == MLP_H - 1 ? 0.f : acc[i];
            }
            if (warp == 1) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float acc[32];
                    umma::tmem_ld32(dd + lanes + 80u + 32u * half, acc);
                    if (tid == MLP_H - 1) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) out[MLP_H * MLP_IN + MLP_H * MLP_H + 32 * half + i] = acc[i];
                    }
                }
            }
        } else {
            float acc[32];
            umma::tmem_ld32(dd + lanes + 64u, acc);
#pragma unroll
            for (int i = 0; i < MLP_IN; ++i) out[(tid - MLP_H) * MLP_IN + i] = acc[i];
        }
    } else {
        if (tid == 0) atomicExch(status, 1);
        for (int e = tid; e < MLP_NW; e += 128) out[e] = __int_as_float(0x7fc00000);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, TCB_COLS);
    }
}

// Softmax cross-entropy per city over its k consecutive rows.  target: per city a bitmask of
// the candidate ranks that are best-tour neighbours (cities with no such rank are skipped).
// dz[row] = softmax - y; loss per city into city_loss (0 when skipped).
__global__ void mlp_loss_kernel(const float* __restrict__ z, const uint32_t* __restrict__ target, int cities, int k,
                                float* __restrict__ dz, float* __restrict__ city_loss) {
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < cities; c += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t tm = target[c];
        const float zi = lane < k ? z[(size_t)c * k + lane] : -FLT_MAX;
        float mx = zi;
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
        const float e = lane < k ? __expf(zi - mx) : 0.f;
        float se = e;
        for (int o = 16; o; o >>= 1) se += __shfl_xor_sync(FULL, se, o);
        const int nt = __popc(tm);
        const float y = (nt > 0 && ((tm >> lane) & 1u)) ? 1.f / (float)nt : 0.f;
        const float p = e / se;
        if (lane < k) dz[(size_t)c * k + lane] = nt > 0 ? p - y : 0.f;
        float l = (y > 0.f) ? -y * (zi - mx - __logf(se)) : 0.f;
        for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(FULL, l, o);
        if (lane == 0) city_loss[c] = nt > 0 ? l : 0.f;
    }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int blocks, int stride, int elems, float scale,
                                  float* __restrict__ grad) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < elems; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < blocks; ++b) s += partial[(size_t)b * stride + e];
        grad[e] = s * scale;
    }
}

// Adam on FP32 master weights; BF16 copies refreshed.  mask: 1 = trainable entry.
__global__ void mlp_adam_kernel(float* __restrict__ w, float* __restrict__ m1, float* __restrict__ m2,
                                const float* __restrict__ grad, const uint8_t* __restrict__ mask, int elems, float lr,
                                float b1, float b2, float eps, float c1, float c2, bf16* __restrict__ wb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < elems; e += gridDim.x * blockDim.x) {
        if (mask[e]) {
            const float gr = grad[e];
            const float a = b1 * m1[e] + (1.f - b1) * gr;
            const float bsq = b2 * m2[e] + (1.f - b2) * gr * gr;
            m1[e] = a;
            m2[e] = bsq;
            w[e] -= lr * (a / c1) / (sqrtf(bsq / c2) + eps);
        }
        wb[e] = __float2bfloat16_rn(w[e]);
    }
}

// ---------------------------------------------------------------- features of candidate edges
// Row (i, r) for candidate j = cand[i][r]:
//   f0 = d_ij / dbar_i (dbar_i = mean candidate distance of i), f1 = r / (k - 1),
//   f2 = (x_j - x_i) / dbar_i, f3 = (y_j - y_i) / dbar_i,
//   f4 = deg_j / 32 where deg_j = distinct neighbours of j over the l_best tours of ants 0 .. D-1,
//   f5 = 1 (bias input), f6..f15 = 0.
__global__ void edge_features_kernel(const double* __restrict__ xy, const int* __restrict__ cand, int n, int k,
                                     const int* __restrict__ deg, bf16* __restrict__ X) {
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        const double xi = xy[2 * i], yi = xy[2 * i + 1];
        double d = 0.0, dx = 0.0, dy = 0.0;
        int j = 0;
        if (lane < k) {
            j = cand[(size_t)i * k + lane];
            dx = xy[2 * j] - xi;
            dy = xy[2 * j + 1] - yi;
            d = sqrt(dx * dx + dy * dy);
        }
        float s = lane < k ? (float)d : 0.f;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        const float dbar = fmaxf(s / (float)k, 1e-30f);
        if (lane < k) {
            uint4* row = reinterpret_cast<uint4*>(X + ((size_t)i * k + lane) * MLP_IN);
            const float f1 = k > 1 ? (float)lane / (float)(k - 1) : 0.f;
            row[0] = make_uint4(pack_bf16((float)d / dbar, f1), pack_bf16((float)dx / dbar, (float)dy / dbar),
                                pack_bf16((float)deg[j] * (1.f / 32.f), 1.f), 0u);
            row[1] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// deg[j] = number of distinct cities among j's neighbours in the l_best tours of ants 0 .. D-1
// (D <= 16: at most 32 entries, one per lane; equal entries found with __match_any_sync).
__global__ void neighbour_degree_kernel(const int* __restrict__ nb, int n, int m, int D, int* __restrict__ deg) {
    const int lane = threadIdx.x & 31;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += (gridDim.x * blockDim.x) >> 5) {
        const int x = lane < 2 * D ? nb[(size_t)j * m * 2 + lane] : -1 - lane;  // distinct dummies
        const unsigned same = __match_any_sync(FULL, x);
        const bool first = lane < 2 * D && (__ffs(same) - 1) == lane;
        const int cnt = __popc(__ballot_sync(FULL, first));
        if (lane == 0) deg[j] = cnt;
    }
}


// best-tour labels: per city the bitmask of candidate ranks holding its two neighbours in the
// l_best tour of the best ant (the tour of length C_gbest).
__global__ void tour_labels_kernel(const uint8_t* __restrict__ nbrank, const int* __restrict__ gbest_ant, int n, int m,
                                   int k, uint32_t* __restrict__ target) {
    const int a = *gbest_ant;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t rs = nbrank[((size_t)i * m + a) * 2], rp = nbrank[((size_t)i * m + a) * 2 + 1];
        target[i] = (rs < (uint32_t)k ? 1u << rs : 0u) | (rp < (uint32_t)k ? 1u << rp : 0u);
    }
}

// Validate learned scores (finite and > 0), or convert them into the FP64 eta^beta table.
__global__ void check_scores_kernel(const float* __restrict__ score, long long count, int* __restrict__ errflag) {
    bool bad = false;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
        bad |= !(score[e] > 0.f && score[e] <= FLT_MAX);
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(errflag, DEVERR_BAD_SCORE);
}

__global__ void scores_to_eta_kernel(const float* __restrict__ score, const double* __restrict__ xy,
                                     const int* __restrict__ cand, int n, int k, double beta,
                                     double* __restrict__ etab) {
    const long long count = (long long)n * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
        if (score) {
            etab[e] = (double)score[e];
        } else {  // the plain heuristic, as the candidate-list builder computes it
            const int i = (int)(e / k), j = cand[e];
            etab[e] = eta_pow_from_d2(dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1]), beta);
        }
    }
}

__global__ void sum_kernel(const float* __restrict__ v, int count, float scale, float* __restrict__ out) {
    __shared__ float part[32];
    float s = 0.f;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += v[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = t * scale;
    }
}

// ---------------------------------------------------------------- the network handle

struct aco_mlp {
    cudaStream_t stream;
    long long max_rows;
    int step;
    float* w;       // FP32 master weights W1 | W2 | w3
    float* m1;      // Adam moments
    float* m2;
    float* grad;
    uint8_t* mask;  // trainable entries
    bf16* wb;       // BF16 copies used by the kernels
    float* z;       // max_rows
    float* dz;      // max_rows
    float* closs;   // max_rows (per city, cities <= rows)
    bf16* h1;       // max_rows * 64
    bf16* h2;
    float* partial; // blocks * MLP_NW: per block of MLP_RPB rows its part of the gradient
    int* status;    // set by a forward or backward whose wait for an MMA gave up
    int tc_grid;    // CTAs of the forward: resident CTAs per SM x SMs
    char err[256];
};

static MlpWeights weights_of(const aco_mlp* h) {
    return MlpWeights{h->wb, h->wb + MLP_H * MLP_IN, h->wb + MLP_H * MLP_IN + MLP_H * MLP_H};
}

static void host_mask(uint8_t* mk) {
    for (int u = 0; u < MLP_H; ++u)
        for (int c = 0; c < MLP_IN; ++c) mk[u * MLP_IN + c] = (u < MLP_H - 1 && c < 6) ? 1 : 0;
    for (int u = 0; u < MLP_H; ++u)
        for (int c = 0; c < MLP_H; ++c) mk[MLP_H * MLP_IN + u * MLP_H + c] = u < MLP_H - 1 ? 1 : 0;
    for (int c = 0; c < MLP_H; ++c) mk[MLP_H * MLP_IN + MLP_H * MLP_H + c] = 1;
}

static void free_mlp(aco_mlp* h) {
    void* ptrs[] = {h->w, h->m1, h->m2, h->grad, h->mask, h->wb, h->z, h->dz, h->closs,
                    h->h1, h->h2, h->partial, h->status};
    for (void* q : ptrs)
        if (q) cudaFree(q);
}

static int blocks_for(long long rows, int per_block) {
    long long b = (rows + per_block - 1) / per_block;
    return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

static aco_status mlp_launch_ok(aco_mlp* h, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return ACO_OK;
    snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
    return ACO_ERR_CUDA;
}

extern "C" const char* aco_mlp_last_error(const aco_mlp* h) { return h ? h->err : ""; }

// Launch shapes of the tensor-core kernels: their shared memory admits so few CTAs per SM that the
// CTAs' tensor-memory allocations (512 columns per SM) always fit and tcgen05.alloc never waits;
// refused otherwise.  Returns the forward's grid in h->tc_grid.
static aco_status setup_tc_kernel(aco_mlp* h, const void* kernel, int smem, int max_per_sm, const char* name,
                                  int* occ_out) {
    int occ = 0;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 128, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(h->err, sizeof(h->err), "%s setup: %s", name, cudaGetErrorString(e));
        return ACO_ERR_CUDA;
    }
    if (occ < 1 || occ > max_per_sm) {
        snprintf(h->err, sizeof(h->err), "%s setup: %d resident CTAs per SM (1..%d needed)", name, occ, max_per_sm);
        return ACO_ERR_CUDA;
    }
    *occ_out = occ;
    return ACO_OK;
}

static aco_status setup_forward_tc(aco_mlp* h) {
    int dev = 0, sms = 0, occ = 0, occ_b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        snprintf(h->err, sizeof(h->err), "tensor-core setup: no device");
        return ACO_ERR_CUDA;
    }
    aco_status st = setup_tc_kernel(h, (const void*)mlp_forward_tc_kernel, TC_SMEM, TC_MAX_CTAS_PER_SM, "forward", &occ);
    if (st == ACO_OK)
        st = setup_tc_kernel(h, (const void*)mlp_backward_tc_kernel, TCB_SMEM, TCB_MAX_CTAS_PER_SM, "backward", &occ_b);
    h->tc_grid = occ * sms;
    return st;
}

static void launch_forward(aco_mlp* h, const bf16* X, long long rows, float* z, float* score, float beta, bf16* h1,
                           bf16* h2) {
    const long long tiles = (rows + 127) / 128;
    const int grid = (int)(tiles < h->tc_grid ? tiles : h->tc_grid);
    mlp_forward_tc_kernel<<<grid, 128, TC_SMEM, h->stream>>>(weights_of(h), X, rows, z, score, beta, h1, h2, h->status);
}

extern "C" aco_status aco_mlp_create(const float* w_host, int64_t max_rows, void* stream, aco_mlp** out) {
    ACO_RANGE("aco_mlp_create");
    if (!out || !w_host || max_rows < 16 || max_rows > (1LL << 30)) return ACO_ERR_INVALID_ARG;
    *out = nullptr;
    for (int e = 0; e < MLP_NW; ++e)
        if (!isfinite(w_host[e])) return ACO_ERR_INVALID_ARG;
    aco_mlp* h = new (std::nothrow) aco_mlp();
    if (!h) return ACO_ERR_OOM;
    memset(h, 0, sizeof(*h));
    h->stream = (cudaStream_t)stream;
    h->max_rows = max_rows;
    const long long blocks = (max_rows + MLP_RPB - 1) / MLP_RPB;
    bool ok = true;
    ok &= cudaMalloc(&h->w, sizeof(float) * MLP_NW) == cudaSuccess;
    ok &= cudaMalloc(&h->m1, sizeof(float) * MLP_NW) == cudaSuccess;
    ok &= cudaMalloc(&h->m2, sizeof(float) * MLP_NW) == cudaSuccess;
    ok &= cudaMalloc(&h->grad, sizeof(float) * MLP_NW) == cudaSuccess;
    ok &= cudaMalloc(&h->mask, MLP_NW) == cudaSuccess;
    ok &= cudaMalloc(&h->wb, sizeof(bf16) * MLP_NW) == cudaSuccess;
    ok &= cudaMalloc(&h->z, sizeof(float) * max_rows) == cudaSuccess;
    ok &= cudaMalloc(&h->dz, sizeof(float) * max_rows) == cudaSuccess;
    ok &= cudaMalloc(&h->closs, sizeof(float) * max_rows) == cudaSuccess;
    ok &= cudaMalloc(&h->h1, sizeof(bf16) * MLP_H * max_rows) == cudaSuccess;
    ok &= cudaMalloc(&h->h2, sizeof(bf16) * MLP_H * max_rows) == cudaSuccess;
    ok &= cudaMalloc(&h->partial, sizeof(float) * MLP_NW * blocks) == cudaSuccess;
    ok &= cudaMalloc(&h->status, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_mlp(h);
        delete h;
        return ACO_ERR_OOM;
    }
    uint8_t mk[MLP_NW];
    host_mask(mk);
    float w0[MLP_NW];
    for (int e = 0; e < MLP_NW; ++e) w0[e] = mk[e] ? w_host[e] : 0.f;
    cudaMemcpyAsync(h->w, w0, sizeof(w0), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->mask, mk, sizeof(mk), cudaMemcpyHostToDevice, h->stream);
    cudaMemsetAsync(h->m1, 0, sizeof(float) * MLP_NW, h->stream);
    cudaMemsetAsync(h->m2, 0, sizeof(float) * MLP_NW, h->stream);
    cudaMemsetAsync(h->grad, 0, sizeof(float) * MLP_NW, h->stream);
    cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    // BF16 copies: an Adam step with zero learning rate leaves the masters and refreshes them
    mlp_adam_kernel<<<blocks_for(MLP_NW, 256), 256, 0, h->stream>>>(h->w, h->m1, h->m2, h->grad, h->mask, MLP_NW, 0.f,
                                                                    0.9f, 0.999f, 1e-8f, 1.f, 1.f, h->wb);
    aco_status st = mlp_launch_ok(h, "create");
    if (st == ACO_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = ACO_ERR_CUDA;
    if (st == ACO_OK) st = setup_forward_tc(h);
    if (st != ACO_OK) {
        free_mlp(h);
        delete h;
        return st;
    }
    *out = h;
    return ACO_OK;
}

extern "C" void aco_mlp_destroy(aco_mlp* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_mlp(h);
    delete h;
}

extern "C" aco_status aco_mlp_get_weights(aco_mlp* h, float* w_host) {
    if (!h || !w_host) return ACO_ERR_INVALID_ARG;
    int failed = 0;
    cudaError_t e = cudaMemcpyAsync(w_host, h->w, sizeof(float) * MLP_NW, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&failed, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        snprintf(h->err, sizeof(h->err), "get_weights: %s", cudaGetErrorString(e));
        return ACO_ERR_CUDA;
    }
    if (failed) {
        snprintf(h->err, sizeof(h->err), "a forward or backward pass gave up waiting for a tensor-core MMA");
        return ACO_ERR_TIMEOUT;
    }
    return ACO_OK;
}

extern "C" aco_status aco_mlp_forward(aco_mlp* h, const uint16_t* X_dev, int64_t rows, float* z_dev,
                                      float* score_dev, float beta) {
    ACO_RANGE("aco_mlp_forward");
    if (!h || !X_dev || rows < 0 || (!z_dev && !score_dev) || !isfinite(beta)) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(X_dev, 4) || aco_misaligned(z_dev, 4) || aco_misaligned(score_dev, 4)) return ACO_ERR_INVALID_ARG;
    if (rows == 0) return ACO_OK;
    launch_forward(h, (const bf16*)X_dev, rows, z_dev, score_dev, beta, nullptr, nullptr);
    return mlp_launch_ok(h, "mlp_forward_tc_kernel");
}

// forward with stored activations, loss, backward: gradient of scale * (summed loss) into
// h->grad; the loss into loss_dev[0] if given.
static aco_status mlp_backward(aco_mlp* h, const bf16* X, const uint32_t* target, int cities, int k, float scale,
                               float* loss_dev) {
    const int rows = cities * k;
    cudaStream_t s = h->stream;
    launch_forward(h, X, rows, h->z, nullptr, 1.f, h->h1, h->h2);
    mlp_loss_kernel<<<blocks_for(cities, 8), 256, 0, s>>>(h->z, target, cities, k, h->dz, h->closs);
    if (loss_dev) sum_kernel<<<1, 1024, 0, s>>>(h->closs, cities, scale, loss_dev);
    const int blocks = (rows + MLP_RPB - 1) / MLP_RPB;
    mlp_backward_tc_kernel<<<blocks, 128, TCB_SMEM, s>>>(weights_of(h), X, h->dz, scale, rows, h->h1, h->h2,
                                                         h->partial, h->status);
    mlp_reduce_kernel<<<blocks_for(MLP_NW, 256), 256, 0, s>>>(h->partial, blocks, MLP_NW, MLP_NW, 1.f, h->grad);
    return mlp_launch_ok(h, "mlp backward");
}

extern "C" aco_status aco_mlp_backward(aco_mlp* h, const uint16_t* X_dev, const uint32_t* target_dev, int32_t cities,
                                       int32_t k, float scale, float* grad_dev, float* loss_dev) {
    ACO_RANGE("aco_mlp_backward");
    if (!h || !X_dev || !target_dev || cities < 1 || k < 1 || k > 32 || !isfinite(scale)) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(X_dev, 4) || aco_misaligned(target_dev, 4) || aco_misaligned(grad_dev, 4) || aco_misaligned(loss_dev, 4))
        return ACO_ERR_INVALID_ARG;
    if ((long long)cities * k > h->max_rows) return ACO_ERR_INVALID_ARG;
    aco_status st = mlp_backward(h, (const bf16*)X_dev, target_dev, cities, k, scale, loss_dev);
    if (st == ACO_OK && grad_dev)
        cudaMemcpyAsync(grad_dev, h->grad, sizeof(float) * MLP_NW, cudaMemcpyDeviceToDevice, h->stream);
    return st == ACO_OK ? mlp_launch_ok(h, "backward copy") : st;
}

static aco_status mlp_adam(aco_mlp* h, const float* grad, float lr) {
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)h->step), c2 = 1.f - powf(b2, (float)h->step);
    mlp_adam_kernel<<<blocks_for(MLP_NW, 256), 256, 0, h->stream>>>(h->w, h->m1, h->m2, grad, h->mask, MLP_NW, lr, b1,
                                                                    b2, 1e-8f, c1, c2, h->wb);
    return mlp_launch_ok(h, "mlp_adam_kernel");
}

extern "C" aco_status aco_mlp_adam(aco_mlp* h, const float* grad_dev, float lr) {
    ACO_RANGE("aco_mlp_adam");
    if (!h || !(lr >= 0.f) || !isfinite(lr)) return ACO_ERR_INVALID_ARG;
    return mlp_adam(h, grad_dev ? grad_dev : h->grad, lr);
}

extern "C" aco_status aco_mlp_train(aco_mlp* h, const uint16_t* X_dev, const uint32_t* target_dev, int32_t cities,
                                    int32_t k, int32_t batch_cities, int32_t steps, float lr, float* loss_dev) {
    ACO_RANGE("aco_mlp_train");
    if (!h || !X_dev || !target_dev || cities < 1 || k < 1 || k > 32 || batch_cities < 1 || steps < 0 ||
        !(lr >= 0.f) || !isfinite(lr))
        return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(X_dev, 4) || aco_misaligned(target_dev, 4) || aco_misaligned(loss_dev, 4)) return ACO_ERR_INVALID_ARG;
    if ((long long)batch_cities * k > h->max_rows) return ACO_ERR_INVALID_ARG;
    const bf16* X = (const bf16*)X_dev;
    const int nb = (cities + batch_cities - 1) / batch_cities;
    for (int t = 0; t < steps; ++t) {
        const int b = t % nb;
        const int c0 = b * batch_cities;
        const int cn = cities - c0 < batch_cities ? cities - c0 : batch_cities;
        aco_status st = mlp_backward(h, X + (size_t)c0 * k * MLP_IN, target_dev + c0, cn, k, 1.f / (float)cn,
                                     loss_dev ? loss_dev + t : nullptr);
        if (st != ACO_OK) return st;
        st = mlp_adam(h, h->grad, lr);
        if (st != ACO_OK) return st;
    }
    return ACO_OK;
}

// ---------------------------------------------------------------- instance side
extern "C" aco_status aco_edge_features(aco_instance* inst, int32_t degree_ants, uint16_t* X_dev) {
    ACO_RANGE("aco_edge_features");
    if (!inst || !X_dev) return ACO_ERR_INVALID_ARG;
    // a feature row (16 BF16 values) is written as two 16-byte words
    if (aco_misaligned(X_dev, 16)) return set_err(inst, ACO_ERR_INVALID_ARG, "edge_features: X_dev not 16-byte aligned");
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL || !inst->cand_built || !inst->initialized)
        return set_err(inst, ACO_ERR_STATE, "edge_features: needs candidate lists and l_best tours");
    if (degree_ants < 1 || degree_ants > 16 || degree_ants > inst->p.m)
        return set_err(inst, ACO_ERR_INVALID_ARG, "edge_features: degree_ants must be in 1 .. min(m, 16)");
    const int n = inst->p.n, k = inst->p.k;
    neighbour_degree_kernel<<<blocks_for(n, 8), 256, 0, inst->stream>>>(inst->nb, n, inst->p.m, degree_ants, inst->deg);
    edge_features_kernel<<<blocks_for(n, 8), 256, 0, inst->stream>>>(inst->xy, inst->cand, n, k, inst->deg, (bf16*)X_dev);
    return check_launch(inst, "edge_features_kernel");
}

extern "C" aco_status aco_tour_labels(aco_instance* inst, uint32_t* target_dev) {
    ACO_RANGE("aco_tour_labels");
    if (!inst || !target_dev) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(target_dev, 4)) return set_err(inst, ACO_ERR_INVALID_ARG, "tour_labels: target_dev not 4-byte aligned");
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL || !inst->initialized)
        return set_err(inst, ACO_ERR_STATE, "tour_labels: needs l_best tours");
    if (inst->p.k > 32) return set_err(inst, ACO_ERR_INVALID_ARG, "tour_labels: k > 32");
    tour_labels_kernel<<<blocks_for(inst->p.n, 256), 256, 0, inst->stream>>>(inst->nbrank, inst->gbest_ant, inst->p.n,
                                                                            inst->p.m, inst->p.k, target_dev);
    return check_launch(inst, "tour_labels_kernel");
}

extern "C" aco_status aco_set_edge_scores(aco_instance* inst, const float* score_dev) {
    ACO_RANGE("aco_set_edge_scores");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(score_dev, 4)) return set_err(inst, ACO_ERR_INVALID_ARG, "set_edge_scores: score_dev not 4-byte aligned");
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL || !inst->cand_built)
        return set_err(inst, ACO_ERR_STATE, "set_edge_scores: needs candidate lists");
    if (inst->constructed) return set_err(inst, ACO_ERR_STATE, "set_edge_scores: tours constructed, update pending");
    const long long count = (long long)inst->p.n * inst->p.k;
    if (score_dev) {
        check_scores_kernel<<<blocks_for(count, 256), 256, 0, inst->stream>>>(score_dev, count, inst->errflag);
        aco_status st = check_launch(inst, "check_scores_kernel");
        if (st == ACO_OK) st = sync_and_check(inst, "set_edge_scores");
        if (st != ACO_OK) return st;
    }
    scores_to_eta_kernel<<<blocks_for(count, 256), 256, 0, inst->stream>>>(score_dev, inst->xy, inst->cand, inst->p.n,
                                                                          inst->p.k, inst->p.beta, inst->etab);
    aco_status st = check_launch(inst, "scores_to_eta_kernel");
    if (st != ACO_OK) return st;
    st = launch_reweight(inst);
    if (st != ACO_OK) return st;
    inst->scored = score_dev != nullptr;
    return ACO_OK;
}

// update_dev.cuh -- device steps of the l_best update (Algorithm 1's replacement, C_gbest and the
// Section 3 pheromone of the candidate edges), shared by the update kernels of update.cu and the
// persistent batched kernel.
#pragma once
#include <float.h>
#include <math.h>

#include "common.cuh"

// Neighbour entries of city c in ant a's l_best: successor, predecessor and their candidate ranks.
__device__ __forceinline__ void set_neighbours(int* __restrict__ nb, uint8_t* __restrict__ nbrank,
                                               const int* __restrict__ cand, int m, int k, int a, int c, int succ,
                                               int pred) {
    const size_t e = ((size_t)c * m + a) * 2;  // even: the pair is 8-byte (ids) and 2-byte (ranks) aligned
    *reinterpret_cast<int2*>(nb + e) = make_int2(succ, pred);
    uint8_t rs, rp;
    ranks_of(cand, k, c, succ, pred, rs, rp);
    *reinterpret_cast<uint16_t*>(nbrank + e) = (uint16_t)(rs | (rp << 8));
}

// Algorithm 1's replacement for ant a (one warp): when the new tour is strictly shorter than the
// ant's l_best it becomes the l_best: the rebuilt positions (or the whole tour), the neighbour
// entries of the cities they touch, the length and its exact fixed-point value.
// NT threads take the ant (a warp, or a whole block when NT > 32); thread `lane` of them.  Every
// thread reads C_lbest before the first synchronisation and thread 0 writes it after the last.
template <int NT>
__device__ __forceinline__ void group_sync() {
    if (NT == 32) __syncwarp();
    else __syncthreads();
}

template <int NT = 32>
__device__ __forceinline__ void commit_ant(const CommitArgs& C, int a, int lane) {
    const int n = C.n, m = C.m, k = C.k;
    const AntIter it = C.antit[a];
    if (!(it.newlen < C.clen[a])) return;
    int* L = C.lbest + (size_t)a * n;
    const int* S = C.seg + (size_t)a * n;
    if (it.s < 0) {
        for (int t = lane; t < n; t += NT) L[t] = S[t];
        group_sync<NT>();
        for (int t = lane; t < n; t += NT)
            set_neighbours(C.nb, C.nbrank, C.cand, m, k, a, S[t], S[t + 1 == n ? 0 : t + 1], S[t == 0 ? n - 1 : t - 1]);
    } else {
        const int e = L[(it.s + it.P - 1) % n];
        const int start = L[it.s];
        const int M = it.M;
        group_sync<NT>();
        for (int t = lane; t < M; t += NT) L[(it.s + it.P + t) % n] = S[t];
        for (int t = lane; t < M; t += NT) {
            const int pc = t == 0 ? e : S[t - 1];
            const int sc = t == M - 1 ? start : S[t + 1];
            set_neighbours(C.nb, C.nbrank, C.cand, m, k, a, S[t], sc, pc);
        }
        if (lane == 0) {
            const size_t ee = ((size_t)e * m + a) * 2;
            C.nb[ee] = S[0];
            C.nbrank[ee] = rank_of(C.cand, k, e, S[0]);
            const size_t es = ((size_t)start * m + a) * 2 + 1;
            C.nb[es] = S[M - 1];
            C.nbrank[es] = rank_of(C.cand, k, start, S[M - 1]);
        }
    }
    if (lane == 0) {
        C.clen[a] = it.newlen;
        C.cfix[2 * a] = it.fix_lo;
        C.cfix[2 * a + 1] = it.fix_hi;
        atomicAdd(&C.counters[CNT_IMPROVED], 1ull);
    }
}

// C_gbest = min_a C_a (lowest ant among equals) and every ant's deposit weight
// q_a = round(C_gbest / C_a * 2^32), by one warp (the same values as gbest_q_kernel).
__device__ __forceinline__ void gbest_warp(const GbestArgs& G, int lane) {
    const int m = G.m;
    double v = DBL_MAX * 2;  // +inf
    int idx = 0x7fffffff;
    for (int a = lane; a < m; a += 32) {
        const double c = G.clen[a];
        if (c < v || (c == v && a < idx)) { v = c; idx = a; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (G.keep_prev && !(v < *G.gbest)) {
        v = *G.gbest;
        idx = *G.gbest_ant;
    }
    __syncwarp();
    if (lane == 0) {
        *G.gbest = v;
        *G.gbest_ant = idx;
    }
    if (G.q)
        for (int a = lane; a < m; a += 32) G.q[a] = __double2ull_rn(__dmul_rn(__ddiv_rn(v, G.clen[a]), 4294967296.0));
}

// The pheromone row of city i from its integer sum Q (lane r < k holds rank r): tau = tau0 +
// Q 2^-32, the Eq. 1 weight tau^alpha eta^beta in FP64 and its FP32 screen copy (negative for the
// whole row when some weight is not FP32-normal), the row flag and, when kept, Q itself.
__device__ __forceinline__ void finish_row(const RebuildArgs& R, int i, unsigned long long Q, double eta, int lane) {
    const int k = R.k;
    bool flag = false;
    float w32 = 0.f;
    if (lane < k) {
        const size_t e = (size_t)i * k + lane;
        const double tau = __dadd_rn(R.tau0, __dmul_rn(__ull2double_rn(Q), 0x1.0p-32));
        const double wv = __dmul_rn(R.ia >= 0 ? pow_int(tau, R.ia) : powr(tau, R.alpha), eta);
        w32 = __double2float_rn(wv);
        // not finite: all exponent bits set (tested on the bit pattern, off the FP64 pipe)
        if ((__double_as_longlong(wv) & 0x7ff0000000000000LL) == 0x7ff0000000000000LL)
            atomicOr(R.errflag, DEVERR_NONFINITE);
        flag = !(w32 >= FLT_MIN && w32 <= FLT_MAX);
        R.W64[e] = wv;
        if (R.Qt) R.Qt[e] = Q;
    }
    const unsigned fl = __ballot_sync(0xffffffffu, flag);
    // a row the FP32 screen cannot represent carries negative screen weights: the construction
    // kernel then evaluates it exactly in FP64
    if (lane < k) R.candw[(size_t)i * k + lane].w = fl ? -1.0f : w32;
    if (lane == 0) R.rowflag[i] = fl ? 1 : 0;
}

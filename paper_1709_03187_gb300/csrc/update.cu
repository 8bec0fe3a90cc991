// update.cu -- pheromone update and tour lengths.
//
// Scalable form (Section 3, Algorithm 1):
//   commit_kernel      l_best_a <- new tour when strictly shorter (Algorithm 1, last step of the
//                      ant loop); rewrites only the rebuilt positions and the neighbour entries
//                      (succ, pred and their candidate ranks) of the M + 2 cities they touch.
//   gbest_q_kernel     C_gbest = min_a C_a (lowest ant on ties); per-ant deposit weight
//                      q_a = round(C_gbest / C_a * 2^32)  (Section 3: quality of g_best over
//                      quality of l_best, in (0, 1]).
//   rebuild_kernel     the pheromone of every candidate edge,
//                      Q_ir = sum_a q_a [cand_ir is succ_a(i) or pred_a(i)],
//                      tau_ir = tau0 + Q_ir 2^-32, and the Eq. 1 weight tau^alpha eta^beta in
//                      FP64 plus its FP32 screen copy.  Edges of replaced l_best tours have
//                      dropped out of the neighbour table (the P-ACO form of evaporation) and
//                      the new ones entered (deposit).  This is a streaming pass over the
//                      n x m table of neighbour ranks (2 bytes per city and ant).
// Dense form (Section 2): Eq. 2 then Eq. 3-5 on the n x n matrix.
// Tour lengths: exact 2^-96 fixed-point sums (order-free), one rounding.
#include <float.h>
#include <math.h>

#include "common.cuh"
#include "update_dev.cuh"

#define FULL 0xffffffffu

// One block of NT threads per ant (a warp for the batched colonies, where block b is ant slot b,
// naming (instance, ant); a wider block for a single colony, so that the longest rebuilt segment
// is spread over more threads).
template <bool BATCH, int NT>
__global__ void __launch_bounds__(NT) commit_kernel(const __grid_constant__ CommitArgs Cp,
                                                    const CommitArgs* __restrict__ batch, const int2* __restrict__ slot,
                                                    int slots, int ant0) {
    int a = ant0 + (int)blockIdx.x, inst = 0;
    if (BATCH) {
        if ((int)blockIdx.x >= slots) return;
        const int2 sa = slot[blockIdx.x];
        inst = sa.x;
        a = sa.y;
    }
    const CommitArgs& C = BATCH ? batch[inst] : Cp;
    commit_ant<NT>(C, a, threadIdx.x);
}

// One block per colony: C_gbest, its ant, and the per-ant deposit weights.  keep_prev: fold in
// the previous g_best (dense mode keeps the best over all iterations).
template <bool BATCH>
__global__ void gbest_q_kernel(const __grid_constant__ GbestArgs Gp, const GbestArgs* __restrict__ batch) {
    const GbestArgs& G = BATCH ? batch[blockIdx.x] : Gp;
    const int m = G.m;
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ double cg_s;
    double v = DBL_MAX * 2;  // +inf
    int idx = 0x7fffffff;
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
        const double c = G.clen[a];
        if (c < v || (c == v && a < idx)) { v = c; idx = a; }
    }
    for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(FULL, v, o);
        const int oi = __shfl_xor_sync(FULL, idx, o);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = v; si[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] < v || (sv[w] == v && si[w] < idx)) { v = sv[w]; idx = si[w]; }
        if (G.keep_prev && !(v < *G.gbest)) {
            v = *G.gbest;
            idx = *G.gbest_ant;
        }
        *G.gbest = v;
        *G.gbest_ant = idx;
        cg_s = v;
    }
    __syncthreads();
    if (G.q) {
        const double cg = cg_s;
        for (int a = threadIdx.x; a < m; a += blockDim.x)
            G.q[a] = __double2ull_rn(__dmul_rn(__ddiv_rn(cg, G.clen[a]), 4294967296.0));
    }
}

// One warp per city; lane-private histograms in shared memory (conflict-free column per lane).
// Single colony: warps stride over all cities.  Batched colonies: block b covers the city range
// blockmap[b] = (instance, first city, end city) of one instance.
template <bool BATCH>
__global__ void __launch_bounds__(256) rebuild_kernel(const __grid_constant__ RebuildArgs Rp,
                                                      const RebuildArgs* __restrict__ batch,
                                                      const int4* __restrict__ blockmap) {
    extern __shared__ unsigned long long sm[];
    int4 bm = make_int4(0, 0, 0, 0);
    if (BATCH) bm = blockmap[blockIdx.x];
    const RebuildArgs& R = BATCH ? batch[bm.x] : Rp;
    const int n = R.n, m = R.m, k = R.k, use_ants = R.use_ants;
    const double tau0 = R.tau0, alpha = R.alpha;
    const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_cap = BATCH ? R.m_cap : m;
    unsigned long long* qs = sm;                                      // m
    unsigned long long* hist = sm + m_cap + (size_t)w * k * 32;      // [k][32]

    if (use_ants)
        for (int a = threadIdx.x; a < m; a += blockDim.x) qs[a] = R.q[a];
    __syncthreads();
    const bool vec = (m & 7) == 0;
    const int i0 = BATCH ? bm.y + w : blockIdx.x * warps + w;
    const int iend = BATCH ? bm.z : n;
    const int istep = BATCH ? warps : gridDim.x * warps;
    // m <= 1024, m % 8 == 0: lane l always holds the ranks of ants hb * 256 + 8 l .. + 7
    // (hb < 4), so their weights stay in registers for every city of the warp
    const bool regq = use_ants && vec && m <= 1024;
    unsigned long long qr[4][8];
    if (regq) {
#pragma unroll
        for (int hb = 0; hb < 4; ++hb)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int a = hb * 256 + lane * 8 + j;
                qr[hb][j] = a < m ? qs[a] : 0ull;
            }
    }
    uint4 nxt[4];  // rank bytes of the warp's next city (fast path), requested one city ahead
    double enxt = 0.0;  // and its eta^beta entry of this lane's rank
    if (regq && i0 < iend && lane < k) enxt = R.etab[(size_t)i0 * k + lane];
    if (regq && i0 < iend) {
        const uint8_t* row = R.nbrank + (size_t)i0 * m * 2;
#pragma unroll
        for (int hb = 0; hb < 4; ++hb) {
            const int a0 = hb * 256 + lane * 8;
            nxt[hb] = a0 < m ? __ldcs(reinterpret_cast<const uint4*>(row + 2 * (size_t)a0)) : make_uint4(~0u, ~0u, ~0u, ~0u);
        }
    }
    for (int i = i0; i < iend; i += istep) {
        unsigned long long Q = 0;
        double ecur = -1.0;  // eta^beta of (i, lane) when prefetched, else read below
        if (use_ants) {
            for (int r = 0; r < k; ++r) hist[r * 32 + lane] = 0ull;
            const uint8_t* row = R.nbrank + (size_t)i * m * 2;
            if (regq) {
                uint4 v[4];
#pragma unroll
                for (int hb = 0; hb < 4; ++hb) v[hb] = nxt[hb];
                ecur = enxt;
                if (i + istep < iend && lane < k) enxt = R.etab[(size_t)(i + istep) * k + lane];
                if (i + istep < iend) {
                    const uint8_t* nrow = R.nbrank + (size_t)(i + istep) * m * 2;
#pragma unroll
                    for (int hb = 0; hb < 4; ++hb) {
                        const int a0 = hb * 256 + lane * 8;
                        nxt[hb] = a0 < m ? __ldcs(reinterpret_cast<const uint4*>(nrow + 2 * (size_t)a0))
                                         : make_uint4(~0u, ~0u, ~0u, ~0u);
                    }
                }
                unsigned long long* hl = hist + lane;
#pragma unroll
                for (int hb = 0; hb < 4; ++hb) {
                    const uint32_t wv[4] = {v[hb].x, v[hb].y, v[hb].z, v[hb].w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const uint32_t r = (wv[h] >> (8 * b)) & 0xFFu;
                            if (r < (uint32_t)k) hl[r * 32] += qr[hb][2 * h + (b >> 1)];
                        }
                    }
                }
            } else if (vec) {
                // the row's rank bytes, four 16-byte loads per lane in flight
                for (int base = 0; base < m; base += 1024) {
                    uint4 v[4];
#pragma unroll
                    for (int hb = 0; hb < 4; ++hb) {
                        const int a0 = base + hb * 256 + lane * 8;
                        v[hb] = a0 < m ? __ldcs(reinterpret_cast<const uint4*>(row + 2 * (size_t)a0))
                                       : make_uint4(~0u, ~0u, ~0u, ~0u);
                    }
#pragma unroll
                    for (int hb = 0; hb < 4; ++hb) {
                        const int a0 = base + hb * 256 + lane * 8;
                        const uint32_t wv[4] = {v[hb].x, v[hb].y, v[hb].z, v[hb].w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
#pragma unroll
                            for (int g = 0; g < 2; ++g) {
                                const uint32_t pair = wv[h] >> (16 * g);
                                const uint32_t rs = pair & 0xFFu, rp = (pair >> 8) & 0xFFu;
                                if (rs < (uint32_t)k || rp < (uint32_t)k) {
                                    const unsigned long long qa = qs[a0 + 2 * h + g];
                                    if (rs < (uint32_t)k) hist[rs * 32 + lane] += qa;
                                    if (rp < (uint32_t)k) hist[rp * 32 + lane] += qa;
                                }
                            }
                        }
                    }
                }
            } else {
                for (int a = lane; a < m; a += 32) {
                    const uint32_t rs = row[2 * a], rp = row[2 * a + 1];
                    const unsigned long long qa = qs[a];
                    if (rs < (uint32_t)k) hist[rs * 32 + lane] += qa;
                    if (rp < (uint32_t)k) hist[rp * 32 + lane] += qa;
                }
            }
            __syncwarp();
            if (lane < k) {
                // lane r sums the 32 columns of rank r starting at column r (conflict-free banks),
                // in four independent integer chains
                const unsigned long long* h = hist + lane * 32;
                unsigned long long q4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                for (int l = 0; l < 32; ++l) q4[l & 3] += h[(l + lane) & 31];
                Q = (q4[0] + q4[1]) + (q4[2] + q4[3]);
            }
            __syncwarp();
        }
        const double eta = lane < k ? (regq ? ecur : R.etab[(size_t)i * k + lane]) : 0.0;
        finish_row(R, i, Q, eta, lane);
    }
}

void fill_commit_args(const aco_instance* inst, CommitArgs& C) {
    C.n = inst->p.n; C.m = inst->p.m; C.k = inst->p.k; C.cand = inst->cand; C.lbest = inst->lbest; C.nb = inst->nb;
    C.nbrank = inst->nbrank; C.seg = inst->seg; C.antit = inst->antit; C.clen = inst->clen; C.cfix = inst->cfix;
    C.counters = inst->counters;
}

void fill_gbest_args(const aco_instance* inst, int keep_prev, GbestArgs& G) {
    G.m = inst->p.m; G.clen = inst->clen; G.gbest = inst->gbest; G.gbest_ant = inst->gbest_ant;
    G.q = inst->p.mode == ACO_MODE_LBEST_PARTIAL ? inst->q : nullptr; G.keep_prev = keep_prev;
}

void fill_rebuild_args(const aco_instance* inst, int use_ants, RebuildArgs& R) {
    const aco_params& p = inst->p;
    R.n = p.n; R.m = p.m; R.k = p.k; R.tau0 = p.tau0; R.alpha = p.alpha; R.use_ants = use_ants; R.m_cap = p.m;
    R.ia = (p.alpha >= 0.0 && p.alpha <= 64.0 && floor(p.alpha) == p.alpha) ? (int)p.alpha : -1;
    R.nbrank = inst->nbrank; R.q = inst->q; R.etab = inst->etab; R.candw = inst->candw; R.W64 = inst->W64;
    R.rowflag = inst->rowflag; R.errflag = inst->errflag;
    R.Qt = inst->Qt;
}

size_t rebuild_smem_bytes(int m_cap, int k, int warps) {
    return sizeof(unsigned long long) * ((size_t)m_cap + (size_t)warps * k * 32);
}

static aco_status launch_rebuild(aco_instance* inst, int use_ants) {
    const aco_params& p = inst->p;
    const int warps = 8;
    RebuildArgs R;
    fill_rebuild_args(inst, use_ants, R);
    const size_t smem = rebuild_smem_bytes(p.m, p.k, warps);
    const int blocks = (int)fmin((double)inst->num_sms * 4, (double)ceil_div(p.n, warps));
    cudaFuncSetAttribute(rebuild_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rebuild_kernel<false><<<blocks, 32 * warps, smem, inst->stream>>>(R, nullptr, nullptr);
    return check_launch(inst, "rebuild_kernel");
}

// Batched update: commit (one block per ant slot), C_gbest (one block per colony), rebuild
// (block map over every colony's cities).
cudaError_t launch_update_batch(const CommitArgs* cargs, const int2* slot, int slots, const GbestArgs* gargs,
                                int count, const RebuildArgs* rargs, const int4* blockmap, int rblocks, int m_cap,
                                int k, cudaStream_t s) {
    CommitArgs c0{};
    commit_kernel<true, 32><<<slots, 32, 0, s>>>(c0, cargs, slot, slots, 0);
    GbestArgs g0{};
    gbest_q_kernel<true><<<count, 256, 0, s>>>(g0, gargs);
    RebuildArgs r0{};
    const size_t smem = rebuild_smem_bytes(m_cap, k, 8);
    if (smem > 48 * 1024) cudaFuncSetAttribute(rebuild_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rebuild_kernel<true><<<rblocks, 256, smem, s>>>(r0, rargs, blockmap);
    return cudaGetLastError();
}

__global__ void fill_inf_kernel(double* __restrict__ v, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) v[i] = INFINITY;
}

aco_status launch_lbest_init_weights(aco_instance* inst) {
    // C_lbest = +inf: the first tour of every ant is accepted (Algorithm 1, initial tours)
    fill_inf_kernel<<<ceil_div(inst->p.m, 256), 256, 0, inst->stream>>>(inst->clen, inst->p.m);
    fill_inf_kernel<<<1, 32, 0, inst->stream>>>(inst->gbest, 1);
    aco_status st = check_launch(inst, "fill_inf_kernel");
    if (st != ACO_OK) return st;
    return launch_rebuild(inst, 0);
}

// Candidate-edge weights recomputed from the current eta^beta table (after the table changes).
aco_status launch_reweight(aco_instance* inst) { return launch_rebuild(inst, inst->initialized ? 1 : 0); }

aco_status launch_update_lbest(aco_instance* inst) {
    const aco_params& p = inst->p;
    CommitArgs C;
    fill_commit_args(inst, C);
    if (!inst->initialized) {
        // the first commit: every ant writes a whole tour's entries at random cities of the
        // neighbour tables, one 1024-thread block per ant, 128 ants per launch (the first update
        // at 200,000 cities measured 13.9 ms so, against 16.0 ms in launches of 64 ants, 31.6 ms
        // of 32 and 14.0-14.3 ms with every ant in one launch)
        constexpr int G = 128;
        for (int a0 = 0; a0 < p.m; a0 += G)
            commit_kernel<false, 1024><<<p.m - a0 < G ? p.m - a0 : G, 1024, 0, inst->stream>>>(C, nullptr, nullptr, 0,
                                                                                               a0);
    } else {
        commit_kernel<false, 256><<<p.m, 256, 0, inst->stream>>>(C, nullptr, nullptr, 0, 0);
    }
    aco_status st = check_launch(inst, "commit_kernel");
    if (st != ACO_OK) return st;
    GbestArgs G;
    fill_gbest_args(inst, 0, G);
    gbest_q_kernel<false><<<1, 1024, 0, inst->stream>>>(G, nullptr);
    st = check_launch(inst, "gbest_q_kernel");
    if (st != ACO_OK) return st;
    return launch_rebuild(inst, 1);
}

// ------------------------------------------------------------------ exact tour lengths
__global__ void tour_length_kernel(const double* __restrict__ xy, const int* __restrict__ tours, int n, int count,
                                   double* __restrict__ out_len, unsigned long long* __restrict__ out_fix,
                                   int* __restrict__ errflag) {
    __shared__ unsigned long long red[2][32];
    for (int c = blockIdx.x; c < count; c += gridDim.x) {
        const int* T = tours + (size_t)c * n;
        u128 acc = 0;
        bool bad = false;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int i = T[p], j = T[p + 1 == n ? 0 : p + 1];
            if ((unsigned)i >= (unsigned)n || (unsigned)j >= (unsigned)n) { bad = true; continue; }
            acc += len_to_fix(__dsqrt_rn(dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1])));
        }
        if (bad) atomicOr(errflag, DEVERR_BAD_TOUR);
        acc = warp_sum_u128(acc);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) { red[0][w] = (unsigned long long)acc; red[1][w] = (unsigned long long)(acc >> 64); }
        __syncthreads();
        if (threadIdx.x == 0) {
            u128 t = 0;
            for (int v = 0; v < (int)(blockDim.x >> 5); ++v) t += (((u128)red[1][v]) << 64) | red[0][v];
            out_len[c] = fix_to_len(t);
            if (out_fix) { out_fix[2 * c] = (unsigned long long)t; out_fix[2 * c + 1] = (unsigned long long)(t >> 64); }
        }
        __syncthreads();
    }
}

aco_status launch_tour_lengths(aco_instance* inst, const int32_t* tours, int32_t count, double* out) {
    const int blocks = (int)fmin((double)count, (double)inst->num_sms * 8);
    tour_length_kernel<<<blocks, 256, 0, inst->stream>>>(inst->xy, tours, inst->p.n, count, out, nullptr,
                                                         inst->errflag);
    return check_launch(inst, "tour_length_kernel");
}

// ------------------------------------------------------------------ checkpoint restore
__global__ void neighbours_all_kernel(int n, int m, int k, const int* __restrict__ cand,
                                      const int* __restrict__ lbest, int* __restrict__ nb,
                                      uint8_t* __restrict__ nbrank) {
    const long long total = (long long)n * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / n), t = (int)(e % n);
        const int* L = lbest + (size_t)a * n;
        set_neighbours(nb, nbrank, cand, m, k, a, L[t], L[t + 1 == n ? 0 : t + 1], L[t == 0 ? n - 1 : t - 1]);
    }
}

aco_status launch_set_lbest(aco_instance* inst, const int32_t* lbest) {
    const aco_params& p = inst->p;
    cudaStream_t s = inst->stream;
    cudaMemcpyAsync(inst->lbest, lbest, sizeof(int32_t) * (size_t)p.m * p.n, cudaMemcpyDeviceToDevice, s);
    tour_length_kernel<<<(int)fmin((double)p.m, (double)inst->num_sms * 8), 256, 0, s>>>(
        inst->xy, inst->lbest, p.n, p.m, inst->clen, inst->cfix, inst->errflag);
    const long long total = (long long)p.n * p.m;
    neighbours_all_kernel<<<(int)fmin((double)inst->num_sms * 16, (double)ceil_div(total, 256)), 256, 0, s>>>(
        p.n, p.m, p.k, inst->cand, inst->lbest, inst->nb, inst->nbrank);
    aco_status st = check_launch(inst, "set_lbest");
    if (st != ACO_OK) return st;
    GbestArgs G;
    fill_gbest_args(inst, 0, G);
    gbest_q_kernel<false><<<1, 1024, 0, s>>>(G, nullptr);
    st = check_launch(inst, "gbest_q_kernel");
    if (st != ACO_OK) return st;
    return launch_rebuild(inst, 1);
}

// ------------------------------------------------------------------ dense mode (Section 2)
// One warp per row: W = tau^alpha eta^beta, FP32 copy, row flag.
__global__ void dense_weights_kernel(int n, double alpha, const double* __restrict__ tau,
                                     const double* __restrict__ etab_d, double* __restrict__ W64,
                                     float* __restrict__ W32, uint8_t* __restrict__ rowflag,
                                     int* __restrict__ errflag) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        bool flag = false;
        for (int j = lane; j < n; j += 32) {
            const size_t e = (size_t)i * n + j;
            double w = 0.0;
            if (j != i) {
                w = __dmul_rn(powr(tau[e], alpha), etab_d[e]);
                if (!isfinite(w)) atomicOr(errflag, DEVERR_NONFINITE);
            }
            const float w32 = __double2float_rn(w);
            if (j != i) flag |= !(w32 >= FLT_MIN && w32 <= FLT_MAX);
            W64[e] = w;
            W32[e] = w32;
        }
        const unsigned fl = __ballot_sync(FULL, flag);
        if (lane == 0) rowflag[i] = fl ? 1 : 0;
    }
}

aco_status launch_dense_init(aco_instance* inst) {
    const int n = inst->p.n;
    const int blocks = (int)fmin((double)inst->num_sms * 4, (double)ceil_div(n, 8));
    dense_weights_kernel<<<blocks, 256, 0, inst->stream>>>(n, inst->p.alpha, inst->tau, inst->etab_d, inst->W64d,
                                                            inst->W32d, inst->rowflag, inst->errflag);
    if (!inst->initialized) fill_inf_kernel<<<1, 32, 0, inst->stream>>>(inst->gbest, 1);
    return check_launch(inst, "dense_weights_kernel");
}

__global__ void succ_pred_kernel(int n, int m, const int* __restrict__ tours, int* __restrict__ succ,
                                 int* __restrict__ pred) {
    const long long total = (long long)n * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / n), t = (int)(e % n);
        const int* T = tours + (size_t)a * n;
        const int c = T[t];
        succ[(size_t)a * n + c] = T[t + 1 == n ? 0 : t + 1];
        pred[(size_t)a * n + c] = T[t == 0 ? n - 1 : t - 1];
    }
}

// Eq. 2 then Eq. 3-5 for every ordered pair (i, j), i != j; the deposit sum runs over ants in
// index order.
__global__ void dense_tau_kernel(int n, int m, double keep, const int* __restrict__ succ,
                                 const int* __restrict__ pred, const double* __restrict__ clen,
                                 double* __restrict__ tau) {
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double ev = __dmul_rn(keep, tau[e]);
        if (i == j) {  // Eq. 2 applies to every entry; the diagonal receives no deposit
            tau[e] = ev;
            continue;
        }
        double s = 0.0;
        for (int a = 0; a < m; ++a) {
            const size_t o = (size_t)a * n + i;
            if (succ[o] == j || pred[o] == j) s = __dadd_rn(s, __ddiv_rn(1.0, clen[a]));
        }
        tau[e] = __dadd_rn(ev, s);
    }
}

aco_status launch_update_dense(aco_instance* inst) {
    const aco_params& p = inst->p;
    cudaStream_t s = inst->stream;
    const long long nm = (long long)p.n * p.m, nn = (long long)p.n * p.n;
    succ_pred_kernel<<<(int)fmin((double)inst->num_sms * 8, (double)ceil_div(nm, 256)), 256, 0, s>>>(
        p.n, p.m, inst->tours, inst->succ_d, inst->pred_d);
    const double keep = 1.0 - p.rho;
    dense_tau_kernel<<<(int)fmin((double)inst->num_sms * 8, (double)ceil_div(nn, 256)), 256, 0, s>>>(
        p.n, p.m, keep, inst->succ_d, inst->pred_d, inst->clen, inst->tau);
    GbestArgs G;
    fill_gbest_args(inst, 1, G);
    gbest_q_kernel<false><<<1, 1024, 0, s>>>(G, nullptr);
    aco_status st = check_launch(inst, "dense update");
    if (st != ACO_OK) return st;
    const int blocks = (int)fmin((double)inst->num_sms * 4, (double)ceil_div(p.n, 8));
    dense_weights_kernel<<<blocks, 256, 0, s>>>(p.n, p.alpha, inst->tau, inst->etab_d, inst->W64d, inst->W32d,
                                                inst->rowflag, inst->errflag);
    // counts the tours deposited this iteration
    return check_launch(inst, "dense_weights_kernel");
}

// ------------------------------------------------------------------ diagnostic: Eq. 1 probabilities
__global__ void step_probs_kernel(int mode, int n, int k, int city, const uint32_t* __restrict__ bits,
                                  const CandW* __restrict__ candw, const float* __restrict__ W32d,
                                  float* __restrict__ probs, int* __restrict__ exhausted) {
    const int lane = threadIdx.x;
    if (mode == ACO_MODE_LBEST_PARTIAL) {
        bool feas = false;
        float w = 0.f;
        if (lane < k) {
            const CandW e = candw[(size_t)city * k + lane];
            feas = !((bits[e.city >> 5] >> (e.city & 31)) & 1u);
            w = feas ? e.w : 0.f;
        }
        float S = w;
        for (int o = 1; o < 32; o <<= 1) {
            const float v = __shfl_up_sync(FULL, S, o);
            if (lane >= o) S = __fadd_rn(S, v);
        }
        const float T = __shfl_sync(FULL, S, 31);
        const unsigned fm = __ballot_sync(FULL, feas);
        if (lane < k) probs[lane] = fm ? __fdiv_rn(w, T) : 0.f;
        if (lane == 0) *exhausted = fm ? 0 : 1;
    } else {
        float s = 0.f;
        for (int j = lane; j < n; j += 32)
            if (!((bits[j >> 5] >> (j & 31)) & 1u)) s = __fadd_rn(s, W32d[(size_t)city * n + j]);
        for (int o = 16; o; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(FULL, s, o));
        for (int j = lane; j < n; j += 32) {
            const bool v = (bits[j >> 5] >> (j & 31)) & 1u;
            probs[j] = v ? 0.f : __fdiv_rn(W32d[(size_t)city * n + j], s);
        }
        if (lane == 0) *exhausted = 0;
    }
}

aco_status launch_step_probs(aco_instance* inst, int32_t city, const uint32_t* bits, float* probs, int32_t* exhausted) {
    step_probs_kernel<<<1, 32, 0, inst->stream>>>(inst->p.mode, inst->p.n, inst->p.k, city, bits, inst->candw,
                                                  inst->W32d, probs, exhausted);
    return check_launch(inst, "step_probs_kernel");
}

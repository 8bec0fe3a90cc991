// construct.cu -- tour construction launches of a single colony (Section 2 Eq. 1; Section 3.1
// Algorithm 1), the dense Section 2 form, tour lengths and tour output.  The device code of
// the candidate-list construction is in construct_dev.cuh.
#include "construct_dev.cuh"

void fill_lbest_args(const aco_instance* inst, int32_t iteration, LbestArgs& A) {
    const aco_params& p = inst->p;
    A.n = p.n; A.m = p.m; A.k = p.k;
    A.alpha = p.alpha; A.beta = p.beta; A.tau0 = p.tau0; A.f = p.max_mod_frac; A.p_partial = p.p_partial;
    A.seed = p.seed; A.fallback = p.fallback; A.iteration = iteration; A.initialized = inst->initialized ? 1 : 0;
    A.selection = p.selection;
    A.ucap = inst->ucap; A.coord_r = inst->coord_r;
    A.ant0 = inst->ant0;
    A.kx = inst->ext ? inst->kx : 0;
    A.ext = inst->ext;
    A.far = inst->far;
    const bool ia_ok = p.alpha >= 0 && p.alpha <= 16 && floor(p.alpha) == p.alpha;
    const bool ib_ok = p.beta >= 0 && p.beta <= 16 && floor(p.beta) == p.beta;
    A.ia = ia_ok ? (int)p.alpha : -1;
    A.ib = ib_ok ? (int)p.beta : -1;
    A.tau0f = (float)p.tau0;
    A.tau0powf = (float)pow(p.tau0, ia_ok ? (double)(int)p.alpha : p.alpha);
    A.xy = inst->xy; A.xy32 = inst->xy32; A.grid = inst->grid_dev; A.city_cell = inst->city_cell;
    A.cell_start = inst->cell_start; A.cell_city = inst->cell_city; A.cell_xy = inst->cell_xy; A.candw = inst->candw;
    A.W64 = inst->W64; A.lbest = inst->lbest; A.nb = inst->nb; A.nbrank = inst->nbrank;
    A.q = inst->q; A.cfix = inst->cfix;
    A.seg = inst->seg; A.antit = inst->antit; A.accq = inst->accq; A.bel = inst->bel; A.btx = inst->btx; A.btq = inst->btq; A.ghk = inst->ghk; A.ghq = inst->ghq; A.ulist = inst->ulist;
    A.fcnt = inst->fcnt; A.ccnt = inst->ccnt; A.csize = inst->csize; A.ncells = inst->ncells;
    A.ncoarse = inst->ncoarse; A.cgx = inst->cgx; A.cgy = inst->cgy; A.uxy = inst->uxy;
    A.counters = inst->counters; A.errflag = inst->errflag;
    A.async_share = inst->async_share && inst->Qt ? 1 : 0;
    A.Qt = inst->Qt; A.clen = inst->clen; A.cfix_w = inst->cfix; A.lbest_w = inst->lbest; A.nb_w = inst->nb; A.nbrank_w = inst->nbrank;
    A.candw_w = inst->candw; A.W64_w = inst->W64; A.rowflag_w = inst->rowflag; A.etab = inst->etab; A.cand = inst->cand;
}

size_t lbest_args_size() { return sizeof(LbestArgs); }

void fill_lbest_args_bytes(const aco_instance* inst, int32_t iteration, void* out) {
    fill_lbest_args(inst, iteration, *reinterpret_cast<LbestArgs*>(out));
}

// Dynamic shared memory of one ant slot (16-byte multiple) at stage width sk; the batched
// launches stage at STAGE_K.
static size_t construct_smem_per_ant(int n, int k, int sk) {
    return (bits_offset(k, sk) + sizeof(uint32_t) * (size_t)((n + 31) / 32) + 15) & ~(size_t)15;
}
size_t construct_smem_per_ant(int n, int k) { return construct_smem_per_ant(n, k, STAGE_K); }

aco_status launch_construct_lbest(aco_instance* inst, int32_t iteration) {
    LbestArgs A;
    fill_lbest_args(inst, iteration, A);
    const aco_params& p = inst->p;
    // even k above STAGE_K (up to STAGE_K_WIDE) takes the instantiation with the wider stage
    const int sk = single_stage_width(p.k);
    const size_t smem = construct_smem_per_ant(p.n, p.k, sk);
    auto kern = sk == STAGE_K ? construct_lbest_kernel<false, 1, 8> : construct_lbest_kernel<false, 1, 8, STAGE_K_WIDE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_err(inst, ACO_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
    }
    BatchMap none{};
    kern<<<inst->ant1 - inst->ant0, 32, smem, inst->stream>>>(A, none);
    return check_launch(inst, "construct_lbest_kernel");
}

// ------------------------------------------------------------------ dense mode (Section 2)
// One warp per ant; lane l owns cities [l*c, (l+1)*c), c = ceil(n/32).  FP32 screen of the
// index-order wheel, exact FP64 sequential wheel when the screen is inconclusive.
__global__ void __launch_bounds__(32) construct_dense_kernel(int n, unsigned long long seed, int iteration,
                                                             const float* __restrict__ W32,
                                                             const double* __restrict__ W64,
                                                             const uint8_t* __restrict__ rowflag,
                                                             int* __restrict__ tours,
                                                             unsigned long long* __restrict__ counters) {
    extern __shared__ uint32_t bits[];
    const int a = blockIdx.x, lane = threadIdx.x;
    const int W = (n + 31) >> 5;
    const int c = (n + 31) / 32;
    const int b0 = lane * c, b1 = min(n, b0 + c);
    int* T = tours + (size_t)a * n;
    const Draw4 d1 = aco_draw(seed, 0, a, iteration, PURPOSE_START);
    const int start = (int)below(d1.x0, (uint32_t)n);
    for (int w = lane; w < W; w += 32) bits[w] = 0u;
    __syncwarp();
    if (lane == 0) {
        bits[start >> 5] = 1u << (start & 31);
        T[0] = start;
    }
    __syncwarp();
    int cur = start;
    double my_u = 0.0;
    unsigned long long nres = 0;
    const float depth_eps = __fmul_rn((float)(4 * (c + 8)), 0x1.0p-24f);
    for (int t = 0; t < n - 1; ++t) {
        if ((t & 31) == 0) {
            const Draw4 d = aco_draw(seed, (uint32_t)(t + lane), a, iteration, PURPOSE_WHEEL);
            my_u = unit53(d.x0, d.x1);
        }
        const double u = __shfl_sync(FULL, my_u, t & 31);
        const float* row = W32 + (size_t)cur * n;
        float part = 0.f;
        for (int j = b0; j < b1; ++j)
            if (!is_visited(bits, j)) part = __fadd_rn(part, row[j]);
        float S = part;  // inclusive scan of per-lane partial sums
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float v = __shfl_up_sync(FULL, S, o);
            if (lane >= o) S = __fadd_rn(S, v);
        }
        const float T32 = __shfl_sync(FULL, S, 31);
        const float tf = __fmul_rn(__double2float_rn(u), T32);
        const float delta = __fmul_rn(T32, depth_eps);
        int pick = -1;
        bool exact = rowflag[cur] != 0 || !(T32 > 0.f);
        if (!exact) {
            // this lane's chunk holds the pick if its exclusive prefix <= tf < inclusive prefix
            const float excl = __fsub_rn(S, part);  // approximate exclusive prefix for the margin test only
            float run = __shfl_up_sync(FULL, S, 1);
            if (lane == 0) run = 0.f;
            int mine = -1;
            bool unsafe = false;
            if (run <= tf && tf < S) {
                float cum = run, prev = run;
                for (int j = b0; j < b1; ++j) {
                    if (is_visited(bits, j)) continue;
                    prev = cum;
                    cum = __fadd_rn(cum, row[j]);
                    if (cum > tf) {
                        mine = j;
                        unsafe = !(__fsub_rn(tf, prev) > delta && __fsub_rn(cum, tf) > delta);
                        break;
                    }
                }
                if (mine < 0) unsafe = true;
            }
            (void)excl;
            const unsigned have = __ballot_sync(FULL, mine >= 0 || unsafe);
            const unsigned bad = __ballot_sync(FULL, unsafe);
            if (have == 0 || bad != 0) exact = true;
            else pick = __shfl_sync(FULL, mine, __ffs(have) - 1);
        }
        if (exact) {
            ++nres;
            // FP64 sequential wheel in index order over every unvisited city (all lanes alike)
            const double* r64 = W64 + (size_t)cur * n;
            double tot = 0.0;
            int lowest = -1, last = -1;
            for (int j = 0; j < n; ++j)
                if (!is_visited(bits, j)) {
                    if (lowest < 0) lowest = j;
                    tot = __dadd_rn(tot, r64[j]);
                    if (r64[j] > 0.0) last = j;
                }
            if (last < 0) {
                pick = lowest;
            } else {
                const double target = __dmul_rn(u, tot);
                double cum = 0.0;
                pick = last;
                for (int j = 0; j < n; ++j) {
                    if (is_visited(bits, j)) continue;
                    cum = __dadd_rn(cum, r64[j]);
                    if (r64[j] > 0.0 && cum > target) { pick = j; break; }
                }
            }
        }
        if (lane == 0) {
            bits[pick >> 5] |= 1u << (pick & 31);
            T[t + 1] = pick;
        }
        __syncwarp();
        cur = pick;
    }
    if (lane == 0) {
        atomicAdd(&counters[CNT_DECISIONS], (unsigned long long)(n - 1));
        atomicAdd(&counters[CNT_RESOLVES], nres);
        atomicAdd(&counters[CNT_FULL], 1ull);
    }
}

__global__ void tour_length_kernel(const double* __restrict__ xy, const int* __restrict__ tours, int n, int count,
                                   double* __restrict__ out_len, unsigned long long* __restrict__ out_fix,
                                   int* __restrict__ errflag);

aco_status launch_construct_dense(aco_instance* inst, int32_t iteration) {
    const aco_params& p = inst->p;
    const size_t smem = sizeof(uint32_t) * (size_t)((p.n + 31) / 32);
    construct_dense_kernel<<<p.m, 32, smem, inst->stream>>>(p.n, p.seed, iteration, inst->W32d, inst->W64d,
                                                             inst->rowflag, inst->tours, inst->counters);
    aco_status st = check_launch(inst, "construct_dense_kernel");
    if (st != ACO_OK) return st;
    tour_length_kernel<<<p.m, 256, 0, inst->stream>>>(inst->xy, inst->tours, p.n, p.m, inst->clen, inst->cfix,
                                                      inst->errflag);
    return check_launch(inst, "tour_length_kernel");
}

// New tours in the l_best layout (partial: l_best with the rebuilt positions replaced).
__global__ void write_new_tours_kernel(int n, const int* __restrict__ lbest, const int* __restrict__ seg,
                                       const AntIter* __restrict__ antit, int* __restrict__ out,
                                       double* __restrict__ len_out) {
    const int a = blockIdx.x;
    const AntIter it = antit[a];
    const int* L = lbest + (size_t)a * n;
    const int* S = seg + (size_t)a * n;
    int* O = out ? out + (size_t)a * n : nullptr;
    if (O) {
        if (it.s < 0) {
            for (int t = threadIdx.x; t < n; t += blockDim.x) O[t] = S[t];
        } else {
            for (int t = threadIdx.x; t < n; t += blockDim.x) O[t] = L[t];
            __syncthreads();
            for (int t = threadIdx.x; t < it.M; t += blockDim.x) O[(it.s + it.P + t) % n] = S[t];
        }
    }
    if (len_out && threadIdx.x == 0) len_out[a] = it.newlen;
}

aco_status launch_write_new_tours(aco_instance* inst, int32_t* tours_out, double* len_out) {
    const aco_params& p = inst->p;
    if (p.mode == ACO_MODE_DENSE) {
        if (tours_out)
            cudaMemcpyAsync(tours_out, inst->tours, sizeof(int32_t) * (size_t)p.m * p.n, cudaMemcpyDeviceToDevice,
                            inst->stream);
        if (len_out)
            cudaMemcpyAsync(len_out, inst->clen, sizeof(double) * p.m, cudaMemcpyDeviceToDevice, inst->stream);
        return check_launch(inst, "copy new tours");
    }
    write_new_tours_kernel<<<p.m, 256, 0, inst->stream>>>(p.n, inst->lbest, inst->seg, inst->antit, tours_out,
                                                           len_out);
    return check_launch(inst, "write_new_tours_kernel");
}

// construct.cu -- tour construction (Section 2 Eq. 1; Section 3.1 Algorithm 1).
//
// One warp per ant.  The ant's visited set is an n-bit bitset in shared memory.
//
// Decision at city i (candidate-list form): lane r < k loads candidate r of row i as one 8-byte
// (city, FP32 weight) pair and tests its visited bit.  The FP32 weights of unvisited candidates
// go through a warp inclusive scan; the draw u picks the first rank whose prefix exceeds
// u * total.  The FP32 screen is accepted only when u * total is at least 32 * 2^-24 * total
// away from both bounding prefix sums, which is more than the worst-case FP32 error, so the
// pick equals the FP64 sequential wheel's pick.  Otherwise (or when a row's weights are not
// FP32-normal) the decision is re-evaluated exactly: the FP64 weights summed in rank order,
// exactly as Eq. 1 is defined on the host side.
//
// Exhausted list (every candidate visited): argmax over the unvisited cities of
// tau_ij^alpha eta_ij^beta (ties to the lowest index), where tau_ij = tau0 + Q_ij 2^-32 and Q_ij
// sums the weights of the ants whose l_best has edge (i,j) (read from the neighbour table of
// city i).  In a partial rebuild the unvisited cities are the remaining discarded ones; in a
// full construction the unboosted maximum is the nearest unvisited city, found exactly by a
// ring search over the city grid.
#include <float.h>
#include <math.h>

#include "common.cuh"

#define FULL 0xffffffffu

struct LbestArgs {
    int n, m, k;
    double alpha, beta, tau0, f, p_partial;
    unsigned long long seed;
    int fallback, iteration, initialized;
    const double* __restrict__ xy;
    const GridDesc* __restrict__ grid;
    const int* __restrict__ city_cell;
    const int* __restrict__ cell_start;
    const int* __restrict__ cell_city;
    const double* __restrict__ cell_xy;
    const CandW* __restrict__ candw;
    const double* __restrict__ W64;
    const uint8_t* __restrict__ rowflag;
    const int* __restrict__ lbest;
    const int* __restrict__ nb;
    const unsigned long long* __restrict__ q;
    const unsigned long long* __restrict__ cfix;
    int* __restrict__ seg;
    AntIter* __restrict__ antit;
    unsigned long long* __restrict__ accq;
    unsigned long long* __restrict__ counters;
    int* __restrict__ errflag;
};

__device__ __forceinline__ bool is_visited(const uint32_t* bits, int c) { return (bits[c >> 5] >> (c & 31)) & 1u; }

// FP64 sequential wheel over the candidate row (rank order), identical to Eq. 1's definition.
// Returns the picked rank or -1 when no unvisited candidate has a positive weight.
__device__ int wheel_exact_row(const double* __restrict__ w64row, unsigned fmask, int k, double u) {
    double tot = 0.0;
    for (int r = 0; r < k; ++r)
        if ((fmask >> r) & 1u) tot = __dadd_rn(tot, w64row[r]);
    if (!(tot > 0.0)) return -1;
    const double target = __dmul_rn(u, tot);
    double cum = 0.0;
    int last = -1;
    for (int r = 0; r < k; ++r) {
        if (!((fmask >> r) & 1u)) continue;
        const double w = w64row[r];
        cum = __dadd_rn(cum, w);
        if (w > 0.0) {
            last = r;
            if (cum > target) return r;
        }
    }
    return last;
}

__device__ __forceinline__ double weight_of(const LbestArgs& A, double tau0pow, unsigned long long Qb, double d2) {
    const double tp = Qb ? powr(__dadd_rn(A.tau0, __dmul_rn(__ull2double_rn(Qb), 0x1.0p-32)), A.alpha) : tau0pow;
    return __dmul_rn(tp, eta_pow_from_d2(d2, A.beta));
}

// (w desc, city asc) warp argmax; returns the winner's city (uniform) and its weight.
__device__ __forceinline__ int warp_argmax(double& w, int& c, double& d2) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double ow = __shfl_xor_sync(FULL, w, o);
        const int oc = __shfl_xor_sync(FULL, c, o);
        const double od = __shfl_xor_sync(FULL, d2, o);
        if (ow > w || (ow == w && oc < c)) { w = ow; c = oc; d2 = od; }
    }
    return c;
}

// Add the l_best weights of the unvisited neighbours of `cur` into accq (city-indexed, per ant).
// clear = true undoes it (sets the touched entries back to zero).
__device__ void boost_pass(const LbestArgs& A, int a, int cur, const uint32_t* bits, bool clear, int lane) {
    if (!A.initialized) return;
    unsigned long long* acc = A.accq + (size_t)a * A.n;
    const int* row = A.nb + (size_t)cur * A.m * 2;
    for (int b = lane; b < A.m; b += 32) {
        const int2 e = *reinterpret_cast<const int2*>(row + 2 * b);
        if (!is_visited(bits, e.x)) {
            if (clear) acc[e.x] = 0ull; else atomicAdd(&acc[e.x], A.q[b]);
        }
        if (!is_visited(bits, e.y)) {
            if (clear) acc[e.y] = 0ull; else atomicAdd(&acc[e.y], A.q[b]);
        }
    }
    __syncwarp();
}

// Exhausted-list rule.  Returns the chosen city (uniform across the warp).
__device__ int exhausted_choice(const LbestArgs& A, int a, int cur, double u, bool partial, int s, int P, int M,
                                const uint32_t* bits, int lane) {
    const int n = A.n;
    const unsigned long long* acc = A.accq + (size_t)a * n;
    const double qx = A.xy[2 * cur], qy = A.xy[2 * cur + 1];
    const double tau0pow = powr(A.tau0, A.alpha);
    boost_pass(A, a, cur, bits, false, lane);
    int choice = -1;
    if (A.fallback == 0) {
        double bw = -1.0, bd = DBL_MAX;
        int bc = 0x7fffffff;
        if (partial) {
            const int* L = A.lbest + (size_t)a * n;
            for (int t = lane; t < M; t += 32) {
                const int x = L[(s + P + t) % n];
                if (is_visited(bits, x)) continue;
                const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
                const double w = weight_of(A, tau0pow, acc[x], d2);
                if (w > bw || (w == bw && x < bc)) { bw = w; bc = x; bd = d2; }
            }
            choice = warp_argmax(bw, bc, bd);
        } else {
            // boosted neighbours with their true weight
            if (A.initialized) {
                const int* row = A.nb + (size_t)cur * A.m * 2;
                for (int b = lane; b < 2 * A.m; b += 32) {
                    const int x = row[b];
                    if (is_visited(bits, x)) continue;
                    const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
                    const double w = weight_of(A, tau0pow, acc[x], d2);
                    if (w > bw || (w == bw && x < bc)) { bw = w; bc = x; bd = d2; }
                }
            }
            // unboosted maximum = nearest unvisited city: ring search over the grid
            const GridDesc g = *A.grid;
            const int cell = A.city_cell[cur];
            const int cx = cell % g.gx, cy = cell / g.gx;
            double nd = DBL_MAX, nw = -1.0;  // lane-local best of the search (weight at tau0)
            int nc = 0x7fffffff;
            for (int r = 0;; ++r) {
                const int ncell = r == 0 ? 1 : 8 * r;
                for (int c0 = 0; c0 < ncell; c0 += 32) {
                    int pb = 0, pe = 0;
                    if (c0 + lane < ncell) {
                        int x, y;
                        const int idx = c0 + lane;
                        if (r == 0) { x = cx; y = cy; }
                        else if (idx < 2 * r + 1) { x = cx - r + idx; y = cy - r; }
                        else if (idx < 4 * r + 2) { x = cx - r + (idx - 2 * r - 1); y = cy + r; }
                        else if (idx < 6 * r + 1) { x = cx - r; y = cy - r + 1 + (idx - 4 * r - 2); }
                        else { x = cx + r; y = cy - r + 1 + (idx - 6 * r - 1); }
                        if (x >= 0 && y >= 0 && x < g.gx && y < g.gy) {
                            const int c = y * g.gx + x;
                            pb = A.cell_start[c];
                            pe = A.cell_start[c + 1];
                        }
                    }
                    for (; pb < pe; ++pb) {
                        const int x = A.cell_city[pb];
                        if (is_visited(bits, x)) continue;
                        const double d2 = dist2(qx, qy, A.cell_xy[2 * pb], A.cell_xy[2 * pb + 1]);
                        if (!(d2 <= __dmul_rn(nd, 1.0 + 0x1.0p-40))) continue;  // cannot tie the best weight
                        const double w = __dmul_rn(tau0pow, eta_pow_from_d2(d2, A.beta));
                        if (w > nw || (w == nw && x < nc)) {
                            nw = w; nc = x;
                            nd = fmin(nd, d2);
                        }
                    }
                }
                // warp-uniform best distance so far
                double wd = nd;
#pragma unroll
                for (int o = 16; o; o >>= 1) wd = fmin(wd, __shfl_xor_sync(FULL, wd, o));
                const double lb = ring_lower_bound(g, qx, qy, cx, cy, r);
                if (lb < 0.0) break;
                if (wd < DBL_MAX && __dmul_rn(lb, lb) > __dmul_rn(wd, 1.0 + 0x1.0p-40)) break;
            }
            double dd = nd;
            warp_argmax(nw, nc, dd);
            // combine: the nearest city's tau0 weight vs the boosted neighbours' true weights
            double cbw = bw, cbd = bd;
            int cbc = bc;
            warp_argmax(cbw, cbc, cbd);
            if (nw > cbw || (nw == cbw && nc < cbc)) { cbw = nw; cbc = nc; }
            choice = cbc;
        }
    } else {
        // Eq. 1 wheel over every unvisited city in index order (FP64, sequential: all lanes
        // evaluate the same sums; the words of the bitset are screened in parallel).
        const int W = (n + 31) >> 5;
        double tot = 0.0;
        int lowest = -1, last = -1;
        for (int pass = 0; pass < 2 && choice < 0; ++pass) {
            const double target = __dmul_rn(u, tot);
            double cum = 0.0;
            for (int wb = 0; wb < W && choice < 0; wb += 32) {
                const int wi = wb + lane;
                uint32_t free_bits = 0;
                if (wi < W) {
                    free_bits = ~bits[wi];
                    if (wi == W - 1 && (n & 31)) free_bits &= (1u << (n & 31)) - 1u;
                }
                unsigned nz = __ballot_sync(FULL, free_bits != 0);
                while (nz && choice < 0) {
                    const int src = __ffs(nz) - 1;
                    nz &= nz - 1;
                    uint32_t fb = __shfl_sync(FULL, free_bits, src);
                    const int base = (wb + src) << 5;
                    while (fb) {
                        const int x = base + __ffs(fb) - 1;
                        fb &= fb - 1;
                        const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
                        const double w = weight_of(A, tau0pow, acc[x], d2);
                        if (pass == 0) {
                            if (lowest < 0) lowest = x;
                            tot = __dadd_rn(tot, w);
                            if (w > 0.0) last = x;
                        } else {
                            cum = __dadd_rn(cum, w);
                            if (w > 0.0 && cum > target) { choice = x; break; }
                        }
                    }
                }
            }
            if (pass == 0 && last < 0) choice = lowest;
        }
        if (choice < 0) choice = last;
    }
    boost_pass(A, a, cur, bits, true, lane);
    if (choice < 0) {
        if (lane == 0) atomicOr(A.errflag, DEVERR_NO_CHOICE);
        choice = cur;
    }
    return choice;
}

// Exact length of the edges (from[e], to[e]) of a path given by a generator.
__device__ __forceinline__ u128 edge_fix(const double* __restrict__ xy, int i, int j) {
    return len_to_fix(__dsqrt_rn(dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1])));
}

__global__ void __launch_bounds__(32) construct_lbest_kernel(LbestArgs A) {
    extern __shared__ uint32_t bits[];
    const int a = blockIdx.x, lane = threadIdx.x;
    const int n = A.n, k = A.k;
    const int W = (n + 31) >> 5;
    bool partial = false;
    if (A.initialized) {
        partial = true;
        if (A.p_partial < 1.0) {
            const Draw4 d = aco_draw(A.seed, 0, a, A.iteration, PURPOSE_COIN);
            partial = unit53(d.x0, d.x1) < A.p_partial;
        }
    }
    const int* L = A.lbest + (size_t)a * n;
    int* seg = A.seg + (size_t)a * n;
    int cur, steps, s = -1, P = 0, M, start;
    if (partial) {
        const Draw4 d1 = aco_draw(A.seed, 0, a, A.iteration, PURPOSE_START);
        s = (int)below(d1.x0, (uint32_t)n);
        long long fm = (long long)floor(__dmul_rn(A.f, (double)n));
        long long pmin = (long long)n - fm;
        if (pmin < 1) pmin = 1;
        if (pmin > n - 1) pmin = n - 1;
        const Draw4 d2 = aco_draw(A.seed, 0, a, A.iteration, PURPOSE_KEEP);
        P = (int)pmin + (int)below(d2.x0, (uint32_t)(n - pmin));
        M = n - P;
        for (int w = lane; w < W; w += 32) bits[w] = 0xFFFFFFFFu;
        __syncwarp();
        for (int t = lane; t < M; t += 32) {
            const int c = L[(s + P + t) % n];
            atomicAnd(&bits[c >> 5], ~(1u << (c & 31)));
        }
        cur = L[(s + P - 1) % n];
        start = L[s];
        steps = M;
    } else {
        const Draw4 d1 = aco_draw(A.seed, 0, a, A.iteration, PURPOSE_START);
        start = (int)below(d1.x0, (uint32_t)n);
        for (int w = lane; w < W; w += 32) bits[w] = 0u;
        __syncwarp();
        if (lane == 0) {
            bits[start >> 5] = 1u << (start & 31);
            seg[0] = start;
        }
        cur = start;
        steps = n - 1;
        M = n - 1;
    }
    __syncwarp();
    const int outbase = partial ? 0 : 1;
    double my_u = 0.0;
    unsigned long long nfall = 0, nres = 0;
    for (int t = 0; t < steps; ++t) {
        if ((t & 31) == 0) {
            const Draw4 d = aco_draw(A.seed, (uint32_t)(t + lane), a, A.iteration, PURPOSE_WHEEL);
            my_u = unit53(d.x0, d.x1);
        }
        const double u = __shfl_sync(FULL, my_u, t & 31);
        int c = -1;
        float w = 0.f;
        bool feas = false;
        if (lane < k) {
            const CandW e = A.candw[(size_t)cur * k + lane];
            c = e.city;
            w = e.w;
            feas = !is_visited(bits, c);
        }
        const unsigned fmask = __ballot_sync(FULL, feas);
        int pick = -1;
        if (fmask) {
            bool exact = A.rowflag[cur] != 0;
            if (!exact) {
                float S = feas ? w : 0.f;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float v = __shfl_up_sync(FULL, S, o);
                    if (lane >= o) S = __fadd_rn(S, v);
                }
                const float T = __shfl_sync(FULL, S, 31);
                const float tf = __fmul_rn(__double2float_rn(u), T);
                const unsigned gt = __ballot_sync(FULL, feas && S > tf);
                const float lo_all = __shfl_up_sync(FULL, S, 1);
                exact = true;
                if (gt) {
                    const int r = __ffs(gt) - 1;
                    const float hi = __shfl_sync(FULL, S, r);
                    const float lo = r > 0 ? __shfl_sync(FULL, lo_all, r) : 0.f;
                    const float delta = __fmul_rn(T, 0x1.0p-19f);
                    if (__fsub_rn(tf, lo) > delta && __fsub_rn(hi, tf) > delta) {
                        pick = r;
                        exact = false;
                    }
                }
            }
            if (exact) {
                ++nres;
                pick = wheel_exact_row(A.W64 + (size_t)cur * k, fmask, k, u);
            }
        }
        int j;
        if (pick >= 0) {
            j = __shfl_sync(FULL, c, pick);
        } else {
            ++nfall;
            j = exhausted_choice(A, a, cur, u, partial, s, P, M, bits, lane);
        }
        if (lane == 0) {
            bits[j >> 5] |= 1u << (j & 31);
            seg[outbase + t] = j;
        }
        __syncwarp();
        cur = j;
    }
    __syncwarp();
    // exact length of the new tour
    u128 acc_new = 0, acc_old = 0;
    if (partial) {
        const int e = L[(s + P - 1) % n];
        for (int ei = lane; ei <= M; ei += 32) {
            const int fo = ei == 0 ? e : L[(s + P + ei - 1) % n];
            const int to_ = ei == M ? start : L[(s + P + ei) % n];
            const int fn = ei == 0 ? e : seg[ei - 1];
            const int tn = ei == M ? start : seg[ei];
            acc_old += edge_fix(A.xy, fo, to_);
            acc_new += edge_fix(A.xy, fn, tn);
        }
    } else {
        for (int ei = lane; ei < n; ei += 32) acc_new += edge_fix(A.xy, seg[ei], seg[ei + 1 == n ? 0 : ei + 1]);
    }
    acc_new = warp_sum_u128(acc_new);
    acc_old = warp_sum_u128(acc_old);
    if (lane == 0) {
        u128 total = acc_new;
        if (partial) {
            const u128 old = (((u128)A.cfix[2 * a + 1]) << 64) | A.cfix[2 * a];
            total = old - acc_old + acc_new;
        }
        AntIter it;
        it.s = s; it.P = P; it.M = M; it.start = start;
        it.newlen = fix_to_len(total);
        it.fix_lo = (unsigned long long)total;
        it.fix_hi = (unsigned long long)(total >> 64);
        A.antit[a] = it;
        atomicAdd(&A.counters[CNT_DECISIONS], (unsigned long long)steps);
        atomicAdd(&A.counters[CNT_FALLBACKS], nfall);
        atomicAdd(&A.counters[CNT_RESOLVES], nres);
        atomicAdd(&A.counters[partial ? CNT_PARTIAL : CNT_FULL], 1ull);
    }
}

aco_status launch_construct_lbest(aco_instance* inst, int32_t iteration) {
    LbestArgs A;
    const aco_params& p = inst->p;
    A.n = p.n; A.m = p.m; A.k = p.k;
    A.alpha = p.alpha; A.beta = p.beta; A.tau0 = p.tau0; A.f = p.max_mod_frac; A.p_partial = p.p_partial;
    A.seed = p.seed; A.fallback = p.fallback; A.iteration = iteration; A.initialized = inst->initialized ? 1 : 0;
    A.xy = inst->xy; A.grid = inst->grid_dev; A.city_cell = inst->city_cell; A.cell_start = inst->cell_start;
    A.cell_city = inst->cell_city; A.cell_xy = inst->cell_xy; A.candw = inst->candw; A.W64 = inst->W64;
    A.rowflag = inst->rowflag; A.lbest = inst->lbest; A.nb = inst->nb; A.q = inst->q; A.cfix = inst->cfix;
    A.seg = inst->seg; A.antit = inst->antit; A.accq = inst->accq; A.counters = inst->counters;
    A.errflag = inst->errflag;
    const size_t smem = sizeof(uint32_t) * (size_t)((p.n + 31) / 32);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(construct_lbest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return set_err(inst, ACO_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
    }
    construct_lbest_kernel<<<p.m, 32, smem, inst->stream>>>(A);
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

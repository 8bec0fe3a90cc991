// construct_dev.cuh -- device code of the tour construction, shared by the single-colony
// launches (construct.cu) and the batched ones (construct_batch.cu).
//
// Tour construction (Section 2 Eq. 1; Section 3.1 Algorithm 1).
//
// One warp per ant.  The ant's visited set is an n-bit bitset in shared memory.
//
// Decision at city i (candidate-list form): lane r < k loads candidate r of row i as one 8-byte
// (city, FP32 weight) pair and tests its visited bit.  The FP32 weights of unvisited candidates
// go through a warp inclusive scan; the draw u picks the first rank whose prefix exceeds
// u * total.  The FP32 screen is accepted only when u * total is at least 32 * 2^-24 * total
// away from both bounding prefix sums, which is more than the worst-case FP32 error, so the
// pick equals the FP64 sequential wheel's pick.  Otherwise (or when a row's weights are not
// FP32-normal, marked by negative screen weights) the decision is re-evaluated exactly: the
// FP64 weights summed in rank order, exactly as Eq. 1 is defined.  While the current decision
// is computed, the rows of every unvisited candidate are copied (cp.async) into a shared-memory
// staging buffer, so the next decision reads its row from shared memory (even k <= 16, and in a
// single colony even k <= 24 with a wider buffer; other rows are read from global memory).
//
// Exhausted list (every candidate visited): argmax over the unvisited cities of
// tau_ij^alpha eta_ij^beta (ties to the lowest index), where tau_ij = tau0 + Q_ij 2^-32 and Q_ij
// sums the weights of the ants whose l_best has edge (i,j) (read from the neighbour table of
// city i).  For cities with Q_ij = 0 the weight only falls with d_ij, so:
//   * partial rebuild: the remaining discarded cities sit in a compacted per-ant list with FP32
//     coordinates; an FP32 distance screen with a rigorous error bound keeps the near-nearest
//     cities, and only those get the exact FP64 weight;
//   * full construction: the nearest unvisited city is found exactly by a ring search over the
//     city grid;
// and the few unvisited l_best neighbours of city i get their exact boosted weight.
//
// Independent Roulette (selection = 1, Section 3): each unvisited candidate's exact weight times
// its own Philox uniform, the largest product wins.  Asynchronous sharing (opt-in, Section 3):
// an improved partial rebuild commits its l_best and moves its pheromone at the end of its own
// construction, inside the launch (async_commit).
#pragma once

#include <float.h>
#include <math.h>

#include "common.cuh"
#include "update_dev.cuh"

#define FULL 0xffffffffu

struct LbestArgs {
    int n, m, k;
    double alpha, beta, tau0, f, p_partial;
    unsigned long long seed;
    int fallback, iteration, initialized;
    int selection;  // 0 = Eq. 1 wheel, 1 = Independent Roulette
    int ucap;       // capacity of the per-ant remaining-city list
    int ant0;       // first ant of the launch (a rank's share of a sharded colony)
    int kx;         // extended list length (0 = none)
    const int* __restrict__ ext;                 // n*kx nearest cities (candidates first)
    const int* __restrict__ far;                 // n*ACO_KF nearest cities, or null
    float coord_r;  // max |coordinate| (FP32 screen error bound)
    int ia, ib;     // alpha, beta as small integers (0..16) for the FP32 screen, else -1
    float tau0f, tau0powf;  // tau0 and tau0^alpha in FP32
    const double* __restrict__ xy;
    const float2* __restrict__ xy32;
    const GridDesc* __restrict__ grid;
    const int* __restrict__ city_cell;
    const int* __restrict__ cell_start;
    const int* __restrict__ cell_city;
    const double* __restrict__ cell_xy;
    const CandW* __restrict__ candw;
    const double* __restrict__ W64;
    const int* __restrict__ lbest;
    const int* __restrict__ nb;
    const uint8_t* __restrict__ nbrank;
    const unsigned long long* __restrict__ q;
    const unsigned long long* __restrict__ cfix;
    int* __restrict__ seg;
    AntIter* __restrict__ antit;
    unsigned long long* __restrict__ accq;
    unsigned short* __restrict__ bel;
    int* __restrict__ btx;
    unsigned long long* __restrict__ btq;
    int* __restrict__ fcnt;                // per-ant unvisited cities per grid cell (full constructions)
    int* __restrict__ ccnt;                // and per coarse block of ACO_CBLK x ACO_CBLK cells
    const int* __restrict__ csize;         // cities per coarse block
    int ncells, ncoarse, cgx, cgy;
    int* __restrict__ ghk;                 // per-ant global hash of boosted cities (2m slots, -1 = empty)
    unsigned long long* __restrict__ ghq;  // and their summed weights (0 when empty)
    int* __restrict__ ulist;
    float2* __restrict__ uxy;
    unsigned long long* __restrict__ counters;
    int* __restrict__ errflag;
    // asynchronous sharing: an improved partial rebuild commits inside the launch (these tables
    // are then written while other ants read them)
    int async_share;
    unsigned long long* Qt;  // n*k integer pheromone of the candidate edges
    double* clen;
    unsigned long long* cfix_w;
    int* lbest_w;
    int* nb_w;
    uint8_t* nbrank_w;
    CandW* candw_w;
    double* W64_w;
    uint8_t* rowflag_w;
    const double* etab;
    const int* cand;
};

// Batched launches: ant slot -> (instance, ant); per-instance descriptors; device iteration.
struct BatchMap {
    const LbestArgs* args;
    const int2* slot;
    const int* iteration;
    int slots;
    int smem_per_ant;
};

__device__ __forceinline__ bool is_visited(const uint32_t* bits, int c) { return (bits[c >> 5] >> (c & 31)) & 1u; }

// FP64 sequential wheel over the candidate row (rank order), identical to Eq. 1's definition.
// Returns the picked rank or -1 when no unvisited candidate has a positive weight.
static __device__ int wheel_exact_row(const double* __restrict__ w64row, unsigned fmask, int k, double u) {
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

__device__ __forceinline__ bool better(double w, int c, double bw, int bc) { return w > bw || (w == bw && c < bc); }

// (w desc, city asc) warp argmax; every lane ends with the winner.
__device__ __forceinline__ void warp_argmax(double& w, int& c) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double ow = __shfl_xor_sync(FULL, w, o);
        const int oc = __shfl_xor_sync(FULL, c, o);
        if (better(ow, oc, w, c)) { w = ow; c = oc; }
    }
}

// ---------------------------------------------------------------- FP32-screened exhausted step
// FP32 estimate of tau^alpha eta^beta from an FP32 tau and squared distance (integer exponents).
__device__ __forceinline__ float weight_f32(float tauf, float d2f, int ia, int ib) {
    float tp = 1.f;
    for (int i = 0; i < ia; ++i) tp = __fmul_rn(tp, tauf);
    float e = 1.f;
    if ((ib & 1) == 0) {
        const float inv = __frcp_rn(d2f);
        for (int i = 0; i < (ib >> 1); ++i) e = __fmul_rn(e, inv);
    } else {
        const float inv = rsqrtf(d2f);
        for (int i = 0; i < ib; ++i) e = __fmul_rn(e, inv);
    }
    return __fmul_rn(tp, e);
}

__device__ __forceinline__ void top2_push(float w, int x, float& w1, int& x1, float& w2) {
    if (w > w1 || (w == w1 && x < x1)) {
        w2 = w1;
        w1 = w;
        x1 = x;
    } else if (w > w2) {
        w2 = w;
    }
}

// Unvisited l_best neighbours of `cur` that are not candidates.  Only entries whose candidate
// rank is 0xFF (the neighbour is not a candidate) can be unvisited at an exhausted step.  Phase A
// lists those entries of the 2-byte rank row of `cur` (the row is usually requested into
// registers before the remaining-city scan, so its latency overlaps that scan); phase B gathers
// their neighbour ids together and lists the unvisited ones with the weight of the ant each entry
// belongs to.  The lists are per-ant global scratch of capacity 2m (every entry fits) and are
// filled with warp-aggregated offsets.  The integer pheromone of a city is the sum of the weights
// of its entries; equal cities are merged in a hash (shared memory for short lists).
#define BHASH 128     // slots of the per-ant hash of boosted cities (distinct unvisited neighbours)
#define BHASH_MAX 96  // more distinct cities than this: the listed path decides

struct BoostSmem {
    unsigned long long hq[BHASH];  // summed integer pheromone of the city in each slot
    int hkey[BHASH];               // city, -1 = empty (kept empty between exhausted steps)
    int hcount;                    // distinct cities inserted
};

__device__ __forceinline__ unsigned bhash_slot(int x) { return ((unsigned)x * 2654435761u) >> 25; }

// Empties the hash (four slots per lane).
__device__ __forceinline__ void bhash_clear(BoostSmem& sh, int lane) {
    __syncwarp();
#pragma unroll
    for (int s4 = 0; s4 < BHASH / 32; ++s4) {
        sh.hkey[lane + 32 * s4] = -1;
        sh.hq[lane + 32 * s4] = 0ull;
    }
    if (lane == 0) sh.hcount = 0;
    __syncwarp();
}

// For 2m <= 2048 (m a multiple of 8) each lane holds 64 bytes of the rank row.
struct RankRow {
    uint4 v[4];
};

__device__ __forceinline__ void load_rank_row(const LbestArgs& A, int cur, int lane, RankRow& rr) {
    const uint8_t* rrow = A.nbrank + (size_t)cur * A.m * 2;
    const int E = 2 * A.m;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int b0 = h * 512 + lane * 16;
        rr.v[h] = b0 < E ? __ldcs(reinterpret_cast<const uint4*>(rrow + b0)) : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Offsets for a warp-wide append: lane contributes `cnt` items; returns where they go and adds
// the warp total to `total`.
__device__ __forceinline__ int warp_offsets(int cnt, int& total, int lane) {
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += v;
    }
    const int base = total + inc - cnt;
    total += __shfl_sync(FULL, inc, 31);
    return base;
}

// Phase A over one 2048-byte block of the rank row held in registers.
__device__ __forceinline__ void list_nonc(unsigned short* el, int& ne, const RankRow& rr, int base, int lane) {
    uint32_t msk[16];
    int c = 0;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint32_t wv[4] = {rr.v[h].x, rr.v[h].y, rr.v[h].z, rr.v[h].w};
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            msk[h * 4 + g] = __vcmpeq4(wv[g], 0xFFFFFFFFu);  // 0xFF in every byte equal to 0xFF
            c += __popc(msk[h * 4 + g]) >> 3;
        }
    }
    int off = warp_offsets(c, ne, lane);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int b0 = base + h * 512 + lane * 16;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint32_t mm = msk[h * 4 + g];
            while (mm) {
                const int byte = (__ffs(mm) - 1) >> 3;
                mm &= ~(0xFFu << (8 * byte));
                el[off++] = (unsigned short)(b0 + 4 * g + byte);
            }
        }
    }
}

// Lists the unvisited non-candidate l_best neighbours of `cur` with their ant's weight in the
// ant's scratch (tx, tq); returns their number.
static __device__ int collect_boosted(const LbestArgs& A, int a, int cur, const uint32_t* bits, int lane, const RankRow* pre) {
    const size_t cap = (size_t)2 * A.m;
    unsigned short* el = A.bel + (size_t)a * cap;
    int* tx = A.btx + (size_t)a * cap;
    unsigned long long* tq = A.btq + (size_t)a * cap;
    const uint8_t* rrow = A.nbrank + (size_t)cur * A.m * 2;
    const int* irow = A.nb + (size_t)cur * A.m * 2;
    const int E = 2 * A.m;  // entries: (ant, side) -> index 2*ant + side
    int ne = 0;
    if (pre) {
        list_nonc(el, ne, *pre, 0, lane);
    } else if ((A.m & 7) == 0) {
        for (int base = 0; base < E; base += 2048) {
            RankRow rr;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int b0 = base + h * 512 + lane * 16;
                rr.v[h] = b0 < E ? __ldcs(reinterpret_cast<const uint4*>(rrow + b0)) : make_uint4(0u, 0u, 0u, 0u);
            }
            list_nonc(el, ne, rr, base, lane);
        }
    } else {
        for (int e0 = 0; e0 < E; e0 += 32) {
            const int e = e0 + lane;
            const bool f = e < E && rrow[e] == 0xFF;
            int off = warp_offsets(f ? 1 : 0, ne, lane);
            if (f) el[off] = (unsigned short)e;
        }
    }
    __syncwarp();
    int nt = 0;
    for (int t0 = 0; t0 < ne; t0 += 128) {
        int e4[4], x4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int idx = t0 + 32 * h + lane;
            e4[h] = idx < ne ? (int)el[idx] : -1;
            x4[h] = e4[h] >= 0 ? __ldcs(irow + e4[h]) : -1;
        }
        int c = 0;
        bool un[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            un[h] = x4[h] >= 0 && !is_visited(bits, x4[h]);
            c += un[h] ? 1 : 0;
        }
        int off = warp_offsets(c, nt, lane);
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if (un[h]) {
                tx[off] = x4[h];
                tq[off] = A.q[e4[h] >> 1];
                ++off;
            }
    }
    __syncwarp();
    return nt;
}

// Argmax over the listed cities of their weight: FP32 estimates into a top-2 (fast path) or exact
// FP64 weights into (bw, bc).  Duplicated cities are evaluated once, with the sum of the weights
// of all their entries.
template <bool EXACT>
__device__ void boosted_eval(const LbestArgs& A, int a, int cur, int nt, BoostSmem& sh, int lane, double qx,
                             double qy, double tau0pow, double& bw, int& bc, float& w1, int& x1, float& w2,
                             float& dmin) {
    const size_t cap = (size_t)2 * A.m;
    const int* gx = A.btx + (size_t)a * cap;
    const unsigned long long* gq = A.btq + (size_t)a * cap;
    if (nt <= 32) {  // one entry per lane; equal cities grouped by a match
        const int x = lane < nt ? gx[lane] : -1 - lane;
        const unsigned long long qq = lane < nt ? gq[lane] : 0ull;
        const unsigned grp = __match_any_sync(FULL, x);
        const int gsize = __popc(grp);
        const int maxg = __reduce_max_sync(FULL, (unsigned)gsize);
        unsigned long long Qx = 0;
        unsigned g = grp;
        for (int it = 0; it < maxg; ++it) {
            const int src = g ? __ffs(g) - 1 : lane;
            g &= g - 1;
            const unsigned long long v = __shfl_sync(FULL, qq, src);
            if (it < gsize) Qx += v;
        }
        if (lane < nt && lane == __ffs(grp) - 1) {
            if (EXACT) {
                const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
                const double w = weight_of(A, tau0pow, Qx, d2);
                if (better(w, x, bw, bc)) { bw = w; bc = x; }
            } else {
                const float2 q32 = A.xy32[cur];
                const float2 px = A.xy32[x];
                const float dx = __fsub_rn(px.x, q32.x), dy = __fsub_rn(px.y, q32.y);
                const float d2f = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                const float tauf = __fadd_rn(A.tau0f, __fmul_rn(__ull2float_rn(Qx), 0x1.0p-32f));
                dmin = fminf(dmin, d2f);
                top2_push(weight_f32(tauf, d2f, A.ia, A.ib), x, w1, x1, w2);
            }
        }
        __syncwarp();
        return;
    }
    // equal cities merged by their summed weights in a hash: the shared-memory one (empty
    // between uses) for up to BHASH_MAX entries, else the ant's global one (capacity 2m, which
    // every list fits); each slot is evaluated once and emptied
    const bool small = nt <= BHASH_MAX;
    int* keys = small ? sh.hkey : A.ghk + (size_t)a * cap;
    unsigned long long* qs = small ? sh.hq : A.ghq + (size_t)a * cap;
    const int hcap = small ? BHASH : (int)cap;
    for (int t = lane; t < nt; t += 32) {
        const int x = gx[t];
        const unsigned long long q = gq[t];
        unsigned h = small ? bhash_slot(x) : (unsigned)(((unsigned long long)((unsigned)x * 2654435761u) * hcap) >> 32);
        for (int pr = 0; pr < hcap; ++pr) {
            const int old = atomicCAS(&keys[h], -1, x);
            if (old == -1 || old == x) {
                atomicAdd(&qs[h], q);
                break;
            }
            h = h + 1 == (unsigned)hcap ? 0u : h + 1;
        }
    }
    __syncwarp();
    const float2 q32 = A.xy32[cur];
    for (int s0 = 0; s0 < hcap; s0 += 32) {
        const int slot = s0 + lane;
        const int x = slot < hcap ? *reinterpret_cast<volatile int*>(&keys[slot]) : -1;
        if (x < 0) continue;
        const unsigned long long Qx = *reinterpret_cast<volatile unsigned long long*>(&qs[slot]);
        keys[slot] = -1;
        qs[slot] = 0ull;
        if (EXACT) {
            const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
            const double w = weight_of(A, tau0pow, Qx, d2);
            if (better(w, x, bw, bc)) { bw = w; bc = x; }
        } else {
            const float2 px = A.xy32[x];
            const float dx = __fsub_rn(px.x, q32.x), dy = __fsub_rn(px.y, q32.y);
            const float d2f = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            const float tauf = __fadd_rn(A.tau0f, __fmul_rn(__ull2float_rn(Qx), 0x1.0p-32f));
            dmin = fminf(dmin, d2f);
            top2_push(weight_f32(tauf, d2f, A.ia, A.ib), x, w1, x1, w2);
        }
    }
    if (small && lane == 0) sh.hcount = 0;
    __syncwarp();
}

// Error bound of the FP32 squared distance d2f against the exact FP64 one, for coordinates of
// magnitude <= R rounded to FP32: |d2f - d2| <= 2^-21 (2 R sqrt(d2) + 2 d2) + 2^-44 R^2 (generous).
__device__ __forceinline__ float d2_bound(float d2, float R) {
    return __fadd_rn(__fmul_rn(0x1.0p-21f, __fadd_rn(__fmul_rn(2.f * R, __fsqrt_rn(d2)), __fmul_rn(2.f, d2))),
                     __fmul_rn(0x1.0p-44f, __fmul_rn(R, R)));
}

// Partial rebuild: argmax over the remaining discarded cities (compacted list, FP32 screen).
// Pass 1 (eight loads per lane in flight) compacts the list in place (visited cities drop out)
// and keeps, per lane, the two smallest screened distances and where the smallest now sits.
// Only cities whose screened distance is within the error bound of the minimum can carry the
// largest weight; they get the exact FP64 weight.  A second pass over the list is needed only
// when some lane holds two such cities.
static __device__ void remaining_argmax(const LbestArgs& A, int a, int cur, const uint32_t* bits, int& ucount, int lane,
                                 double qx, double qy, double tau0pow, double& bw, int& bc) {
    int* ul = A.ulist + (size_t)a * A.ucap;
    float2* uxy = A.uxy + (size_t)a * A.ucap;
    const float2 q32 = A.xy32[cur];
    float m1 = FLT_MAX, m2 = FLT_MAX;
    int i1 = -1;
    int cnt = 0;
    for (int base = 0; base < ucount; base += 256) {
        int id[8];
        float2 p[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int idx = base + 32 * h + lane;
            id[h] = -1;
            p[h] = make_float2(0.f, 0.f);
            if (idx < ucount) {
                id[h] = ul[idx];
                p[h] = uxy[idx];
            }
        }
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const bool keep = id[h] >= 0 && !is_visited(bits, id[h]);
            const unsigned b = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = cnt + __popc(b & ((1u << lane) - 1u));
                ul[pos] = id[h];
                uxy[pos] = p[h];
                const float dx = __fsub_rn(p[h].x, q32.x), dy = __fsub_rn(p[h].y, q32.y);
                const float d2f = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (d2f < m1) { m2 = m1; m1 = d2f; i1 = pos; }
                else if (d2f < m2) { m2 = d2f; }
            }
            cnt += __popc(b);
        }
    }
    ucount = cnt;
    float best = m1;
#pragma unroll
    for (int o = 16; o; o >>= 1) best = fminf(best, __shfl_xor_sync(FULL, best, o));
    __syncwarp();
    if (cnt == 0) return;
    const float R = A.coord_r;
    const float hi = __fadd_rn(__fmul_rn(best, 1.0f + 0x1.0p-18f), __fmul_rn(2.f, d2_bound(best, R)));
    const float thr = __fadd_rn(hi, __fmul_rn(2.f, d2_bound(hi, R)));
    if (__any_sync(FULL, m2 <= thr)) {
        for (int idx = lane; idx < cnt; idx += 32) {
            const float2 p = uxy[idx];
            const float dx = __fsub_rn(p.x, q32.x), dy = __fsub_rn(p.y, q32.y);
            const float d2f = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (d2f <= thr) {
                const int x = ul[idx];
                const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
                const double w = __dmul_rn(tau0pow, eta_pow_from_d2(d2, A.beta));
                if (better(w, x, bw, bc)) { bw = w; bc = x; }
            }
        }
    } else if (m1 <= thr) {
        const int x = ul[i1];
        const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
        const double w = __dmul_rn(tau0pow, eta_pow_from_d2(d2, A.beta));
        if (better(w, x, bw, bc)) { bw = w; bc = x; }
    }
}

// Cell (x, y) of the `idx`-th cell on the Chebyshev ring r around (cx, cy) of a gx x gy grid;
// false outside the grid.
__device__ __forceinline__ bool ring_xy(int cx, int cy, int r, int idx, int gx, int gy, int& x, int& y) {
    if (r == 0) { x = cx; y = cy; }
    else if (idx < 2 * r + 1) { x = cx - r + idx; y = cy - r; }
    else if (idx < 4 * r + 2) { x = cx - r + (idx - 2 * r - 1); y = cy + r; }
    else if (idx < 6 * r + 1) { x = cx - r; y = cy - r + 1 + (idx - 4 * r - 2); }
    else { x = cx + r; y = cy - r + 1 + (idx - 6 * r - 1); }
    return x >= 0 && y >= 0 && x < gx && y < gy;
}

// Lower bound on the distance from (qx, qy) to any point outside the grid cells [x0, x1] x [y0, y1];
// -1 when the block covers the whole grid.
__device__ __forceinline__ double block_lower_bound(const GridDesc& g, double qx, double qy, int x0, int x1, int y0,
                                                    int y1) {
    double lb = 1e300;
    bool open = false;
    if (x0 > 0) { lb = fmin(lb, qx - (g.xmin + (double)x0 * g.h)); open = true; }
    if (x1 < g.gx - 1) { lb = fmin(lb, (g.xmin + (double)(x1 + 1) * g.h) - qx); open = true; }
    if (y0 > 0) { lb = fmin(lb, qy - (g.ymin + (double)y0 * g.h)); open = true; }
    if (y1 < g.gy - 1) { lb = fmin(lb, (g.ymin + (double)(y1 + 1) * g.h) - qy); open = true; }
    if (!open) return -1.0;
    lb -= g.margin;
    return lb < 0.0 ? 0.0 : lb;
}

// Unvisited cities of grid cell c at tau0: exact weights of the cities that can reach the lane's
// nearest (nd: the lane's smallest squared distance so far).
__device__ __forceinline__ void scan_cell(const LbestArgs& A, int c, const uint32_t* bits, double qx, double qy,
                                          double tau0pow, double& nd, double& bw, int& bc) {
    for (int pb = A.cell_start[c], pe = A.cell_start[c + 1]; pb < pe; ++pb) {
        const int x = A.cell_city[pb];
        if (is_visited(bits, x)) continue;
        const double d2 = dist2(qx, qy, A.cell_xy[2 * pb], A.cell_xy[2 * pb + 1]);
        if (!(d2 <= __dmul_rn(nd, 1.0 + 0x1.0p-40))) continue;  // cannot reach the best weight
        const double w = __dmul_rn(tau0pow, eta_pow_from_d2(d2, A.beta));
        if (better(w, x, bw, bc)) { bw = w; bc = x; }
        nd = fmin(nd, d2);
    }
}

__device__ __forceinline__ bool ring_done(const GridDesc& g, double nd, double lb) {
    double wd = nd;
#pragma unroll
    for (int o = 16; o; o >>= 1) wd = fmin(wd, __shfl_xor_sync(FULL, wd, o));
    if (lb < 0.0) return true;
    return wd < DBL_MAX && __dmul_rn(lb, lb) > __dmul_rn(wd, 1.0 + 0x1.0p-40);
}

// Full construction: nearest unvisited city (weight at tau0), every contender's weight exact.  The
// ant's per-cell and per-block counts of unvisited cities let the search skip empty cells: rings
// of cells 0..3 around the current city first, then rings of coarse blocks, each stopping as
// soon as nothing outside the searched square can be nearer than the nearest found.
static __device__ void nearest_unvisited_exact(const LbestArgs& A, int a, int cur, const uint32_t* bits, int lane, double qx,
                                        double qy, double tau0pow, double& bw, int& bc) {
    const GridDesc g = *A.grid;
    const int* fc = A.fcnt + (size_t)a * A.ncells;
    const int* cc = A.ccnt + (size_t)a * A.ncoarse;
    const int cell = A.city_cell[cur];
    const int cx = cell % g.gx, cy = cell / g.gx;
    double nd = DBL_MAX;
    for (int r = 0; r <= 3; ++r) {
        const int ncell = r == 0 ? 1 : 8 * r;
        for (int c0 = 0; c0 < ncell; c0 += 32) {
            int x, y;
            if (c0 + lane < ncell && ring_xy(cx, cy, r, c0 + lane, g.gx, g.gy, x, y)) {
                const int c = y * g.gx + x;
                if (__ldcg(fc + c) > 0) scan_cell(A, c, bits, qx, qy, tau0pow, nd, bw, bc);
            }
        }
        if (ring_done(g, nd, ring_lower_bound(g, qx, qy, cx, cy, r))) return;
    }
    const int CX = cx / ACO_CBLK, CY = cy / ACO_CBLK;
    for (int rho = 0;; ++rho) {
        const int nc = rho == 0 ? 1 : 8 * rho;
        for (int c0 = 0; c0 < nc; c0 += 32) {
            int X, Y, C = -1;
            if (c0 + lane < nc && ring_xy(CX, CY, rho, c0 + lane, A.cgx, A.cgy, X, Y)) C = Y * A.cgx + X;
            unsigned ne = __ballot_sync(FULL, C >= 0 && __ldcg(cc + C) > 0);
            while (ne) {  // the warp scans each non-empty block: its cells, two per lane
                const int src = __ffs(ne) - 1;
                ne &= ne - 1;
                const int Cs = __shfl_sync(FULL, C, src);
                const int X0 = (Cs % A.cgx) * ACO_CBLK, Y0 = (Cs / A.cgx) * ACO_CBLK;
                for (int f = lane; f < ACO_CBLK * ACO_CBLK; f += 32) {
                    const int fx = X0 + f % ACO_CBLK, fy = Y0 + f / ACO_CBLK;
                    if (fx < g.gx && fy < g.gy && __ldcg(fc + fy * g.gx + fx) > 0)
                        scan_cell(A, fy * g.gx + fx, bits, qx, qy, tau0pow, nd, bw, bc);
                }
            }
        }
        const double lb = block_lower_bound(g, qx, qy, (CX - rho) * ACO_CBLK, (CX + rho + 1) * ACO_CBLK - 1,
                                            (CY - rho) * ACO_CBLK, (CY + rho + 1) * ACO_CBLK - 1);
        if (ring_done(g, nd, lb)) return;
    }
}

// Per lane: the two smallest squared distances seen and the city of the smallest (lowest index
// among equals).
struct Near2 {
    double d1, d2;
    int c1;
};

__device__ __forceinline__ void near_push(Near2& s, double d, int x) {
    if (x == s.c1) return;  // the same city seen again (block rings overlap the cell rings)
    if (d < s.d1 || (d == s.d1 && x < s.c1)) {
        s.d2 = s.d1;
        s.d1 = d;
        s.c1 = x;
    } else if (d < s.d2) {
        s.d2 = d;
    }
}

// The unvisited cities of the lane's cell (c >= 0 with unvisited cities, else -1), spread over
// the warp: an inclusive scan of the cell sizes, then every lane takes one city slot at a time
// and finds its cell by a binary search over the scan (shuffles).
__device__ __forceinline__ void scan_cells_flat(const LbestArgs& A, int c, const uint32_t* bits, double qx, double qy,
                                                int lane, Near2& s) {
    int pb = 0, nc = 0;
    if (c >= 0) {
        pb = A.cell_start[c];
        nc = A.cell_start[c + 1] - pb;
    }
    int incl = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int T = __shfl_sync(FULL, incl, 31);
    for (int s0 = 0; s0 < T; s0 += 32) {
        const int slot = s0 + lane;
        int lo = 0, hi = 31;
#pragma unroll
        for (int it = 0; it < 5; ++it) {
            const int mid = (lo + hi) >> 1;
            const int v = __shfl_sync(FULL, incl, mid);
            if (v > slot) hi = mid;
            else lo = mid + 1;
        }
        const int excl = __shfl_sync(FULL, incl - nc, lo);
        const int base = __shfl_sync(FULL, pb, lo);
        if (slot < T) {
            const int p = base + (slot - excl);
            const int x = A.cell_city[p];
            if (!is_visited(bits, x)) near_push(s, dist2(qx, qy, A.cell_xy[2 * p], A.cell_xy[2 * p + 1]), x);
        }
    }
}

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Full construction: nearest unvisited city (weight at tau0) by squared distances alone.  The
// weight only falls as the distance grows, so the city of smallest d^2 wins unless another city
// lies within 2^-40 of it (a possible tie of the rounded weights): then the exact search decides.
static __device__ void nearest_unvisited(const LbestArgs& A, int a, int cur, const uint32_t* bits, int lane, double qx,
                                  double qy, double tau0pow, double& bw, int& bc) {
    const GridDesc g = *A.grid;
    const int* fc = A.fcnt + (size_t)a * A.ncells;
    const int* cc = A.ccnt + (size_t)a * A.ncoarse;
    const int cell = A.city_cell[cur];
    const int cx = cell % g.gx, cy = cell / g.gx;
    Near2 s{DBL_MAX, DBL_MAX, 0x7fffffff};
    bool done = false;
    for (int r = 0; r <= 3 && !done; ++r) {
        const int ncell = r == 0 ? 1 : 8 * r;
        for (int c0 = 0; c0 < ncell; c0 += 32) {
            int x, y, c = -1;
            if (c0 + lane < ncell && ring_xy(cx, cy, r, c0 + lane, g.gx, g.gy, x, y) && __ldcg(fc + y * g.gx + x) > 0)
                c = y * g.gx + x;
            scan_cells_flat(A, c, bits, qx, qy, lane, s);
        }
        const double lb = ring_lower_bound(g, qx, qy, cx, cy, r);
        const double wd = warp_min_d(s.d1);
        done = lb < 0.0 || (wd < DBL_MAX && __dmul_rn(lb, lb) > __dmul_rn(wd, 1.0 + 0x1.0p-40));
    }
    const int CX = cx / ACO_CBLK, CY = cy / ACO_CBLK;
    for (int rho = 0; !done; ++rho) {
        const int nc = rho == 0 ? 1 : 8 * rho;
        for (int c0 = 0; c0 < nc; c0 += 32) {
            int X, Y, C = -1;
            if (c0 + lane < nc && ring_xy(CX, CY, rho, c0 + lane, A.cgx, A.cgy, X, Y)) C = Y * A.cgx + X;
            unsigned ne = __ballot_sync(FULL, C >= 0 && __ldcg(cc + C) > 0);
            while (ne) {  // each non-empty block: its cells, two per lane
                const int src = __ffs(ne) - 1;
                ne &= ne - 1;
                const int Cs = __shfl_sync(FULL, C, src);
                const int X0 = (Cs % A.cgx) * ACO_CBLK, Y0 = (Cs / A.cgx) * ACO_CBLK;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int f = lane + 32 * h;
                    const int fx = X0 + f % ACO_CBLK, fy = Y0 + f / ACO_CBLK;
                    int c = -1;
                    if (fx < g.gx && fy < g.gy && __ldcg(fc + fy * g.gx + fx) > 0) c = fy * g.gx + fx;
                    scan_cells_flat(A, c, bits, qx, qy, lane, s);
                }
            }
        }
        const double lb = block_lower_bound(g, qx, qy, (CX - rho) * ACO_CBLK, (CX + rho + 1) * ACO_CBLK - 1,
                                            (CY - rho) * ACO_CBLK, (CY + rho + 1) * ACO_CBLK - 1);
        const double wd = warp_min_d(s.d1);
        done = lb < 0.0 || (wd < DBL_MAX && __dmul_rn(lb, lb) > __dmul_rn(wd, 1.0 + 0x1.0p-40));
    }
    const double D = warp_min_d(s.d1);
    const double thr = __dmul_rn(D, 1.0 + 0x1.0p-40);
    if (__any_sync(FULL, s.d2 <= thr)) {  // two cities within the tie margin on one lane
        nearest_unvisited_exact(A, a, cur, bits, lane, qx, qy, tau0pow, bw, bc);
        return;
    }
    if (s.d1 <= thr) {
        const double w = __dmul_rn(tau0pow, eta_pow_from_d2(s.d1, A.beta));
        if (better(w, s.c1, bw, bc)) { bw = w; bc = s.c1; }
    }
}

// The counts of a full construction: every cell's city count, then each chosen city removed
// (deferred: the cities chosen since the last exhausted step, read back from the tour).
static __device__ void counts_init(const LbestArgs& A, int a, int lane) {
    int* fc = A.fcnt + (size_t)a * A.ncells;
    int* cc = A.ccnt + (size_t)a * A.ncoarse;
    for (int c = lane; c < A.ncells; c += 32) fc[c] = A.cell_start[c + 1] - A.cell_start[c];
    for (int c = lane; c < A.ncoarse; c += 32) cc[c] = A.csize[c];
}

static __device__ void counts_remove(const LbestArgs& A, int a, const int* seg, int from, int to, int lane) {
    const GridDesc& g = *A.grid;
    int* fc = A.fcnt + (size_t)a * A.ncells;
    int* cc = A.ccnt + (size_t)a * A.ncoarse;
    for (int p = from + lane; p < to; p += 32) {
        const int c = A.city_cell[seg[p]];
        atomicSub(fc + c, 1);
        atomicSub(cc + ((c / g.gx) / ACO_CBLK) * A.cgx + (c % g.gx) / ACO_CBLK, 1);
    }
    __syncwarp();
}

// Eq. 1 wheel over every unvisited city in index order (fallback = 1), FP64, sequential order.
static __device__ int wheel_all_unvisited(const LbestArgs& A, int a, int cur, double u, const uint32_t* bits, int lane,
                                   double qx, double qy, double tau0pow) {
    const int n = A.n;
    unsigned long long* acc = A.accq + (size_t)a * n;
    // integer pheromone of the unvisited l_best neighbours into acc (cleared below)
    const int* row = A.nb + (size_t)cur * A.m * 2;
    if (A.initialized)
        for (int b = lane; b < 2 * A.m; b += 32) {
            const int x = row[b];
            if (!is_visited(bits, x)) atomicAdd(&acc[x], A.q[b >> 1]);
        }
    __syncwarp();
    const int W = (n + 31) >> 5;
    double tot = 0.0;
    int lowest = -1, last = -1, choice = -1;
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
                    const double w = weight_of(A, tau0pow, __ldcg(&acc[x]), d2);
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
    __syncwarp();
    if (A.initialized)
        for (int b = lane; b < 2 * A.m; b += 32) {
            const int x = row[b];
            if (!is_visited(bits, x)) acc[x] = 0ull;
        }
    __syncwarp();
    return choice;
}

// The extended list of `cur` holds its kx nearest cities, key (d^2, index), candidates first.  At
// an exhausted step every candidate is visited, so the first unvisited entry of rank >= k is the
// nearest unvisited city c1, and every other unvisited city lies at least as far as the next
// unvisited entry c2 -- or, when there is none, as the last entry (every city outside the list
// is at least that far).  Both helpers give up (false / -1) when the list holds no unvisited city
// or only its last entry; the caller then takes the full path.

// Full construction before any pheromone (initial tours, tau = tau0 everywhere): the nearest
// unvisited city wins unless the runner-up lies within 2^-40 of it (a possible tie of the rounded
// weights), compared exactly in FP64.
static_assert(ACO_KF == 128, "the far list is read as four slots of 32 lanes");

static __device__ int ext_full_choice(const LbestArgs& A, int cur, const uint32_t* bits, int lane) {
    __syncwarp();  // the previous city's visited bit is visible
    const int kx = A.kx, k = A.k;
    int c1, c2;
    if (A.far) {
        // the 128 nearest, entry p in lane p % 32 of slot p / 32: the first two unvisited
        // entries of rank >= k in list order (the last entry bounds every unlisted city)
        int e[ACO_KF / 32], r1 = -1, r2 = -1;
#pragma unroll
        for (int s = 0; s < ACO_KF / 32; ++s) e[s] = __ldg(A.far + (size_t)cur * ACO_KF + 32 * s + lane);
#pragma unroll
        for (int s = 0; s < ACO_KF / 32; ++s) {
            unsigned u = __ballot_sync(FULL, 32 * s + lane >= k && !is_visited(bits, e[s]));
            while (u && r2 < 0) {
                const int p = 32 * s + __ffs(u) - 1;
                u &= u - 1u;
                if (r1 < 0) r1 = p;
                else r2 = p;
            }
        }
        if (r1 < 0 || (r2 < 0 && r1 == ACO_KF - 1)) return -1;
        if (r2 < 0) r2 = ACO_KF - 1;
        const int s1 = r1 >> 5, s2 = r2 >> 5;
        const int v1 = s1 == 0 ? e[0] : s1 == 1 ? e[1] : s1 == 2 ? e[2] : e[3];
        const int v2 = s2 == 0 ? e[0] : s2 == 1 ? e[1] : s2 == 2 ? e[2] : e[3];
        c1 = __shfl_sync(FULL, v1, r1 & 31);
        c2 = __shfl_sync(FULL, v2, r2 & 31);
    } else {
        const int e = lane < kx ? __ldg(A.ext + (size_t)cur * kx + lane) : -1;
        const unsigned um = __ballot_sync(FULL, lane >= k && lane < kx && !is_visited(bits, e));
        const unsigned more = um & (um - 1u);
        const int r1 = __ffs(um) - 1;
        if (um == 0u || (!more && r1 == kx - 1)) return -1;
        const int r2 = more ? __ffs(more) - 1 : kx - 1;
        c1 = __shfl_sync(FULL, e, r1);
        c2 = __shfl_sync(FULL, e, r2);
    }
    const double qx = A.xy[2 * cur], qy = A.xy[2 * cur + 1];
    const double d1 = dist2(qx, qy, A.xy[2 * c1], A.xy[2 * c1 + 1]);
    const double d2 = dist2(qx, qy, A.xy[2 * c2], A.xy[2 * c2 + 1]);
    return d2 > __dmul_rn(d1, 1.0 + 0x1.0p-40) ? c1 : -1;
}

// Partial rebuild: the two nearest remaining cities at tau0 as the remaining-city scan gives them
// (FP32 squared distances; lane 0 holds d1 with its city y1 and the runner-up bound d2s, every
// other lane FLT_MAX), from the extended list instead of a scan.
__device__ __forceinline__ bool ext_nearest(const LbestArgs& A, int cur, const uint32_t* bits, int lane, float2 q32,
                                            float& d1, float& d2s, int& y1) {
    const int kx = A.kx, k = A.k;
    const int e = lane < kx ? __ldg(A.ext + (size_t)cur * kx + lane) : -1;
    const unsigned um = __ballot_sync(FULL, lane >= k && lane < kx && !is_visited(bits, e));
    const unsigned more = um & (um - 1u);
    const int r1 = __ffs(um) - 1;
    if (um == 0u || (!more && r1 == kx - 1)) return false;
    const int r2 = more ? __ffs(more) - 1 : kx - 1;
    const int c1 = __shfl_sync(FULL, e, r1), c2 = __shfl_sync(FULL, e, r2);
    d1 = FLT_MAX;
    d2s = FLT_MAX;
    y1 = 0x7fffffff;
    if (lane == 0) {
        const float2 p1 = A.xy32[c1], p2 = A.xy32[c2];
        const float ax = __fsub_rn(p1.x, q32.x), ay = __fsub_rn(p1.y, q32.y);
        const float bx = __fsub_rn(p2.x, q32.x), by = __fsub_rn(p2.y, q32.y);
        d1 = __fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay));
        d2s = __fadd_rn(__fmul_rn(bx, bx), __fmul_rn(by, by));
        y1 = c1;
    }
    return true;
}

// Exhausted step of a partial rebuild with every weight first estimated in FP32, each with a
// relative error bound E (FP32 coordinates and distances, reciprocal, powers, tau).  If the best
// estimate beats the second best by more than the bounds allow, it is the exact FP64 argmax and
// is returned without any FP64 work; otherwise -1 (the caller then evaluates exactly).  The
// remaining list is compacted on the way.
static __device__ int partial_choice_fast(const LbestArgs& A, int a, int cur, const uint32_t* bits, int& ucount, BoostSmem& sh,
                                   int lane, const RankRow* pre, unsigned long long& nfast) {
    int* ul = A.ulist + (size_t)a * A.ucap;
    float2* uxy = A.uxy + (size_t)a * A.ucap;
    const float2 q32 = A.xy32[cur];
    float w1 = -1.f, w2 = -1.f, dmin = FLT_MAX;
    int x1 = 0x7fffffff;
    // unboosted cities: the weight only falls with the distance, so keep the two nearest
    float d1 = FLT_MAX, d2s = FLT_MAX;
    int y1 = 0x7fffffff;
    int cnt = ucount;
    if (A.kx && ext_nearest(A, cur, bits, lane, q32, d1, d2s, y1)) {
        ++nfast;  // the list is compacted by a later scan
    } else {
    cnt = 0;
    for (int base = 0; base < ucount; base += 256) {
        int id[8];
        float2 p[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int idx = base + 32 * h + lane;
            id[h] = -1;
            p[h] = make_float2(0.f, 0.f);
            if (idx < ucount) {
                id[h] = ul[idx];
                p[h] = uxy[idx];
            }
        }
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const bool keep = id[h] >= 0 && !is_visited(bits, id[h]);
            const unsigned b = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = cnt + __popc(b & ((1u << lane) - 1u));
                if (pos != base + 32 * h + lane) {
                    ul[pos] = id[h];
                    uxy[pos] = p[h];
                }
                const float dx = __fsub_rn(p[h].x, q32.x), dy = __fsub_rn(p[h].y, q32.y);
                const float d2f = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (d2f < d1 || (d2f == d1 && id[h] < y1)) {
                    d2s = d1;
                    d1 = d2f;
                    y1 = id[h];
                } else if (d2f < d2s) {
                    d2s = d2f;
                }
            }
            cnt += __popc(b);
        }
    }
    }
    if (d1 < FLT_MAX) {
        dmin = d1;
        top2_push(__fmul_rn(A.tau0powf, weight_f32(1.f, d1, 0, A.ib)), y1, w1, x1, w2);
        if (d2s < FLT_MAX) w2 = fmaxf(w2, __fmul_rn(A.tau0powf, weight_f32(1.f, d2s, 0, A.ib)));
    }
    ucount = cnt;
    __syncwarp();
    if (A.initialized) {
        const int nt = collect_boosted(A, a, cur, bits, lane, pre);
        double bwd = -1.0;
        int bcd = 0x7fffffff;
        boosted_eval<false>(A, a, cur, nt, sh, lane, 0.0, 0.0, 0.0, bwd, bcd, w1, x1, w2, dmin);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ow1 = __shfl_xor_sync(FULL, w1, o), ow2 = __shfl_xor_sync(FULL, w2, o);
        const int ox1 = __shfl_xor_sync(FULL, x1, o);
        dmin = fminf(dmin, __shfl_xor_sync(FULL, dmin, o));
        if (ow1 > w1 || (ow1 == w1 && ox1 < x1)) {
            w2 = fmaxf(w1, ow2);
            w1 = ow1;
            x1 = ox1;
        } else {
            w2 = fmaxf(w2, ow1);
        }
    }
    if (!(dmin >= 1e-30f) || !(w1 > 0.f) || !(w1 <= FLT_MAX)) return -1;
    // relative error bound of every estimate (largest at the smallest distance)
    const float eps_d = __fdiv_rn(__fmul_rn(1.1f, d2_bound(dmin, A.coord_r)), dmin);
    const float E = __fmul_rn(1.25f, __fadd_rn(__fmul_rn(0.5f * (float)A.ib + 0.5f, eps_d),
                                               __fmul_rn((float)(A.ib + A.ia + 4), 0x1.0p-22f)));
    if (!(E < 0.25f)) return -1;
    if (__fmul_rn(w1, 1.f - E) > __fmul_rn(w2, 1.f + E)) return x1;
    return -1;
}

// Loads of one round (256 entries, 8 per lane) of the remaining-city list.
__device__ __forceinline__ void load_remaining(const int* ul, const float2* uxy, int base, int ucount, int lane,
                                               int (&id)[8], float2 (&p)[8]) {
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const int idx = base + 32 * h + lane;
        id[h] = -1;
        p[h] = make_float2(0.f, 0.f);
        if (idx < ucount) {
            id[h] = ul[idx];
            p[h] = uxy[idx];
        }
    }
}

// One pass over the remaining-city list (round 0 already loaded into id/p; the next round's loads
// in flight while a round is processed): visited cities drop out (the list is compacted in
// place) and the warp keeps, per lane, the two nearest cities at tau0 (d1 with city y1, d2s).
__device__ __forceinline__ void scan_remaining(int* ul, float2* uxy, int& ucount, int lane, float2 q32,
                                               const uint32_t* bits, int (&id)[8], float2 (&p)[8], float& d1,
                                               float& d2s, int& y1) {
    d1 = FLT_MAX;
    d2s = FLT_MAX;
    y1 = 0x7fffffff;
    int cnt = 0;
    const unsigned ltm = (1u << lane) - 1u;
    for (int base = 0; base < ucount; base += 256) {
        int idn[8];
        float2 pn[8];
        load_remaining(ul, uxy, base + 256, ucount, lane, idn, pn);
        bool kp[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) kp[h] = id[h] >= 0 && !is_visited(bits, id[h]);
        unsigned bl[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) bl[h] = __ballot_sync(FULL, kp[h]);
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int pos = cnt + __popc(bl[h] & ltm);
            cnt += __popc(bl[h]);
            if (kp[h] && pos != base + 32 * h + lane) {
                ul[pos] = id[h];
                uxy[pos] = p[h];
            }
        }
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const float dx = __fsub_rn(p[h].x, q32.x), dy = __fsub_rn(p[h].y, q32.y);
            const float v = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            // equal distances need no order here: the runner-up then equals the nearest and the
            // exact path (ties to the lowest index) decides
            const bool lt1 = kp[h] && v < d1;
            const bool lt2 = kp[h] && v < d2s;
            d2s = lt1 ? d1 : (lt2 ? v : d2s);
            y1 = lt1 ? id[h] : y1;
            d1 = lt1 ? v : d1;
        }
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            id[h] = idn[h];
            p[h] = pn[h];
        }
    }
    ucount = cnt;
}

// Warp top-2 of the lanes' FP32 weight estimates, by reductions over the bit patterns of
// non-negative floats (their order): the best estimate (ties: the lower city; one lane is taken as
// its holder) and the best of all the other estimates; the winner is returned when it beats the
// runner-up by more than the estimates' relative error bound E (FP32 coordinates and distances,
// reciprocal, powers, tau; largest at the smallest squared distance dmin), else -1.
__device__ __forceinline__ int top2_decide(const LbestArgs& A, int lane, float w1, int x1, float w2, float dmin) {
    const unsigned wb = __float_as_uint(fmaxf(w1, 0.f));
    const unsigned wmax = __reduce_max_sync(FULL, wb);
    const unsigned xmin = __reduce_min_sync(FULL, wb == wmax ? (unsigned)x1 : 0xFFFFFFFFu);
    const unsigned win = __ballot_sync(FULL, wb == wmax && (unsigned)x1 == xmin);
    const float rest = lane == __ffs(win) - 1 ? w2 : fmaxf(w1, w2);
    w2 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(fmaxf(rest, 0.f))));
    w1 = __uint_as_float(wmax);
    x1 = (int)xmin;
    dmin = __uint_as_float(__reduce_min_sync(FULL, __float_as_uint(dmin)));
    if (!(dmin >= 1e-30f) || !(w1 > 0.f) || !(w1 <= FLT_MAX)) return -1;
    const float eps_d = __fdiv_rn(__fmul_rn(1.1f, d2_bound(dmin, A.coord_r)), dmin);
    const float E = __fmul_rn(1.25f, __fadd_rn(__fmul_rn(0.5f * (float)A.ib + 0.5f, eps_d),
                                               __fmul_rn((float)(A.ib + A.ia + 4), 0x1.0p-22f)));
    if (!(E < 0.25f)) return -1;
    return __fmul_rn(w1, 1.f - E) > __fmul_rn(w2, 1.f + E) ? x1 : -1;
}

// FP32 estimates of the hashed cities (slots lane + 32 s, coordinates in hp) with their tau and of
// the nearest remaining cities at tau0; the best estimate is returned when it wins by more than
// the error bounds allow (the hash is emptied), else -1 (the hash is kept for hashed_exact).
__device__ __forceinline__ int hashed_decision(const LbestArgs& A, BoostSmem& sh, int lane, float2 q32,
                                               const int (&hx)[BHASH / 32], const float2 (&hp)[BHASH / 32],
                                               float d1, float d2s, int y1) {
    float w1 = -1.f, w2 = -1.f, dmin = FLT_MAX;
    int x1 = 0x7fffffff;
    // 3. the hashed cities with their tau
#pragma unroll
    for (int s4 = 0; s4 < BHASH / 32; ++s4) {
        const int x = hx[s4];
        if (x < 0) continue;
        const float dx = __fsub_rn(hp[s4].x, q32.x), dy = __fsub_rn(hp[s4].y, q32.y);
        const float d2f = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        const unsigned long long Q = sh.hq[lane + 32 * s4];
        const float tauf = __fadd_rn(A.tau0f, __fmul_rn(__ull2float_rn(Q), 0x1.0p-32f));
        dmin = fminf(dmin, d2f);
        top2_push(weight_f32(tauf, d2f, A.ia, A.ib), x, w1, x1, w2);
    }
    if (d1 < FLT_MAX) {
        dmin = fminf(dmin, d1);
        top2_push(__fmul_rn(A.tau0powf, weight_f32(1.f, d1, 0, A.ib)), y1, w1, x1, w2);
        if (d2s < FLT_MAX) w2 = fmaxf(w2, __fmul_rn(A.tau0powf, weight_f32(1.f, d2s, 0, A.ib)));
    }
    const int win = top2_decide(A, lane, w1, x1, w2, dmin);
    if (win >= 0) bhash_clear(sh, lane);
    return win;
}

// Exhausted step of a partial rebuild, FP32-screened as partial_choice_fast, with the boosted
// cities aggregated in a shared-memory hash:
//  1. each lane finds the non-candidate entries among its bytes of the rank row of `cur` (held
//     in registers), gathers their neighbour ids and ant weights eight per round, and inserts the
//     unvisited cities into the hash with the summed weights of their entries (shared-memory
//     atomics on integers: the order of the insertions does not matter);
//  2. the coordinates of the hashed cities are requested, and one pass over the remaining-city
//     list (the next round's loads in flight) compacts it and keeps, per lane, the two nearest
//     cities at tau0; a hashed city also counts there at tau0, which only underestimates it;
//  3. the hashed cities are estimated with their tau.
// Returns the city when the best estimate wins by more than the error bounds allow (the hash is
// empty again); -1 when the estimates are too close (the hash is kept for hashed_exact); -2 when
// the hash overflowed (emptied).
static __device__ int partial_choice_hashed(const LbestArgs& A, int a, int cur, const uint32_t* bits, int& ucount,
                                     BoostSmem& sh, int lane, const RankRow& rr, unsigned long long& nfast) {
    int* ul = A.ulist + (size_t)a * A.ucap;
    float2* uxy = A.uxy + (size_t)a * A.ucap;
    const int* irow = A.nb + (size_t)cur * A.m * 2;
    int id[8];
    float2 p[8];
    const float2 q32 = A.xy32[cur];
    float d1, d2s;
    int y1;
    // the nearest remaining cities from the extended list, else by a scan of the remaining list
    const bool from_ext = A.kx && ext_nearest(A, cur, bits, lane, q32, d1, d2s, y1);
    if (!from_ext) load_remaining(ul, uxy, 0, ucount, lane, id, p);  // in flight while the hash is built
    // 1a. entry e of the rank row sits in lane (e % 512) / 16 at byte (e / 512) * 16 + e % 16;
    //     bit 4 * word + byte of bm marks a non-candidate entry
    unsigned long long bm = 0;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint32_t wv[4] = {rr.v[h].x, rr.v[h].y, rr.v[h].z, rr.v[h].w};
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint32_t m8 = __vcmpeq4(wv[g], 0xFFFFFFFFu) & 0x80808080u;
            bm |= (unsigned long long)((m8 * 0x00204081u) >> 28) << (4 * (h * 4 + g));
        }
    }
    // 1b. each lane gathers its own non-candidate entries, eight per round, and inserts them
    bool over = false;
    while (__any_sync(FULL, bm != 0ull)) {
        int x8[8];
        unsigned long long q8[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            int e = -1;
            if (bm) {
                const int b = __ffsll((long long)bm) - 1;
                bm &= bm - 1;
                const int word = b >> 2;
                e = (word >> 2) * 512 + lane * 16 + 4 * (word & 3) + (b & 3);
            }
            x8[h] = e >= 0 ? __ldcs(irow + e) : -1;
            q8[h] = e >= 0 ? __ldg(A.q + (e >> 1)) : 0ull;
        }
        bool unv[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) unv[h] = x8[h] >= 0 && !is_visited(bits, x8[h]);
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            if (!unv[h]) continue;
            unsigned hs = bhash_slot(x8[h]);
            bool done = false;
            for (int pr = 0; pr < BHASH && !done; ++pr) {
                // a slot that already holds the city takes a plain add; an empty one is claimed
                int old = *reinterpret_cast<volatile int*>(&sh.hkey[hs]);
                if (old == -1) old = atomicCAS(&sh.hkey[hs], -1, x8[h]);
                if (old == -1 || old == x8[h]) {
                    atomicAdd(&sh.hq[hs], q8[h]);
                    done = true;
                }
                hs = (hs + 1) & (BHASH - 1);
            }
            if (!done) over = true;
        }
    }
    __syncwarp();
    // 2. coordinates of the hashed cities (four slots per lane) requested before the scan; the
    //    number of distinct cities decides the overflow
    int hx[BHASH / 32];
    float2 hp[BHASH / 32];
    int distinct = 0;
#pragma unroll
    for (int s4 = 0; s4 < BHASH / 32; ++s4) {
        hx[s4] = sh.hkey[lane + 32 * s4];
        hp[s4] = hx[s4] >= 0 ? A.xy32[hx[s4]] : make_float2(0.f, 0.f);
        distinct += __popc(__ballot_sync(FULL, hx[s4] >= 0));
    }
    const bool overflow = __any_sync(FULL, over) || distinct > BHASH_MAX;
    if (overflow) {
        bhash_clear(sh, lane);
        return -2;
    }
    if (from_ext) ++nfast;
    else scan_remaining(ul, uxy, ucount, lane, q32, bits, id, p, d1, d2s, y1);
    return hashed_decision(A, sh, lane, q32, hx, hp, d1, d2s, y1);
}

// Exact FP64 weights of the hashed cities (after partial_choice_hashed returned -1), then the
// hash is emptied.
static __device__ void hashed_exact(const LbestArgs& A, BoostSmem& sh, int lane, double qx, double qy, double tau0pow,
                             double& bw, int& bc) {
#pragma unroll
    for (int s4 = 0; s4 < BHASH / 32; ++s4) {
        const int x = sh.hkey[lane + 32 * s4];
        if (x < 0) continue;
        const double d2 = dist2(qx, qy, A.xy[2 * x], A.xy[2 * x + 1]);
        const double w = weight_of(A, tau0pow, sh.hq[lane + 32 * s4], d2);
        if (better(w, x, bw, bc)) { bw = w; bc = x; }
    }
    bhash_clear(sh, lane);
}

// Exhausted-list rule.  Returns the chosen city (uniform across the warp).
// staged: the candidate rows are staged in shared memory (even k up to the launch's stage width);
// the hashed step serves those colonies, partial_choice_fast the others (measured faster for the
// batched colonies with k = 20, whose rows are not staged).
static __device__ int exhausted_choice(const LbestArgs& A, int a, int cur, double u, bool partial, bool staged,
                                int& ucount, const uint32_t* bits, BoostSmem& sh, int lane, unsigned long long& nfast) {
    __syncwarp();  // the previous city's visited bit (set at the top of the step) is visible
    int choice = -1;
    bool decided = false;
    if (A.fallback == 0) {
        double bw = -1.0;
        int bc = 0x7fffffff;
        // the rank row of `cur` is requested first; its latency overlaps the scan below
        RankRow rr;
        const bool pre = A.initialized && (A.m & 7) == 0 && A.m <= 1024;
        if (pre) load_rank_row(A, cur, lane, rr);
        bool hashed_tie = false;
        if (partial && A.ia >= 0 && A.ib >= 0 && pre && staged) {
            const int fast = partial_choice_hashed(A, a, cur, bits, ucount, sh, lane, rr, nfast);
            if (fast >= 0) return fast;
            hashed_tie = fast == -1;
        } else if (partial && A.ia >= 0 && A.ib >= 0) {
            const int fast = partial_choice_fast(A, a, cur, bits, ucount, sh, lane, pre ? &rr : nullptr, nfast);
            if (fast >= 0) return fast;
        }
        // the FP64 paths (the FP32 screens above settle almost every step without them, so the
        // coordinates and the FP64 power are taken only here)
        const double qx = A.xy[2 * cur], qy = A.xy[2 * cur + 1];
        const double tau0pow = powr(A.tau0, A.alpha);
        if (hashed_tie) {  // near tie: exact weights of the near-nearest and of the hashed cities
            remaining_argmax(A, a, cur, bits, ucount, lane, qx, qy, tau0pow, bw, bc);
            hashed_exact(A, sh, lane, qx, qy, tau0pow, bw, bc);
            decided = true;
        }
        if (!decided) {
            if (partial) remaining_argmax(A, a, cur, bits, ucount, lane, qx, qy, tau0pow, bw, bc);
            else nearest_unvisited(A, a, cur, bits, lane, qx, qy, tau0pow, bw, bc);
            if (A.initialized) {
                const int nt = collect_boosted(A, a, cur, bits, lane, pre ? &rr : nullptr);
                float f1 = -1.f, f2 = -1.f, fd = FLT_MAX;
                int fx = 0;
                boosted_eval<true>(A, a, cur, nt, sh, lane, qx, qy, tau0pow, bw, bc, f1, fx, f2, fd);
            }
        }
        warp_argmax(bw, bc);
        choice = bc;
        if (bw < 0.0) choice = -1;
    } else {
        const double qx = A.xy[2 * cur], qy = A.xy[2 * cur + 1];
        choice = wheel_all_unvisited(A, a, cur, u, bits, lane, qx, qy, powr(A.tau0, A.alpha));
    }
    if (choice < 0 || choice >= A.n) {
        if (lane == 0) atomicOr(A.errflag, DEVERR_NO_CHOICE);
        choice = cur;
    }
    return choice;
}

// Exact length of one edge on the 2^-96 grid.
__device__ __forceinline__ u128 edge_fix(const double* __restrict__ xy, int i, int j) {
    return len_to_fix(__dsqrt_rn(dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1])));
}

#define STAGE_K 16       // candidate rows are staged in shared memory for even k <= STAGE_K,
#define STAGE_K_WIDE 24  // and in a single colony for even k up to STAGE_K_WIDE (a wider stage)

// 16-byte async copy global -> shared, cached in L2 only, with an L2 eviction-priority policy
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, unsigned long long policy) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "l"(policy)
                 : "memory");
}
__device__ __forceinline__ unsigned long long evict_last_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Dynamic shared memory of one ant: [staging rows (if staged)] [BoostSmem] [visited bitset].
// sk: the stage width of the launch (STAGE_K, or STAGE_K_WIDE for a single colony with k above STAGE_K).
__host__ __device__ inline size_t stage_bytes(int k, int sk) { return (k <= sk && !(k & 1)) ? 2 * (size_t)sk * sk * sizeof(CandW) : 0; }
__host__ __device__ inline size_t boost_offset(int k, int sk) { return stage_bytes(k, sk); }
__host__ __device__ inline size_t bits_offset(int k, int sk) { return (boost_offset(k, sk) + sizeof(BoostSmem) + 15) & ~(size_t)15; }
inline int single_stage_width(int k) { return (k > STAGE_K && k <= STAGE_K_WIDE && !(k & 1)) ? STAGE_K_WIDE : STAGE_K; }

// ---------------------------------------------------------------- asynchronous l_best sharing
// Moves ant a's weight q_a from the old to the new neighbour entries (c, 0) = succ and
// (c, 1) = pred of city c (side < 0: both; else that side only): the integer pheromone of each old
// entry's candidate edge loses q_a and each new one's gains it, as two's complement adds on the
// 64-bit table (so the order of all ants' adds does not matter); a removal and an addition on
// the same candidate edge cancel and are skipped.
__device__ __forceinline__ void move_entries(const LbestArgs& A, int a, int c, int side, int succ, int pred,
                                             unsigned long long qa) {
    const int k = A.k;
    const size_t e = ((size_t)c * A.m + a) * 2;
    uint8_t o0 = 0xFF, o1 = 0xFF, n0 = 0xFF, n1 = 0xFF;
    if (side < 0) {
        const uint16_t old2 = *reinterpret_cast<const uint16_t*>(A.nbrank_w + e);
        o0 = (uint8_t)(old2 & 0xFFu);
        o1 = (uint8_t)(old2 >> 8);
        ranks_of(A.cand, k, c, succ, pred, n0, n1);
        A.nb_w[e] = succ;
        A.nb_w[e + 1] = pred;
        *reinterpret_cast<uint16_t*>(A.nbrank_w + e) = (uint16_t)(n0 | (n1 << 8));
    } else {
        o0 = A.nbrank_w[e + side];
        const int nbr = side == 0 ? succ : pred;
        n0 = rank_of(A.cand, k, c, nbr);
        A.nb_w[e + side] = nbr;
        A.nbrank_w[e + side] = n0;
    }
    if (o0 == n0) o0 = n0 = 0xFF;
    else if (o0 == n1) o0 = n1 = 0xFF;
    if (o1 == n0) o1 = n0 = 0xFF;
    else if (o1 == n1) o1 = n1 = 0xFF;
    unsigned long long* Qc = A.Qt + (size_t)c * k;
    if (o0 < (uint8_t)k) atomicAdd(Qc + o0, 0ull - qa);
    if (o1 < (uint8_t)k) atomicAdd(Qc + o1, 0ull - qa);
    if (n0 < (uint8_t)k) atomicAdd(Qc + n0, qa);
    if (n1 < (uint8_t)k) atomicAdd(Qc + n1, qa);
}

// Asynchronous sharing (the paper's CPU colony runs its ants asynchronously, Section 3): a
// partial rebuild strictly shorter than the ant's l_best replaces it at once, before the update
// step: the rebuilt positions of l_best, the neighbour entries of the M + 2 cities they touch,
// the integer pheromone of those entries' candidate edges (the ant keeps the weight q_a of the
// iteration start until the update step recomputes every weight from C_gbest), and the Eq. 1
// weights of the touched cities' rows, recomputed from the table.  Other ants read these values
// while they construct; every value is one aligned 1-, 2-, 4- or 8-byte store, so a reader sees
// an old or a new value.  The update step's commit then finds C_lbest equal to the new length
// and leaves the ant alone.
static __device__ void async_commit(const LbestArgs& A, int a, const AntIter& it, const int* seg, int lane) {
    const int n = A.n, k = A.k, M = it.M;
    if (!(it.newlen < A.clen[a])) return;  // only this ant writes its C_lbest during the launch
    const unsigned long long qa = A.q[a];
    int* L = A.lbest_w + (size_t)a * n;
    const int e = L[(it.s + it.P - 1) % n];  // last preserved city, followed by the segment
    const int start = it.start;              // first preserved city, preceded by the segment
    __syncwarp();
    for (int t = lane; t < M; t += 32) L[(it.s + it.P + t) % n] = seg[t];
    for (int t = lane; t < M + 2; t += 32) {
        if (t < M) move_entries(A, a, seg[t], -1, t == M - 1 ? start : seg[t + 1], t == 0 ? e : seg[t - 1], qa);
        else if (t == M) move_entries(A, a, e, 0, seg[0], 0, qa);
        else move_entries(A, a, start, 1, 0, seg[M - 1], qa);
    }
    __syncwarp();
    // Eq. 1 weights of the touched rows: two rows per group for k <= 16 (a half-warp each), four
    // groups per pass so that their table reads are in flight together
    const int per = k <= 16 ? 2 : 1;
    const int r = per == 2 ? (lane & 15) : lane;
    const int half = per == 2 ? (lane >> 4) : 0;
    const unsigned gmask = per == 2 ? (half ? 0xFFFF0000u : 0x0000FFFFu) : FULL;
    for (int i0 = 0; i0 < M + 2; i0 += 4 * per) {
        int c[4];
        bool act[4];
        unsigned long long Q[4];
        double et[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int i = i0 + g * per + half;
            c[g] = i < M ? seg[i] : i == M ? e : start;
            act[g] = i < M + 2 && r < k;
            const size_t ix = (size_t)c[g] * k + r;
            Q[g] = act[g] ? __ldcg(A.Qt + ix) : 0ull;
            et[g] = act[g] ? A.etab[ix] : 0.0;
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const double tau = __dadd_rn(A.tau0, __dmul_rn(__ull2double_rn(Q[g]), 0x1.0p-32));
            const double wv = __dmul_rn(powr(tau, A.alpha), et[g]);
            const float w32 = __double2float_rn(wv);
            const bool flag = act[g] && !(w32 >= FLT_MIN && w32 <= FLT_MAX);
            const bool fl = (__ballot_sync(FULL, flag) & gmask) != 0u;
            if (act[g]) {
                const size_t ix = (size_t)c[g] * k + r;
                A.W64_w[ix] = wv;
                A.candw_w[ix].w = fl ? -1.0f : w32;
                if (r == 0) A.rowflag_w[c[g]] = fl ? 1 : 0;
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        A.clen[a] = it.newlen;
        A.cfix_w[2 * a] = it.fix_lo;
        A.cfix_w[2 * a + 1] = it.fix_hi;
        atomicAdd(&A.counters[CNT_IMPROVED], 1ull);
    }
    __syncwarp();
}

// One warp per ant.  Single colony: block b is ant b and the descriptor is the launch
// parameter.  Batched colonies (BATCH): warp w of block b takes ant slot b * warps + w, which
// names (instance, ant); the descriptor comes from the per-instance array and the iteration
// from device memory, so one captured launch serves every iteration.
// One ant's tour of the iteration, built by one warp (lane = this thread's lane) in the ant's
// shared memory my_smem: the draws of Algorithm 1, the visited set, the Eq. 1 decisions and the
// exhausted-list steps, and the exact length.  BATCH: the ant belongs to a batched colony.
template <bool BATCH, int SK>
__device__ __forceinline__ void construct_ant(const LbestArgs& A, int a, int iteration, unsigned char* my_smem,
                                              int lane) {
    // double-buffered copies of the candidate rows of the current city's unvisited candidates:
    // the next city is one of them, so its row is in shared memory when the next decision starts
    CandW(*stage)[SK][SK] = reinterpret_cast<CandW(*)[SK][SK]>(my_smem);
    BoostSmem& boost = *reinterpret_cast<BoostSmem*>(my_smem + boost_offset(A.k, SK));
    uint32_t* bits = reinterpret_cast<uint32_t*>(my_smem + bits_offset(A.k, SK));
    const int n = A.n, k = A.k;
    const int W = (n + 31) >> 5;
    bhash_clear(boost, lane);
    bool partial = false;
    if (A.initialized) {
        partial = true;
        if (A.p_partial < 1.0) {
            const Draw4 d = aco_draw(A.seed, 0, a, iteration, PURPOSE_COIN);
            partial = unit53(d.x0, d.x1) < A.p_partial;
        }
    }
    const int* L = A.lbest + (size_t)a * n;
    int* seg = A.seg + (size_t)a * n;
    int cur, steps, s = -1, P = 0, M, start;
    int ucount = 0;
    if (partial) {
        const Draw4 d1 = aco_draw(A.seed, 0, a, iteration, PURPOSE_START);
        s = (int)below(d1.x0, (uint32_t)n);
        long long fm = (long long)floor(__dmul_rn(A.f, (double)n));
        long long pmin = (long long)n - fm;
        if (pmin < 1) pmin = 1;
        if (pmin > n - 1) pmin = n - 1;
        const Draw4 d2 = aco_draw(A.seed, 0, a, iteration, PURPOSE_KEEP);
        P = (int)pmin + (int)below(d2.x0, (uint32_t)(n - pmin));
        M = n - P;
        for (int w = lane; w < W; w += 32) bits[w] = 0xFFFFFFFFu;
        __syncwarp();
        int* ul = A.ulist + (size_t)a * A.ucap;
        float2* uxy = A.uxy + (size_t)a * A.ucap;
        for (int t = lane; t < M; t += 32) {
            int pos = s + P + t;
            pos -= pos >= n ? n : 0;
            pos -= pos >= n ? n : 0;
            const int c = L[pos];
            atomicAnd(&bits[c >> 5], ~(1u << (c & 31)));
            ul[t] = c;
            uxy[t] = A.xy32[c];
        }
        ucount = M;
        cur = L[(s + P - 1) % n];
        start = L[s];
        steps = M;
    } else {
        const Draw4 d1 = aco_draw(A.seed, 0, a, iteration, PURPOSE_START);
        start = (int)below(d1.x0, (uint32_t)n);
        for (int w = lane; w < W; w += 32) bits[w] = 0u;
        if (A.fallback == 0) counts_init(A, a, lane);
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
    const bool staged = (k <= SK) && !(k & 1);
    const unsigned long long keep_pol = evict_last_policy();  // the candidate table stays in L2
    const int scan_lim = k <= 16 ? 16 : 32;  // Kogge-Stone levels needed for k lanes
    double my_u = 0.0;
    float my_uf = 0.f;
    unsigned long long nfall = 0, nres = 0, nfb_m = 0, nfb_scan = 0, nfast = 0;
    const CandW* rowp = A.candw + (size_t)cur * k;  // current row (global or a staged copy)
    int wb = 0;                                      // staging buffer written this step
    int pend = -1;                                   // chosen city whose visited bit is set next step
    int counted = 0;  // full construction: tour positions already removed from the unvisited counts
    for (int t = 0; t < steps; ++t) {
        if ((t & 31) == 0) {
            const Draw4 d = aco_draw(A.seed, (uint32_t)(t + lane), a, iteration, PURPOSE_WHEEL);
            my_u = unit53(d.x0, d.x1);
            my_uf = __double2float_rn(my_u);
        }
        if (staged) {  // copies issued in the previous step have landed
            cp_async_wait_all();
            __syncwarp();
        }
        // the previous step's city is marked now: it is not a candidate of itself, and the
        // warp synchronises before the next candidate test and before any exhausted step
        // (a plain read-modify-write: during the walk lane 0 is the set's only writer)
        if (lane == 0 && pend >= 0) bits[pend >> 5] |= 1u << (pend & 31);
        int c = -1;
        float w = 0.f;
        bool feas = false;
        if (lane < k) {
            const CandW e = rowp[lane];
            c = e.city;
            w = e.w;
            feas = !is_visited(bits, c);
            if (feas && staged) {
                const CandW* src = A.candw + (size_t)c * k;
                CandW* dst = &stage[wb][lane][0];
#pragma unroll
                for (int q = 0; q < SK; q += 2)
                    if (q < k) cp_async16(dst + q, src + q, keep_pol);
            }
        }
        if (staged) cp_async_commit();
        const unsigned fmask = __ballot_sync(FULL, feas);
        int pick = -1;
        if (fmask && A.selection == 1) {
            // Independent Roulette: the candidate's exact weight times its own uniform; the
            // largest positive product wins, ties to the lowest rank.  Screen first: the staged
            // FP32 weight times the FP32 uniform is within 4 * 2^-24 (relative) of the exact
            // product, so a normal best screen product above every other one by the factor
            // 1 + 2^-18 belongs to the exact winner; otherwise (a near tie, or a row the screen
            // cannot represent) the exact FP64 products decide.
            uint32_t xr = 0u;
            if (feas) {
                const Draw4 d = aco_draw(A.seed, 8u * (uint32_t)t + (uint32_t)(lane >> 2), a, iteration, PURPOSE_IR);
                xr = (lane & 3) == 0 ? d.x0 : (lane & 3) == 1 ? d.x1 : (lane & 3) == 2 ? d.x2 : d.x3;
            }
            int p32 = -1;
            if (!__any_sync(FULL, feas && !(w > 0.f))) {
                const float uf = __fmul_rn(__fadd_rn(__uint2float_rn(xr), 0.5f), 0x1.0p-32f);
                const unsigned key = feas ? __float_as_uint(__fmul_rn(w, uf)) : 0u;  // order of non-negative floats
                const unsigned amax = __reduce_max_sync(FULL, key);
                const unsigned win = __ballot_sync(FULL, feas && key == amax);
                if (__popc(win) == 1 && amax >= __float_as_uint(FLT_MIN)) {
                    const int wl = __ffs(win) - 1;
                    const unsigned second = __reduce_max_sync(FULL, lane == wl ? 0u : key);
                    if (__uint_as_float(amax) > __fmul_rn(__uint_as_float(second), 1.0f + 0x1.0p-18f)) p32 = wl;
                }
            }
            if (p32 >= 0) {
                pick = p32;
            } else {
                ++nres;
                double prod = 0.0;
                if (feas) {
                    const double w64 = A.W64[(size_t)cur * k + lane];
                    if (w64 > 0.0) prod = __dmul_rn(w64, __dmul_rn(__dadd_rn(__uint2double_rn(xr), 0.5), 0x1.0p-32));
                }
                double bp = prod;
                int bl = prod > 0.0 ? lane : 32;
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const double ob = __shfl_xor_sync(FULL, bp, o);
                    const int ol = __shfl_xor_sync(FULL, bl, o);
                    if (ob > bp || (ob == bp && ol < bl)) {
                        bp = ob;
                        bl = ol;
                    }
                }
                pick = bl < 32 ? bl : -1;
            }
        } else if (fmask) {
            float S = feas ? w : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                if (o < scan_lim) {
                    const float v = __shfl_up_sync(FULL, S, o);
                    if (lane >= o) S = __fadd_rn(S, v);
                }
            }
            const float T = __shfl_sync(FULL, S, scan_lim - 1);
            bool exact = !(T > 0.f);  // a flagged row carries negative screen weights
            if (!exact) {
                const float tf = __fmul_rn(__shfl_sync(FULL, my_uf, t & 31), T);
                float prev = __shfl_up_sync(FULL, S, 1);
                if (lane == 0) prev = 0.f;
                const float delta = __fmul_rn(T, 0x1.0p-19f);
                // lane r is the pick when prefix(r-1) <= u*T < prefix(r); it is safe when u*T is
                // farther than the FP32 error bound from both prefixes
                const bool isp = feas && S > tf && !(prev > tf);
                const bool safe = __fsub_rn(tf, prev) > delta && __fsub_rn(S, tf) > delta;
                const unsigned pm = __ballot_sync(FULL, isp && safe);
                const unsigned bad = __ballot_sync(FULL, isp && !safe);
                if (pm && !bad) pick = __ffs(pm) - 1;
                else exact = true;
            }
            if (exact) {
                ++nres;
                pick = wheel_exact_row(A.W64 + (size_t)cur * k, fmask, k, __shfl_sync(FULL, my_u, t & 31));
            }
        }
        int j;
        if (pick >= 0) {
            j = __shfl_sync(FULL, c, pick);
            rowp = staged ? &stage[wb][pick][0] : A.candw + (size_t)j * k;
        } else {
            ++nfall;
            nfb_m += (unsigned long long)M;
            nfb_scan += (unsigned long long)(partial ? ucount : n - 1 - t);
            j = -1;
            if (A.kx && A.fallback == 0 && !partial && !A.initialized) {  // the extended list first
                j = ext_full_choice(A, cur, bits, lane);
                if (j >= 0) ++nfast;
            }
            if (j < 0) {
                if (!partial && A.fallback == 0) {  // the cities chosen so far leave the unvisited counts
                    counts_remove(A, a, seg, counted, t + 1, lane);
                    counted = t + 1;
                }
                j = exhausted_choice(A, a, cur, __shfl_sync(FULL, my_u, t & 31), partial,
                                     staged, ucount, bits, boost, lane, nfast);
            }
            rowp = A.candw + (size_t)j * k;
        }
        wb ^= 1;
        if (lane == 0) seg[outbase + t] = j;
        pend = j;
        __syncwarp();
        cur = j;
    }
    if (staged) cp_async_wait_all();
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
    if (!BATCH && A.async_share && partial) async_commit(A, a, it, seg, lane);
    if (lane == 0) {
        A.antit[a] = it;
        atomicAdd(&A.counters[CNT_DECISIONS], (unsigned long long)steps);
        atomicAdd(&A.counters[CNT_FALLBACKS], nfall);
        atomicAdd(&A.counters[CNT_FB_REBUILT], nfb_m);
        atomicAdd(&A.counters[CNT_FB_SCANNED], nfb_scan);
        atomicAdd(&A.counters[CNT_FB_FAST], nfast);
        atomicAdd(&A.counters[CNT_RESOLVES], nres);
        atomicAdd(&A.counters[partial ? CNT_PARTIAL : CNT_FULL], 1ull);
    }
}

template <bool BATCH, int WARPS, int MINB, int SK = STAGE_K>
__global__ void __launch_bounds__(32 * WARPS, MINB) construct_lbest_kernel(const __grid_constant__ LbestArgs Ap,
                                                                                   const __grid_constant__ BatchMap B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int a = Ap.ant0 + (int)blockIdx.x, inst = 0;
    if (BATCH) {
        const int slot = blockIdx.x * WARPS + warp;
        if (slot >= B.slots) return;  // no block-wide synchronisation below: warps are independent
        const int2 sa = B.slot[slot];
        inst = sa.x;
        a = sa.y;
    }
    const LbestArgs& A = BATCH ? B.args[inst] : Ap;
    const int iteration = BATCH ? *B.iteration : Ap.iteration;
    unsigned char* my_smem = smem_raw + (BATCH ? (size_t)warp * B.smem_per_ant : 0);
    construct_ant<BATCH, SK>(A, a, iteration, my_smem, lane);
}

// Host: one batched construction launch of `blocks` blocks of W ants (warps) each, at least MB
// resident blocks per SM (the register cap), `smem` bytes of dynamic shared memory per block.
template <int W, int MB>
cudaError_t launch_batch_schedule(const BatchMap& B, int blocks, size_t smem, cudaStream_t s) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(construct_lbest_kernel<true, W, MB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    LbestArgs dummy{};
    construct_lbest_kernel<true, W, MB><<<blocks, 32 * W, smem, s>>>(dummy, B);
    return cudaGetLastError();
}

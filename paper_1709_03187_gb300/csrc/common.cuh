// common.cuh -- device helpers and the instance layout of the GB300 ACO library.
//
// Numerics shared by every kernel (compiled with --fmad=false so that every FP64 operation is
// a single IEEE rounding):
//  * d_ij = sqrt(dx*dx + dy*dy) in FP64; eta = 1/d (Section 2).
//  * Integer exponents 0..64 are evaluated by repeated multiplication, others by pow().
//  * Tour lengths are exact: each edge length goes onto a 2^-96 fixed-point grid (unsigned
//    128-bit integers), integer sums are order-free, one final round-half-even to FP64.
//  * Section 3 pheromone: w_a = C_gbest / C_a held as round(w_a * 2^32) (uint64), so every
//    pheromone sum is an exact integer Q and tau = tau0 + Q * 2^-32.
//  * Philox4x32-10 (Salmon et al., SC'11) keyed by the seed, counter (index, ant, iteration,
//    purpose); u = 53 bits / 2^53; integers in [0, r) by the multiply-shift (x * r) >> 32.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/aco.h"

#define ACO_MAX_K 32
#define ACO_BATCH_CONFIGS 8    // four-launch schedules the batch autotuner times
#define ACO_PERSIST_CONFIGS 4  // persistent schedules it times as well

typedef unsigned __int128 u128;

// ------------------------------------------------------------------ random numbers
enum : uint32_t { PURPOSE_WHEEL = 0, PURPOSE_START = 1, PURPOSE_KEEP = 2, PURPOSE_COIN = 3, PURPOSE_IR = 4, PURPOSE_LS = 5 };

#define ACO_CBLK 8            // grid cells per edge of a coarse block (nearest-unvisited search)
#define ACO_LS_MAX_ANTS 8     // ants improved by local search per iteration, at most
#define ACO_LS_MAX_PASSES 16  // windowed 2-opt passes, at most
#define ACO_KX 32             // extended neighbour list: the 32 nearest cities (candidates first)
#define ACO_KF 128            // far list of large colonies: the 128 nearest cities (the extended list first)
#define ACO_FAR_MIN_N 8192    // colonies with more cities keep the far list

struct Draw4 { uint32_t x0, x1, x2, x3; };

__device__ __forceinline__ Draw4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ Draw4 aco_draw(uint64_t seed, uint32_t index, uint32_t ant, uint32_t iteration,
                                          uint32_t purpose) {
    return philox4x32_10(index, ant, iteration, purpose, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ double unit53(uint32_t x0, uint32_t x1) {
    const unsigned long long b = ((((unsigned long long)x0) << 32) | x1) >> 11;
    return __dmul_rn(__ull2double_rn(b), 0x1.0p-53);
}

__device__ __forceinline__ uint32_t below(uint32_t x, uint32_t range) {
    return (uint32_t)(((unsigned long long)x * range) >> 32);
}

// ------------------------------------------------------------------ geometry
__device__ __forceinline__ double dist2(double xi, double yi, double xj, double yj) {
    const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__device__ __forceinline__ bool exp_is_small_int(double e) { return e >= 0.0 && e <= 64.0 && floor(e) == e; }

// x^e with the library's convention (repeated multiplication for small integer e).
__device__ __forceinline__ double powr(double x, double e) {
    if (exp_is_small_int(e)) {
        const int t = (int)e;
        double p = 1.0;
        for (int i = 0; i < t; ++i) p = __dmul_rn(p, x);
        return p;
    }
    return pow(x, e);
}

// x^t for a small integer t: the same products as powr (its first factor 1.0 * x is x exactly).
__device__ __forceinline__ double pow_int(double x, int t) {
    if (t == 0) return 1.0;
    double p = x;
    for (int i = 1; i < t; ++i) p = __dmul_rn(p, x);
    return p;
}

__device__ __forceinline__ double eta_pow_from_d2(double d2, double beta) {
    const double eta = __ddiv_rn(1.0, __dsqrt_rn(d2));
    return powr(eta, beta);
}

// ------------------------------------------------------------------ candidate ranks
__device__ __forceinline__ uint8_t rank_of(const int* __restrict__ cand, int k, int city, int other) {
    const int* row = cand + (size_t)city * k;
    for (int r = 0; r < k; ++r)
        if (row[r] == other) return (uint8_t)r;
    return 0xFF;
}

// Candidate ranks of `succ` and `pred` in the list of `c` (0xFF = not a candidate).  For k a
// multiple of 4 the row is read with 16-byte loads in one round and compared in registers.
__device__ __forceinline__ void ranks_of(const int* __restrict__ cand, int k, int c, int succ, int pred, uint8_t& rs,
                                         uint8_t& rp) {
    rs = rp = 0xFF;
    if ((k & 3) == 0 && k <= 32) {
        const int4* row = reinterpret_cast<const int4*>(cand + (size_t)c * k);
        int4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (4 * q < k) v[q] = __ldg(row + q);
#pragma unroll
        for (int q = 7; q >= 0; --q) {  // descending, so the lowest matching rank is kept
            if (4 * q >= k) continue;
            const int e[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int h = 3; h >= 0; --h) {
                if (e[h] == succ) rs = (uint8_t)(4 * q + h);
                if (e[h] == pred) rp = (uint8_t)(4 * q + h);
            }
        }
        return;
    }
    rs = rank_of(cand, k, c, succ);
    rp = rank_of(cand, k, c, pred);
}

// ------------------------------------------------------------------ exact lengths
// Round-half-even of d * 2^96 for finite d >= 0 with d < 2^31.
__device__ __forceinline__ u128 len_to_fix(double d) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;  // zero or subnormal: below half a grid step
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int e = ex - 979;  // value * 2^96 = m * 2^(ex - 1075 + 96)
    if (e >= 0) return ((u128)m) << e;
    const int sh = -e;
    if (sh >= 64) return 0;
    unsigned long long q = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return (u128)q;
}

// Round-half-even of a * 2^-96 to FP64.
__device__ __forceinline__ double fix_to_len(u128 a) {
    if (a == 0) return 0.0;
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    if (msb <= 52) return __dmul_rn(__ull2double_rn(lo), 0x1.0p-96);  // exact
    int shift = msb - 52;
    u128 mant = a >> shift;
    const u128 rem = a & ((((u128)1) << shift) - 1);
    const u128 half = ((u128)1) << (shift - 1);
    if (rem > half || (rem == half && (mant & 1))) ++mant;
    if (mant == (((u128)1) << 53)) { mant >>= 1; ++shift; }
    // mant < 2^53 is exact in FP64; scale by 2^(shift - 96) (exact power of two)
    const double scale = __longlong_as_double((long long)(1023 + shift - 96) << 52);
    return __dmul_rn(__ull2double_rn((unsigned long long)mant), scale);
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int mask) {
    unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
    hi = __shfl_xor_sync(0xffffffffu, hi, mask);
    lo = __shfl_xor_sync(0xffffffffu, lo, mask);
    return (((u128)hi) << 64) | lo;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
    return v;
}

// ------------------------------------------------------------------ device error flags
enum : int {
    DEVERR_DUPLICATE = 1,      // coincident cities (d = 0)
    DEVERR_BAD_TOUR = 2,       // tour index out of range
    DEVERR_NONFINITE = 4,      // eta^beta or a weight is not finite
    DEVERR_NO_CHOICE = 8,      // an ant found no unvisited city (internal inconsistency)
    DEVERR_BAD_SCORE = 16,     // an edge score that is not finite and > 0
    DEVERR_BAD_RECORD = 32,    // an imported commit record that does not fit the colony
};

// ------------------------------------------------------------------ grid
struct GridDesc {
    double xmin, ymin, xmax, ymax;
    double h;        // cell edge
    double margin;   // conservative slack of ring lower bounds
    int gx, gy;      // cells per axis
};

__device__ __forceinline__ int cell_coord(double v, double vmin, double h, int g) {
    int c = (int)floor(__ddiv_rn(__dsub_rn(v, vmin), h));
    return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

// Lower bound on the distance from (qx,qy) to any point outside the block of cells
// [cx-r, cx+r] x [cy-r, cy+r] (sides on the grid boundary are open: nothing lies beyond them).
// Returns a negative value when the block covers the whole grid.
__device__ __forceinline__ double ring_lower_bound(const GridDesc& g, double qx, double qy, int cx, int cy, int r) {
    double lb = 1e300;
    bool open = false;
    if (cx - r > 0) { lb = fmin(lb, qx - (g.xmin + (double)(cx - r) * g.h)); open = true; }
    if (cx + r < g.gx - 1) { lb = fmin(lb, (g.xmin + (double)(cx + r + 1) * g.h) - qx); open = true; }
    if (cy - r > 0) { lb = fmin(lb, qy - (g.ymin + (double)(cy - r) * g.h)); open = true; }
    if (cy + r < g.gy - 1) { lb = fmin(lb, (g.ymin + (double)(cy + r + 1) * g.h) - qy); open = true; }
    if (!open) return -1.0;
    lb -= g.margin;
    return lb < 0.0 ? 0.0 : lb;
}

// ------------------------------------------------------------------ per-ant iteration record
struct AntIter {
    int32_t s;        // start position in l_best (partial) or -1 (full construction)
    int32_t P;        // preserved count (partial) or 0
    int32_t M;        // rebuilt city count
    int32_t start;    // first city (full) / l_best[s] (partial)
    double newlen;    // length of the new tour
    unsigned long long fix_lo, fix_hi;  // its exact fixed-point length
};

// Candidate edge as the construction kernel reads it: city and FP32 screen weight.
struct CandW {
    int32_t city;
    float w;
};

enum : int {
    CNT_DECISIONS = 0, CNT_FALLBACKS, CNT_RESOLVES, CNT_IMPROVED, CNT_PARTIAL, CNT_FULL, CNT_LS_MOVES,
    CNT_FB_REBUILT,   // sum over exhausted-list steps of the ant's rebuilt count M
    CNT_FB_SCANNED,   // sum over exhausted-list steps of the remaining-list entries scanned
    CNT_FB_FAST,      // exhausted-list steps whose nearest remaining city came from the extended list
    CNT_N
};

// ------------------------------------------------------------------ update kernel arguments
struct CommitArgs {
    int n, m, k;
    const int* cand;
    int* lbest;
    int* nb;
    uint8_t* nbrank;
    const int* seg;
    const AntIter* antit;
    double* clen;
    unsigned long long* cfix;
    unsigned long long* counters;
};

struct GbestArgs {
    int m;
    const double* clen;
    double* gbest;
    int* gbest_ant;
    unsigned long long* q;
    int keep_prev;
};

struct RebuildArgs {
    int n, m, k;
    double tau0, alpha;
    int ia;  // alpha as a small integer (0 .. 64), else -1
    int use_ants;
    int m_cap;  // shared-memory slots for per-ant weights (largest m of a batch)
    const uint8_t* nbrank;
    const unsigned long long* q;
    const double* etab;
    CandW* candw;
    double* W64;
    uint8_t* rowflag;
    int* errflag;
    unsigned long long* Qt;  // also stores the integer pheromone Q_ir when not null
};

// ------------------------------------------------------------------ persistent batched launch
struct LbestArgs;  // construct_dev.cuh
struct PersistArgs {
    const LbestArgs* largs;
    const CommitArgs* cargs;
    const GbestArgs* gargs;
    const RebuildArgs* rargs;
    const int2* slot;        // ant slots (instance, ant), longest instance first
    const int4* rmap;        // rebuild chunks (instance, first city, end city)
    int slots, ritems, count, iterations, smem_per_ant, pull, m_cap, k;
    int* iteration;          // device iteration counter, advanced at the end of each iteration
    unsigned* queue;         // work counters of the construct, commit and rebuild phases (zero at launch)
    unsigned* bar;           // barrier: [0] arrivals, [1] generation (arrivals zero at launch)
    unsigned long long wait_ns;
    int* status;             // bit 0: a barrier wait ran out
};

// ------------------------------------------------------------------ instance
struct aco_instance {
    aco_params p;
    cudaStream_t stream;
    int device;
    int num_sms;
    char err[512];

    // host-side progress
    bool cand_built;
    bool constructed;   // construct called, update pending
    bool initialized;   // l_best valid (LBEST) / at least one update (DENSE)
    int32_t iterations;
    int32_t last_iteration;

    // geometry (all modes)
    double* xy;            // n*2
    GridDesc grid;         // host copy
    GridDesc* grid_dev;
    int32_t* city_cell;    // n
    int32_t* cell_start;   // ncells + 1
    int32_t* cell_city;    // n, cities ordered by cell
    double* cell_xy;       // n*2, coordinates in cell order
    int32_t* cell_fill;    // ncells (scratch of the counting sort)
    int32_t ncells_cap;

    // candidate (LBEST) mode
    CandW* candw;          // n*k
    int32_t* cand;         // n*k (plain copy for outputs and rank lookups)
    double* etab;          // n*k eta^beta
    double* W64;           // n*k Eq. 1 weight tau^alpha eta^beta (FP64)
    uint8_t* rowflag;      // n: 1 = the FP32 screen cannot represent the row
    int32_t* lbest;        // m*n
    int32_t* nb;           // n*m*2: (succ, pred) of each city in each ant's l_best
    uint8_t* nbrank;       // n*m*2: candidate ranks of (succ, pred), 0xFF = not a candidate
    double* clen;          // m
    unsigned long long* cfix;  // m*2 exact lengths
    unsigned long long* q;     // m
    double* gbest;             // 1
    int32_t* gbest_ant;        // 1
    int32_t* seg;          // m*n new cities of the iteration
    AntIter* antit;        // m
    unsigned long long* accq;  // m*n scratch of the fallback = 1 wheel (kept zero between uses)
    unsigned short* bel;       // m*2m per-ant list of non-candidate neighbour entries
    int32_t* btx;              // m*2m per-ant list of unvisited non-candidate neighbours
    unsigned long long* btq;   // m*2m and the weight of the ant of each such entry
    int32_t* ghk;              // m*2m per-ant hash of boosted cities (kept all -1 between uses)
    unsigned long long* ghq;   // m*2m their summed weights (kept 0 between uses)
    float2* xy32;          // n FP32 coordinates (distance screen of the exhausted-list rule)
    int32_t* ulist;        // m*ucap remaining discarded cities of each ant's partial rebuild
    float2* uxy;           // m*ucap their FP32 coordinates
    int32_t ucap;          // largest rebuilt count, n - max(1, n - floor(f n))
    double f_cap;          // f at creation: the largest f the per-ant lists are sized for
    double ls_p;           // local search: probability per ant and iteration (0 = off)
    int32_t ls_window;     // and its window W (tour positions)
    int32_t* ls_buf;       // ACO_LS_MAX_ANTS * n working tours (allocated when first enabled)
    int32_t* ls_sel;       // selected ants + count
    int32_t* ls_imp;       // per selected ant and pass: a move was made
    float coord_r;         // max |coordinate| (rounded up)
    int32_t* deg;          // n degree-in-best-tours scratch of the edge features
    int32_t* fcnt;         // m*ncells unvisited cities per grid cell during a full construction
    int32_t* ccnt;         // m*ncoarse and per block of ACO_CBLK x ACO_CBLK cells
    int32_t* csize;        // ncoarse cities per block
    int32_t ncells, ncoarse, cgx, cgy;
    bool scored;           // candidate edges carry learned scores instead of eta^beta
    int32_t async_share;   // partial rebuilds commit inside the construction launch
    unsigned long long* Qt;  // n*k integer pheromone of the candidate edges (allocated with async_share)
    bool in_batch;         // owned by a batch (advanced by the batch's launches only)
    int32_t ant0, ant1;    // the ants this instance constructs (a rank's share of a sharded colony)
    long long* rec_off;    // m: where each imported commit record starts
    int32_t* nrec;         // 1: imported records
    int32_t kx;            // extended list length min(ACO_KX, n - 1) (0 = no extended list)
    int32_t* ext;          // n*kx: the kx nearest other cities, key (d^2, index); its first k are the candidates
    int32_t* far;          // n*ACO_KF when n > ACO_FAR_MIN_N: the ACO_KF nearest, key (d^2, index); ext is its prefix

    // dense mode
    double* tau;           // n*n
    double* etab_d;        // n*n
    double* W64d;          // n*n
    float* W32d;           // n*n
    int32_t* tours;        // m*n
    int32_t* succ_d;       // m*n
    int32_t* pred_d;       // m*n

    // counters / errors
    unsigned long long* counters;  // CNT_N
    int* errflag;
};

// ------------------------------------------------------------------ host helpers
// A caller's buffer is read and written by kernels in units of its element type (or wider):
// true when a non-null pointer is not aligned to `to` bytes.
static inline bool aco_misaligned(const void* p, uintptr_t to) { return p && ((uintptr_t)p & (to - 1)) != 0; }
aco_status set_err(aco_instance* inst, aco_status s, const char* fmt, ...);
aco_status check_launch(aco_instance* inst, const char* what);
aco_status sync_and_check(aco_instance* inst, const char* what);
aco_status launch_reweight(aco_instance* inst);
aco_status launch_local_search(aco_instance* inst, int32_t iteration);

// kernels launched from the API (defined in the .cu files)
aco_status launch_build_grid_and_knn(aco_instance* inst);
aco_status launch_coarse_sizes(aco_instance* inst);
aco_status launch_dense_init(aco_instance* inst);
aco_status launch_lbest_init_weights(aco_instance* inst);
aco_status launch_construct_lbest(aco_instance* inst, int32_t iteration);
aco_status launch_construct_dense(aco_instance* inst, int32_t iteration);
aco_status launch_write_new_tours(aco_instance* inst, int32_t* tours_out, double* len_out);
aco_status launch_update_lbest(aco_instance* inst);
aco_status launch_update_dense(aco_instance* inst);
aco_status launch_tour_lengths(aco_instance* inst, const int32_t* tours, int32_t count, double* out);
aco_status launch_set_lbest(aco_instance* inst, const int32_t* lbest);
aco_status launch_step_probs(aco_instance* inst, int32_t city, const uint32_t* bits, float* probs, int32_t* exhausted);

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// An NVTX range over one ABI call: a named span on a profiler's timeline, nearly free without one.
struct AcoRange {
    explicit AcoRange(const char* name) { nvtxRangePushA(name); }
    ~AcoRange() { nvtxRangePop(); }
};
#define ACO_RANGE(name) AcoRange aco_range_(name)

/*
 * aco_oracle.c -- plain, slow CPU oracle for the ACO hot path of
 * D. M. Chitty, "Applying ACO To Large Scale TSP Instances" (UKCI 2017, arXiv 1709.03187).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the correctness reference that the CUDA library is
 * checked against. Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the library never calls it and shares no code, header or table with it.
 *
 * Everything is FP64 and single-threaded, written as the paper states the method, with the
 * readings below where the paper is silent or garbled:
 *
 *   Problem (Section 2): symmetric Euclidean TSP, d_ij = sqrt(dx*dx + dy*dy), tour length =
 *     sum of the n edges including the closing edge.  The sum is taken exactly: each edge
 *     length is placed on a 2^-96 fixed-point grid (exact for d >= 2^-44), the integers are
 *     added, and the total is rounded once to FP64.  The result is therefore the correctly
 *     rounded sum, independent of summation order.
 *   Eq. 1 (random proportional rule): p_ij = tau_ij^a eta_ij^b / sum_{l in N} tau_il^a eta_il^b,
 *     eta = 1/d.  The wheel is the FP64 cumulative sum in index (dense) or candidate-rank
 *     (candidate lists) order; the pick is the first entry whose cumulative sum exceeds
 *     u * total, u in [0,1) from 53 random bits.
 *   Eq. 2: tau <- (1 - rho) tau on every edge.  Eq. 3-5: tau_ij <- tau_ij + sum_k dtau_ij^k,
 *     dtau = 1/C^k on both (i,j) and (j,i) for every edge of tour k (C^k is the tour length;
 *     the text's "1/C^k is the length" is read as "C^k is the length").
 *   Section 3 (pheromone-matrix-free form): each ant a keeps its best tour l_best_a of length
 *     C_a.  An edge of l_best_a contributes w_a = C_gbest / C_a (a value in (0,1]); the
 *     pheromone of edge (i,j) is tau0 + sum_a w_a [j is a neighbour of i in l_best_a].  Each
 *     w_a is held as a 32-bit binary fraction (round-half-even of w_a * 2^32) so that the sum
 *     over ants is exact and order-free; tau = tau0 + Q * 2^-32 with Q the integer sum.
 *   Candidate lists: the k nearest other cities, key (d^2, index) ascending.  When every
 *     candidate is visited the ant takes argmax over all unvisited j of tau_ij^a eta_ij^b
 *     (ties -> lowest j), or, with fallback = 1, the Eq. 1 wheel over all unvisited cities.
 *   Algorithm 1 (PartialACO): initial tours by full construction (tau = tau0 everywhere, as
 *     there is no l_best yet).  Each iteration each ant draws a start position s in its
 *     l_best, a preserved count P uniform in [max(1, n - floor(f n)), n-1], keeps the P
 *     cities l_best[s..s+P-1] (cyclic), and rebuilds the other M = n - P cities by Eq. 1
 *     starting from l_best[s+P-1]; the tour closes to l_best[s].  The rebuilt cities are
 *     written in place of the discarded ones.  With probability 1 - p_partial the ant builds a
 *     full tour instead.  If the new tour is strictly shorter it replaces l_best.
 *     Pheromone is fixed during an iteration (all ants read the l_best set of the previous
 *     iteration); commits happen after every ant has built its tour.
 *   Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = seed
 *     (low, high word), counter = (index, ant, iteration, purpose); purpose 0 = wheel draw of
 *     decision `index`, 1 = start city / start position, 2 = preserved count, 3 = partial coin,
 *     4 = Independent Roulette draws of decision t (counter index 8 t + r / 4 for rank r).
 *     u = ((x0 << 32 | x1) >> 11) * 2^-53; an integer in [0, r) is (x0 * r) >> 32.
 *   Integer exponents a, b in [0, 64] use repeated multiplication x*x*...*x (left to right);
 *   other exponents call pow().
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction anywhere).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LS_MAX_ANTS 8     /* ants improved by local search per iteration, at most */
#define OR_LS_MAX_PASSES 16  /* windowed 2-opt passes, at most */

/* ------------------------------------------------------------------ Philox4x32-10 (SC'11) */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PH_M0 * c[0];
        uint64_t p1 = (uint64_t)PH_M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += PH_W0; k1 += PH_W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void draw(uint64_t seed, uint32_t index, uint32_t ant, uint32_t iteration, uint32_t purpose,
                 uint32_t out[4]) {
    uint32_t ctr[4] = {index, ant, iteration, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

double or_u53(uint32_t x0, uint32_t x1) {
    uint64_t bits = (((uint64_t)x0 << 32) | x1) >> 11;
    return (double)bits * 0x1.0p-53;
}

uint32_t or_bounded(uint32_t x, uint32_t range) { return (uint32_t)(((uint64_t)x * range) >> 32); }

/* ------------------------------------------------------------------ arithmetic helpers */
static int is_small_int(double e) { return e >= 0.0 && e <= 64.0 && floor(e) == e; }

/* x^e: repeated multiplication for integer e in [0,64], else pow(). */
double or_powr(double x, double e) {
    if (is_small_int(e)) {
        int t = (int)e;
        double p = 1.0;
        for (int i = 0; i < t; ++i) p = p * x;
        return p;
    }
    return pow(x, e);
}

double or_dist2(const double* xy, int i, int j) {
    double dx = xy[2 * i] - xy[2 * j];
    double dy = xy[2 * i + 1] - xy[2 * j + 1];
    return dx * dx + dy * dy;
}

double or_edge_len(const double* xy, int i, int j) { return sqrt(or_dist2(xy, i, j)); }

/* eta^beta with eta = 1/d (Section 2). */
static double eta_pow(const double* xy, int i, int j, double beta) {
    double eta = 1.0 / sqrt(or_dist2(xy, i, j));
    return or_powr(eta, beta);
}

/* Exact tour length: every edge on the 2^-96 grid, integer sum, one final rounding. */
typedef __int128 i128;
static i128 to_fix(double d) { return (i128)nearbyint(ldexp(d, 96)); }
static double from_fix(i128 a) { return ldexp((double)a, -96); }

double or_tour_length(int n, const double* xy, const int32_t* tour) {
    i128 acc = 0;
    for (int p = 0; p < n; ++p) acc += to_fix(or_edge_len(xy, tour[p], tour[(p + 1) % n]));
    return from_fix(acc);
}

void or_tour_lengths(int n, const double* xy, const int32_t* tours, int count, double* out) {
    for (int c = 0; c < count; ++c) out[c] = or_tour_length(n, xy, tours + (size_t)c * n);
}

/* ------------------------------------------------------------------ candidate lists */
/* k nearest other cities of every city, key (d^2, j) ascending; brute force over all j.
 * Returns 0, or -1 if two cities coincide (eta = 1/d is undefined there). */
int or_knn(int n, const double* xy, int k, int32_t* cand) {
    double* kd = (double*)malloc(sizeof(double) * (size_t)k);
    int dup = 0;
    for (int i = 0; i < n; ++i) {
        int32_t* row = cand + (size_t)i * k;
        int filled = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d2 = or_dist2(xy, i, j);
            if (d2 == 0.0) dup = 1;
            /* insertion into the sorted (d2, j) list; j ascending so equal d2 keeps lower j first */
            if (filled == k && !(d2 < kd[k - 1])) continue;
            int pos = filled < k ? filled : k - 1;
            while (pos > 0 && d2 < kd[pos - 1]) {
                kd[pos] = kd[pos - 1];
                row[pos] = row[pos - 1];
                --pos;
            }
            kd[pos] = d2;
            row[pos] = j;
            if (filled < k) ++filled;
        }
    }
    free(kd);
    return dup ? -1 : 0;
}

/* ------------------------------------------------------------------ solver state */
typedef struct {
    int32_t mode; /* 0 = dense (Section 2), 1 = l_best + PartialACO (Section 3) */
    int32_t n, m, k;
    double alpha, beta, rho, tau0;
    double max_mod_frac, p_partial;
    uint64_t seed;
    int32_t fallback; /* 0 = argmax over unvisited, 1 = Eq. 1 wheel over unvisited */
    int32_t selection; /* 0 = Eq. 1 wheel, 1 = Independent Roulette (candidate lists) */
} or_params;

typedef struct {
    or_params p;
    double* xy;      /* n*2 */
    /* dense mode */
    double* tau;     /* n*n */
    double* etab_d;  /* n*n eta^beta */
    /* candidate mode */
    int32_t* cand;   /* n*k */
    double* etab;    /* n*k eta^beta of candidate edges */
    int32_t* lbest;  /* m*n */
    double* clen;    /* m, +inf before the first commit */
    int initialized;
    uint64_t* q;     /* m: round(C_g / C_a * 2^32) */
    uint64_t* Q;     /* n*k pheromone sums of candidate edges */
    int32_t* succ;   /* m*n successor of each city in l_best_a */
    int32_t* pred;   /* m*n predecessor */
    /* the iteration's new tours */
    int32_t* newtour; /* m*n, full tour in l_best layout (dense: construction order) */
    double* newlen;   /* m */
    int32_t* built;   /* m: 1 if ant was constructed this iteration */
    int32_t* seg_s;   /* m: start position s (partial) or -1 (full) */
    int32_t* seg_M;   /* m: rebuilt city count */
    /* local search (Section 3.2 / Section 5): probability per ant and iteration, window */
    double ls_p;
    int32_t ls_window;
    int64_t ls_moves;
    /* counters */
    int64_t decisions, fallbacks, scans;
    int64_t boosted; /* exhausted-list picks with pheromone above tau0 */
    /* scratch */
    unsigned char* visited; /* n */
} or_state;

static void compute_succ_pred(or_state* st) {
    int n = st->p.n;
    for (int a = 0; a < st->p.m; ++a) {
        const int32_t* t = st->lbest + (size_t)a * n;
        for (int pos = 0; pos < n; ++pos) {
            int c = t[pos];
            st->succ[(size_t)a * n + c] = t[(pos + 1) % n];
            st->pred[(size_t)a * n + c] = t[(pos + n - 1) % n];
        }
    }
}

or_state* or_create(const or_params* p, const double* xy) {
    if (p->n < 3 || p->m < 1) return NULL;
    if (p->mode == 1 && (p->k < 1 || p->k > 32 || p->k > p->n - 1)) return NULL;
    or_state* st = (or_state*)calloc(1, sizeof(or_state));
    st->p = *p;
    int n = p->n, m = p->m, k = p->k;
    st->xy = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    memcpy(st->xy, xy, sizeof(double) * 2 * (size_t)n);
    st->visited = (unsigned char*)malloc((size_t)n);
    st->newtour = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
    st->newlen = (double*)malloc(sizeof(double) * (size_t)m);
    st->built = (int32_t*)calloc((size_t)m, sizeof(int32_t));
    st->seg_s = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    st->seg_M = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    if (p->mode == 0) {
        st->tau = (double*)malloc(sizeof(double) * (size_t)n * n);
        st->etab_d = (double*)malloc(sizeof(double) * (size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                st->tau[(size_t)i * n + j] = p->tau0;
                st->etab_d[(size_t)i * n + j] = (i == j) ? 0.0 : eta_pow(st->xy, i, j, p->beta);
            }
    } else {
        st->cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * k);
        if (or_knn(n, st->xy, k, st->cand) != 0) { /* duplicate cities */
            free(st->cand); free(st->xy); free(st->visited); free(st->newtour); free(st->newlen);
            free(st->built); free(st->seg_s); free(st->seg_M); free(st);
            return NULL;
        }
        st->etab = (double*)malloc(sizeof(double) * (size_t)n * k);
        for (int i = 0; i < n; ++i)
            for (int r = 0; r < k; ++r)
                st->etab[(size_t)i * k + r] = eta_pow(st->xy, i, st->cand[(size_t)i * k + r], p->beta);
        st->lbest = (int32_t*)calloc((size_t)m * n, sizeof(int32_t));
        st->clen = (double*)malloc(sizeof(double) * (size_t)m);
        for (int a = 0; a < m; ++a) st->clen[a] = INFINITY;
        st->q = (uint64_t*)calloc((size_t)m, sizeof(uint64_t));
        st->Q = (uint64_t*)calloc((size_t)n * k, sizeof(uint64_t));
        st->succ = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
        st->pred = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
    }
    return st;
}

void or_destroy(or_state* st) {
    if (!st) return;
    free(st->xy); free(st->tau); free(st->etab_d); free(st->cand); free(st->etab);
    free(st->lbest); free(st->clen); free(st->q); free(st->Q); free(st->succ); free(st->pred);
    free(st->newtour); free(st->newlen); free(st->built); free(st->seg_s); free(st->seg_M);
    free(st->visited); free(st);
}

/* ------------------------------------------------------------------ Section 3 pheromone */
/* Deposit of the l_best population: every edge (x,y) of l_best_a adds q_a to the candidate
 * entries (x, rank of y) and (y, rank of x). */
static int rank_in(const or_state* st, int city, int other) {
    const int32_t* row = st->cand + (size_t)city * st->p.k;
    for (int r = 0; r < st->p.k; ++r)
        if (row[r] == other) return r;
    return -1;
}

static void lbest_pheromone(or_state* st) {
    int n = st->p.n, m = st->p.m, k = st->p.k;
    memset(st->Q, 0, sizeof(uint64_t) * (size_t)n * k);
    if (!st->initialized) return;
    double cg = INFINITY;
    for (int a = 0; a < m; ++a) if (st->clen[a] < cg) cg = st->clen[a];
    for (int a = 0; a < m; ++a) st->q[a] = (uint64_t)nearbyint(ldexp(cg / st->clen[a], 32));
    for (int a = 0; a < m; ++a) {
        const int32_t* t = st->lbest + (size_t)a * n;
        for (int pos = 0; pos < n; ++pos) {
            int x = t[pos], y = t[(pos + 1) % n];
            int r = rank_in(st, x, y);
            if (r >= 0) st->Q[(size_t)x * k + r] += st->q[a];
            r = rank_in(st, y, x);
            if (r >= 0) st->Q[(size_t)y * k + r] += st->q[a];
        }
    }
    compute_succ_pred(st);
}

static double tau_from_Q(const or_state* st, uint64_t Q) { return st->p.tau0 + ldexp((double)Q, -32); }

/* tau_ij for any pair, straight from the l_best population (used when the list is exhausted). */
static uint64_t Q_any(const or_state* st, int i, int j) {
    if (!st->initialized) return 0;
    uint64_t s = 0;
    int n = st->p.n;
    for (int a = 0; a < st->p.m; ++a)
        if (st->succ[(size_t)a * n + i] == j || st->pred[(size_t)a * n + i] == j) s += st->q[a];
    return s;
}

/* ------------------------------------------------------------------ Eq. 1 decisions */
/* Eq. 1 wheel over entries w[0..cnt) in the given order; returns the picked position.
 * Entries with w == 0 are infeasible. Returns -1 if no entry has w > 0. */
static int wheel(const double* w, int cnt, double u) {
    double total = 0.0;
    int last = -1;
    for (int e = 0; e < cnt; ++e) {
        total += w[e];
        if (w[e] > 0.0) last = e;
    }
    if (last < 0) return -1;
    double target = u * total;
    double cum = 0.0;
    for (int e = 0; e < cnt; ++e) {
        cum += w[e];
        if (w[e] > 0.0 && cum > target) return e;
    }
    return last; /* u * total rounded up to total */
}

/* One decision of ant `ant` at city i (candidate mode). */
/* Independent Roulette (Section 3): each candidate draws its own uniform and the largest
 * weight x uniform wins.  Among ranks with w[r] > 0, argmax of w[r] * u_r, ties to the lowest
 * rank; u_r = (x + 1/2) 2^-32 with x word r % 4 of the draw (8 t + r / 4, ant, iteration, 4).
 * Returns -1 when no weight is positive (the caller then applies the exhausted-list rule). */
int or_ir_pick(const double* w, int k, uint64_t seed, uint32_t t, uint32_t ant, uint32_t iteration) {
    int best = -1;
    double bp = 0.0;
    for (int r = 0; r < k; ++r) {
        if (!(w[r] > 0.0)) continue;
        uint32_t x[4];
        draw(seed, 8u * t + (uint32_t)(r / 4), ant, iteration, 4, x);
        double u = ((double)x[r % 4] + 0.5) * 0x1.0p-32;
        double prod = w[r] * u;
        if (prod > bp) { bp = prod; best = r; }
    }
    return best;
}

/* Weight tau_ij^alpha eta_ij^beta of the edge (i, j) with tau_ij taken from the whole l_best
 * population (Section 3): the weight Eq. 1 gives an edge once the candidate list is exhausted. */
static double any_weight(const or_state* st, int i, int j) {
    double tau = tau_from_Q(st, Q_any(st, i, j));
    return or_powr(tau, st->p.alpha) * eta_pow(st->xy, i, j, st->p.beta);
}

/* The exhausted-list rule at city i over the unvisited cities (st->visited): the argmax of the
 * weight, ties to the lowest index (fallback 0), or the Eq. 1 wheel over every unvisited city in
 * index order (fallback 1, the ordinary rule of Section 6).  Counts the picks whose pheromone lies
 * above tau0 (an l_best neighbour of i outside its candidate list). */
static int exhausted_pick(or_state* st, int i, double u) {
    const or_params* p = &st->p;
    int n = p->n;
    int pick = -1;
    if (p->fallback == 0) {
        double bw = -1.0;
        for (int j = 0; j < n; ++j) {
            if (st->visited[j]) continue;
            st->scans++;
            double wj = any_weight(st, i, j);
            if (wj > bw) { bw = wj; pick = j; }
        }
    } else {
        double* wa = (double*)malloc(sizeof(double) * (size_t)n);
        int lowest = -1;
        for (int j = 0; j < n; ++j) {
            if (st->visited[j]) { wa[j] = 0.0; continue; }
            if (lowest < 0) lowest = j;
            st->scans++;
            wa[j] = any_weight(st, i, j);
        }
        pick = wheel(wa, n, u);
        free(wa);
        if (pick < 0) pick = lowest;
    }
    if (pick >= 0 && Q_any(st, i, pick) > 0) st->boosted++;
    return pick;
}

static int decide_cand(or_state* st, int ant, int i, uint32_t t, uint32_t iteration) {
    const or_params* p = &st->p;
    int k = p->k;
    uint32_t x[4];
    draw(p->seed, t, (uint32_t)ant, iteration, 0, x);
    double u = or_u53(x[0], x[1]);
    st->decisions++;
    double w[64];
    const int32_t* row = st->cand + (size_t)i * k;
    for (int r = 0; r < k; ++r) {
        if (st->visited[row[r]]) { w[r] = 0.0; continue; }
        st->scans++;
        double tau = tau_from_Q(st, st->Q[(size_t)i * k + r]);
        w[r] = or_powr(tau, p->alpha) * st->etab[(size_t)i * k + r];
    }
    int r = p->selection == 1 ? or_ir_pick(w, k, p->seed, t, (uint32_t)ant, iteration) : wheel(w, k, u);
    if (r >= 0) return row[r];
    /* every candidate visited */
    st->fallbacks++;
    return exhausted_pick(st, i, u);
}

/* One decision at city i (dense mode, Eq. 1 over every unvisited city in index order). */
static int decide_dense(or_state* st, int ant, int i, uint32_t t, uint32_t iteration) {
    const or_params* p = &st->p;
    int n = p->n;
    uint32_t x[4];
    draw(p->seed, t, (uint32_t)ant, iteration, 0, x);
    double u = or_u53(x[0], x[1]);
    st->decisions++;
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    int lowest = -1;
    for (int j = 0; j < n; ++j) {
        if (st->visited[j]) { w[j] = 0.0; continue; }
        if (lowest < 0) lowest = j;
        st->scans++;
        w[j] = or_powr(st->tau[(size_t)i * n + j], p->alpha) * st->etab_d[(size_t)i * n + j];
    }
    int j = wheel(w, n, u);
    free(w);
    return j >= 0 ? j : lowest;
}

/* ------------------------------------------------------------------ tour construction */
static void build_full(or_state* st, int a, uint32_t iteration) {
    int n = st->p.n;
    int32_t* T = st->newtour + (size_t)a * n;
    uint32_t x[4];
    draw(st->p.seed, 0, (uint32_t)a, iteration, 1, x);
    int cur = (int)or_bounded(x[0], (uint32_t)n);
    memset(st->visited, 0, (size_t)n);
    st->visited[cur] = 1;
    T[0] = cur;
    for (int t = 0; t < n - 1; ++t) {
        int j = st->p.mode == 0 ? decide_dense(st, a, cur, (uint32_t)t, iteration)
                                : decide_cand(st, a, cur, (uint32_t)t, iteration);
        st->visited[j] = 1;
        T[t + 1] = j;
        cur = j;
    }
    st->seg_s[a] = -1;
    st->seg_M[a] = n - 1;
}

/* Algorithm 1: keep P cities of l_best from position s, rebuild the other M = n - P. */
static void build_partial(or_state* st, int a, uint32_t iteration) {
    int n = st->p.n;
    const int32_t* L = st->lbest + (size_t)a * n;
    int32_t* T = st->newtour + (size_t)a * n;
    uint32_t x[4];
    draw(st->p.seed, 0, (uint32_t)a, iteration, 1, x);
    int s = (int)or_bounded(x[0], (uint32_t)n);
    int64_t fm = (int64_t)floor(st->p.max_mod_frac * (double)n);
    int64_t pmin = (int64_t)n - fm;
    if (pmin < 1) pmin = 1;
    if (pmin > n - 1) pmin = n - 1;
    draw(st->p.seed, 0, (uint32_t)a, iteration, 2, x);
    int P = (int)pmin + (int)or_bounded(x[0], (uint32_t)((int64_t)n - pmin));
    int M = n - P;
    memcpy(T, L, sizeof(int32_t) * (size_t)n);
    memset(st->visited, 1, (size_t)n);
    for (int q = 0; q < M; ++q) st->visited[L[(s + P + q) % n]] = 0;
    int cur = L[(s + P - 1) % n];
    for (int t = 0; t < M; ++t) {
        int j = decide_cand(st, a, cur, (uint32_t)t, iteration);
        st->visited[j] = 1;
        T[(s + P + t) % n] = j;
        cur = j;
    }
    st->seg_s[a] = s;
    st->seg_M[a] = M;
}

/* Windowed 2-opt (Section 3.2: 2-opt on a constructed tour; Section 5: only edges within W tour
 * positions of each other).  A move (i, j), 2 <= j - i <= W, replaces edges (T[i], T[i+1]) and
 * (T[j], T[j+1]) by (T[i], T[j]) and (T[i+1], T[j+1]), reversing T[i+1..j]; its FP64 gain is
 * (d(a,b) + d(c,d)) - (d(a,c) + d(b,d)) and it is taken when the gain is > 0.  Passes split the
 * positions into blocks at 0, off, off + 2W, off + 4W, ..., n (off = 0 on even passes, W on odd
 * ones); within a block every position i (ascending) scans j = i + 2 .. min(i + W, end - 2)
 * ascending, applies each improving move at once and carries on with the next j.  Moves never
 * cross a block edge, so blocks are independent.  It stops after two passes in a row without a
 * move, or after max_passes.  Returns the number of moves. */
int or_two_opt_windowed(int n, const double* xy, int32_t* T, int W, int max_passes) {
    if (n < 4 || W < 2) return 0;
    int moves = 0, quiet = 0;
    for (int pass = 0; pass < max_passes && quiet < 2; ++pass) {
        const int off = (pass & 1) ? W : 0;
        int improved = 0;
        int b0 = 0;
        while (b0 < n) {
            int b1 = (b0 < off) ? off : b0 + 2 * W;
            if (b1 > n) b1 = n;
            for (int i = b0; i + 3 < b1; ++i) {
                int jmax = i + W < b1 - 2 ? i + W : b1 - 2;
                for (int j = i + 2; j <= jmax; ++j) {
                    int a = T[i], b = T[i + 1], c = T[j], d = T[j + 1];
                    double g = (or_edge_len(xy, a, b) + or_edge_len(xy, c, d)) -
                               (or_edge_len(xy, a, c) + or_edge_len(xy, b, d));
                    if (g > 0.0) {
                        for (int l = i + 1, r = j; l < r; ++l, --r) {
                            int t = T[l]; T[l] = T[r]; T[r] = t;
                        }
                        ++moves;
                        improved = 1;
                    }
                }
            }
            b0 = b1;
        }
        quiet = improved ? 0 : quiet + 1;
    }
    return moves;
}

/* One ant's tour of the iteration: partial rebuild of its l_best (Algorithm 1) or a full
 * construction, then local search if drawn (at most OR_LS_MAX_ANTS ants, counted in *ls_count). */
static void construct_one(or_state* st, int a, int iteration, int* ls_count) {
    int partial = 0;
    if (st->p.mode == 1 && st->initialized) {
        partial = 1;
        if (st->p.p_partial < 1.0) {
            uint32_t x[4];
            draw(st->p.seed, 0, (uint32_t)a, (uint32_t)iteration, 3, x);
            partial = or_u53(x[0], x[1]) < st->p.p_partial;
        }
    }
    if (partial) build_partial(st, a, (uint32_t)iteration);
    else build_full(st, a, (uint32_t)iteration);
    if (st->p.mode == 1 && st->ls_p > 0.0 && *ls_count < OR_LS_MAX_ANTS) {
        uint32_t x[4];
        draw(st->p.seed, 0, (uint32_t)a, (uint32_t)iteration, 5, x);
        if (or_u53(x[0], x[1]) < st->ls_p) {
            ++*ls_count;
            st->ls_moves += or_two_opt_windowed(st->p.n, st->xy, st->newtour + (size_t)a * st->p.n,
                                                st->ls_window, OR_LS_MAX_PASSES);
            st->seg_s[a] = -1;  /* committed as a whole tour */
            st->seg_M[a] = st->p.n - 1;
        }
    }
    st->newlen[a] = or_tour_length(st->p.n, st->xy, st->newtour + (size_t)a * st->p.n);
    st->built[a] = 1;
}

/* Tour construction for every ant (ants == NULL) or for the listed ants only.  rebuild = 0
 * reuses the pheromone computed by the previous call (same l_best population). */
void or_construct_ex(or_state* st, int iteration, const int32_t* ants, int count, int rebuild) {
    int m = st->p.m;
    if (st->p.mode == 1 && rebuild) lbest_pheromone(st);
    if (!ants) count = m;
    memset(st->built, 0, sizeof(int32_t) * (size_t)m);
    int ls_count = 0;
    for (int c = 0; c < count; ++c) construct_one(st, ants ? ants[c] : c, iteration, &ls_count);
}

/* The same construction with the ants spread over `threads` host threads (ant c on thread
 * c mod threads).  Within an iteration the ants only read the shared state (the pheromone is
 * fixed, Section 3 read synchronously) and each writes its own rows, so every thread works on a
 * shallow copy of the state with its own visited scratch and counters; the result is identical
 * to or_construct_ex.  Local search (whose at-most-8 cap follows the ant order) runs sequentially. */
typedef struct {
    or_state view;
    const int32_t* ants;
    int count, first, step, iteration;
} or_worker;

static void* or_worker_run(void* arg) {
    or_worker* w = (or_worker*)arg;
    int ls_count = 0;
    for (int c = w->first; c < w->count; c += w->step) construct_one(&w->view, w->ants ? w->ants[c] : c, w->iteration, &ls_count);
    return NULL;
}

void or_construct_mt(or_state* st, int iteration, const int32_t* ants, int count, int rebuild, int threads) {
    if (!ants) count = st->p.m;
    if (threads > count) threads = count;
    if (threads <= 1 || st->ls_p > 0.0) {
        or_construct_ex(st, iteration, ants, count, rebuild);
        return;
    }
    if (st->p.mode == 1 && rebuild) lbest_pheromone(st);
    memset(st->built, 0, sizeof(int32_t) * (size_t)st->p.m);
    or_worker* w = (or_worker*)calloc((size_t)threads, sizeof(or_worker));
    pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    int* started = (int*)calloc((size_t)threads, sizeof(int));
    for (int t = 0; t < threads; ++t) {
        w[t].view = *st;
        w[t].view.visited = (unsigned char*)malloc((size_t)st->p.n);
        w[t].view.decisions = w[t].view.fallbacks = w[t].view.scans = w[t].view.boosted = 0;
        w[t].ants = ants;
        w[t].count = count;
        w[t].first = t;
        w[t].step = threads;
        w[t].iteration = iteration;
        started[t] = pthread_create(&tid[t], NULL, or_worker_run, &w[t]) == 0;
        if (!started[t]) or_worker_run(&w[t]);
    }
    for (int t = 0; t < threads; ++t) {
        if (started[t]) pthread_join(tid[t], NULL);
        st->decisions += w[t].view.decisions;
        st->fallbacks += w[t].view.fallbacks;
        st->scans += w[t].view.scans;
        st->boosted += w[t].view.boosted;
        free(w[t].view.visited);
    }
    free(w);
    free(tid);
    free(started);
}

void or_construct(or_state* st, int iteration, const int32_t* ants, int count) {
    or_construct_ex(st, iteration, ants, count, 1);
}

/* Pheromone update.  Dense: Eq. 2 then Eq. 3-5 with every ant's new tour.
 * Candidate mode: Algorithm 1's l_best replacement (strictly shorter tours only). */
void or_update(or_state* st) {
    int n = st->p.n, m = st->p.m;
    if (st->p.mode == 0) {
        double keep = 1.0 - st->p.rho;
        for (size_t e = 0; e < (size_t)n * n; ++e) st->tau[e] = keep * st->tau[e];
        int32_t* su = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
        int32_t* pr = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
        for (int a = 0; a < m; ++a) {
            const int32_t* t = st->newtour + (size_t)a * n;
            for (int pos = 0; pos < n; ++pos) {
                su[(size_t)a * n + t[pos]] = t[(pos + 1) % n];
                pr[(size_t)a * n + t[pos]] = t[(pos + n - 1) % n];
            }
        }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i == j) continue;
                double s = 0.0;
                for (int a = 0; a < m; ++a)
                    if (su[(size_t)a * n + i] == j || pr[(size_t)a * n + i] == j) s += 1.0 / st->newlen[a];
                st->tau[(size_t)i * n + j] = st->tau[(size_t)i * n + j] + s;
            }
        free(su);
        free(pr);
        return;
    }
    for (int a = 0; a < m; ++a) {
        if (!st->built[a]) continue;
        if (st->newlen[a] < st->clen[a]) {
            memcpy(st->lbest + (size_t)a * n, st->newtour + (size_t)a * n, sizeof(int32_t) * (size_t)n);
            st->clen[a] = st->newlen[a];
        }
    }
    st->initialized = 1;
}

/* ------------------------------------------------------------------ accessors */
void or_get_lbest(const or_state* st, int32_t* out) {
    memcpy(out, st->lbest, sizeof(int32_t) * (size_t)st->p.m * st->p.n);
}
void or_get_clen(const or_state* st, double* out) { memcpy(out, st->clen, sizeof(double) * (size_t)st->p.m); }
void or_get_newtours(const or_state* st, int32_t* out) {
    memcpy(out, st->newtour, sizeof(int32_t) * (size_t)st->p.m * st->p.n);
}
void or_get_newlen(const or_state* st, double* out) { memcpy(out, st->newlen, sizeof(double) * (size_t)st->p.m); }
void or_get_seg(const or_state* st, int32_t* s_out, int32_t* M_out) {
    memcpy(s_out, st->seg_s, sizeof(int32_t) * (size_t)st->p.m);
    memcpy(M_out, st->seg_M, sizeof(int32_t) * (size_t)st->p.m);
}
void or_get_tau(const or_state* st, double* out) {
    memcpy(out, st->tau, sizeof(double) * (size_t)st->p.n * st->p.n);
}
/* Schedule of the PartialACO parameters between iterations (Section 3.1; Section 7's growing f). */
void or_set_max_mod_frac(or_state* st, double f) { st->p.max_mod_frac = f; }
/* Local search after construction: each ant (index order, at most OR_LS_MAX_ANTS per
 * iteration) whose draw (0, ant, iteration, 5) gives u < p applies the windowed 2-opt. */
void or_set_local_search(or_state* st, double p, int window) { st->ls_p = p; st->ls_window = window; }
int64_t or_ls_moves(const or_state* st) { return st->ls_moves; }
void or_set_p_partial(or_state* st, double p) { st->p.p_partial = p; }

void or_set_tau(or_state* st, const double* tau) {
    memcpy(st->tau, tau, sizeof(double) * (size_t)st->p.n * st->p.n);
}
void or_get_cand(const or_state* st, int32_t* out) {
    memcpy(out, st->cand, sizeof(int32_t) * (size_t)st->p.n * st->p.k);
}
void or_get_etab(const or_state* st, double* out) {
    if (st->p.mode == 0) memcpy(out, st->etab_d, sizeof(double) * (size_t)st->p.n * st->p.n);
    else memcpy(out, st->etab, sizeof(double) * (size_t)st->p.n * st->p.k);
}
void or_get_counters(const or_state* st, int64_t* out4) {
    out4[0] = st->decisions; out4[1] = st->fallbacks; out4[2] = st->scans; out4[3] = st->boosted;
}
void or_reset_counters(or_state* st) { st->decisions = st->fallbacks = st->scans = st->boosted = 0; }
int or_initialized(const or_state* st) { return st->initialized; }

/* Candidate-edge weights tau^alpha * eta^beta of the current l_best population (n*k), i.e.
 * what Eq. 1 multiplies before normalising; also the integer sums Q and the per-ant q. */
void or_cand_weights(or_state* st, double* W, uint64_t* Q_out, uint64_t* q_out) {
    lbest_pheromone(st);
    int n = st->p.n, k = st->p.k;
    for (size_t e = 0; e < (size_t)n * k; ++e)
        W[e] = or_powr(tau_from_Q(st, st->Q[e]), st->p.alpha) * st->etab[e];
    if (Q_out) memcpy(Q_out, st->Q, sizeof(uint64_t) * (size_t)n * k);
    if (q_out) memcpy(q_out, st->q, sizeof(uint64_t) * (size_t)st->p.m);
}

/* Learned proposal: the per-candidate-edge score s_ir replaces eta_ij^beta (j = cand[i][r]) in
 * Eq. 1 for candidate edges; edges outside the candidate list keep eta^beta.  NULL restores the
 * plain heuristic.  Scores must be finite and > 0. */
void or_set_edge_scores(or_state* st, const double* score) {
    int n = st->p.n, k = st->p.k;
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < k; ++r)
            st->etab[(size_t)i * k + r] =
                score ? score[(size_t)i * k + r] : eta_pow(st->xy, i, st->cand[(size_t)i * k + r], st->p.beta);
}

/* The new tour of ant a built elsewhere (a colony split over processes by ants): l_best layout,
 * its length, and whether it was a partial rebuild (s >= 0, M rebuilt cities) or a full tour. */
void or_set_newtour(or_state* st, int a, const int32_t* tour, double len, int s, int M) {
    memcpy(st->newtour + (size_t)a * st->p.n, tour, sizeof(int32_t) * (size_t)st->p.n);
    st->newlen[a] = len;
    st->seg_s[a] = s;
    st->seg_M[a] = M;
    st->built[a] = 1;
}

/* Forget which ants were built (before the tours of another process's ants are set). */
void or_clear_built(or_state* st) { memset(st->built, 0, sizeof(int32_t) * (size_t)st->p.m); }

/* Replace the l_best population (checkpoint restore / teacher forcing). */
void or_set_lbest(or_state* st, const int32_t* lbest, const double* clen) {
    memcpy(st->lbest, lbest, sizeof(int32_t) * (size_t)st->p.m * st->p.n);
    memcpy(st->clen, clen, sizeof(double) * (size_t)st->p.m);
    st->initialized = 1;
}

/* Eq. 1 probabilities at city i for the unvisited set `visited` (1 = visited).
 * Dense mode: out has n entries (0 for visited).  Candidate mode: out has k entries over the
 * candidate list (0 for visited candidates); returns 0 if some candidate is unvisited, else 1
 * (the list is exhausted and the ant takes the fallback). */
int or_step_probs(or_state* st, int i, const unsigned char* visited, double* out) {
    int n = st->p.n;
    if (st->p.mode == 0) {
        double total = 0.0;
        for (int j = 0; j < n; ++j) {
            out[j] = visited[j] ? 0.0 : or_powr(st->tau[(size_t)i * n + j], st->p.alpha) * st->etab_d[(size_t)i * n + j];
            total += out[j];
        }
        for (int j = 0; j < n; ++j) out[j] = out[j] / total;
        return 0;
    }
    lbest_pheromone(st);
    int k = st->p.k;
    double total = 0.0;
    for (int r = 0; r < k; ++r) {
        int j = st->cand[(size_t)i * k + r];
        out[r] = visited[j] ? 0.0 : or_powr(tau_from_Q(st, st->Q[(size_t)i * k + r]), st->p.alpha) * st->etab[(size_t)i * k + r];
        total += out[r];
    }
    if (total == 0.0) return 1;
    for (int r = 0; r < k; ++r) out[r] = out[r] / total;
    return 0;
}

/* The exhausted-list rule (Section 6's fallback to the ordinary rule, with the Section 3
 * pheromone of the l_best population) at city i for the unvisited set `visited` (1 = visited)
 * and the draw u (used by fallback 1): the city picked, exactly as a construction picks it.
 * w_out (n entries, may be NULL): the weight of every unvisited city, 0 for visited ones. */
int or_exhausted_step(or_state* st, int i, const unsigned char* visited, double u, double* w_out) {
    if (st->p.mode != 1) return -1;
    lbest_pheromone(st);
    int n = st->p.n;
    memcpy(st->visited, visited, (size_t)n);
    if (w_out)
        for (int j = 0; j < n; ++j) w_out[j] = visited[j] ? 0.0 : any_weight(st, i, j);
    return exhausted_pick(st, i, u);
}

/* ------------------------------------------------------------------ large-n helpers */
/* Candidate list of one city by brute force (the definition), for sampled checks at large n. */
void or_knn_one(int n, const double* xy, int k, int i, int32_t* row) {
    double kd[64];
    int filled = 0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double d2 = or_dist2(xy, i, j);
        if (filled == k && !(d2 < kd[k - 1])) continue;
        int pos = filled < k ? filled : k - 1;
        while (pos > 0 && d2 < kd[pos - 1]) {
            kd[pos] = kd[pos - 1];
            row[pos] = row[pos - 1];
            --pos;
        }
        kd[pos] = d2;
        row[pos] = j;
        if (filled < k) ++filled;
    }
}

/* The same lists by an x-sweep: cities sorted by x; from each city scan outwards in x order and
 * stop a direction once dx*dx exceeds the k-th best d^2 (d^2 >= dx*dx, so nothing further can
 * enter).  Keys (d^2, j) as in or_knn; results identical.  O(n log n + n * slab). */
static const double* g_sort_xy;
static int cmp_x(const void* a, const void* b) {
    int ia = *(const int*)a, ib = *(const int*)b;
    double xa = g_sort_xy[2 * ia], xb = g_sort_xy[2 * ib];
    if (xa < xb) return -1;
    if (xa > xb) return 1;
    return ia < ib ? -1 : (ia > ib);
}

static void keep_best(double* kd, int32_t* row, int* filled, int k, double d2, int j) {
    if (*filled == k && !(d2 < kd[k - 1] || (d2 == kd[k - 1] && j < row[k - 1]))) return;
    int pos = *filled < k ? *filled : k - 1;
    while (pos > 0 && (d2 < kd[pos - 1] || (d2 == kd[pos - 1] && j < row[pos - 1]))) {
        kd[pos] = kd[pos - 1];
        row[pos] = row[pos - 1];
        --pos;
    }
    kd[pos] = d2;
    row[pos] = j;
    if (*filled < k) ++*filled;
}

int or_knn_sweep(int n, const double* xy, int k, int32_t* cand) {
    int* order = (int*)malloc(sizeof(int) * (size_t)n);
    int* where = (int*)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    g_sort_xy = xy;
    qsort(order, (size_t)n, sizeof(int), cmp_x);
    for (int p = 0; p < n; ++p) where[order[p]] = p;
    int dup = 0;
    double kd[64];
    for (int i = 0; i < n; ++i) {
        int32_t* row = cand + (size_t)i * k;
        int filled = 0;
        int p0 = where[i];
        for (int dir = -1; dir <= 1; dir += 2) {
            for (int p = p0 + dir; p >= 0 && p < n; p += dir) {
                int j = order[p];
                double dx = xy[2 * i] - xy[2 * j];
                if (filled == k && dx * dx > kd[k - 1]) break;
                double d2 = or_dist2(xy, i, j);
                if (d2 == 0.0) dup = 1;
                keep_best(kd, row, &filled, k, d2, j);
            }
        }
    }
    free(order);
    free(where);
    return dup ? -1 : 0;
}

/* l_best-mode state from given candidate lists (skips the O(n^2) brute force at large n). */
or_state* or_create_with_cand(const or_params* p, const double* xy, const int32_t* cand) {
    if (p->mode != 1) return NULL;
    if (p->n < 3 || p->m < 1 || p->k < 1 || p->k > 32 || p->k > p->n - 1) return NULL;
    or_state* st = (or_state*)calloc(1, sizeof(or_state));
    st->p = *p;
    int n = p->n, m = p->m, k = p->k;
    st->xy = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    memcpy(st->xy, xy, sizeof(double) * 2 * (size_t)n);
    st->visited = (unsigned char*)malloc((size_t)n);
    st->newtour = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
    st->newlen = (double*)malloc(sizeof(double) * (size_t)m);
    st->built = (int32_t*)calloc((size_t)m, sizeof(int32_t));
    st->seg_s = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    st->seg_M = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    st->cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * k);
    memcpy(st->cand, cand, sizeof(int32_t) * (size_t)n * k);
    st->etab = (double*)malloc(sizeof(double) * (size_t)n * k);
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < k; ++r)
            st->etab[(size_t)i * k + r] = eta_pow(st->xy, i, st->cand[(size_t)i * k + r], p->beta);
    st->lbest = (int32_t*)calloc((size_t)m * n, sizeof(int32_t));
    st->clen = (double*)malloc(sizeof(double) * (size_t)m);
    for (int a = 0; a < m; ++a) st->clen[a] = INFINITY;
    st->q = (uint64_t*)calloc((size_t)m, sizeof(uint64_t));
    st->Q = (uint64_t*)calloc((size_t)n * k, sizeof(uint64_t));
    st->succ = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
    st->pred = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
    return st;
}

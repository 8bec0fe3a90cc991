/*
 * aco.h -- C ABI of the GB300 (sm_103a) ACO library for the symmetric Euclidean TSP.
 *
 * The library implements the data-parallel hot path of D. M. Chitty, "Applying ACO To Large
 * Scale TSP Instances" (UKCI 2017): tour construction by the random proportional rule
 * (Section 2, Eq. 1), the pheromone update -- evaporation and deposit (Section 2, Eq. 2-5) in
 * the dense form, and the per-ant l_best pheromone source of Section 3 with the PartialACO
 * efficiency measure (Section 3.1, Algorithm 1) in the scalable form -- and the tour-length
 * reduction.  Candidate lists of the k nearest cities (the Ant Colony System device cited in
 * Section 6) restrict each decision in the scalable form.
 *
 * Conventions (every entry point):
 *  - Pointers named *_dev are CUDA device pointers on the instance's device; *_host are host
 *    pointers.  The caller owns every buffer it passes; the library copies what it keeps.
 *  - A device buffer is aligned to its element type (4 bytes for int32, float and BF16 pairs, 8
 *    for FP64; the feature matrix of aco_edge_features 16); a misaligned one gives
 *    ACO_ERR_INVALID_ARG before anything is enqueued.
 *  - All work is enqueued on the instance's stream.  Only the calls documented as
 *    synchronising wait for the device.
 *  - All device memory is allocated by aco_create_instance; no later call allocates.
 *  - No call aborts or throws.  Errors are returned as aco_status; aco_last_error() gives a
 *    message.  A device-side error (e.g. coincident cities) is reported by the next
 *    synchronising call.
 *  - An instance is not thread-safe: one host thread at a time.
 */
#ifndef ACO_H
#define ACO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aco_status {
    ACO_OK = 0,
    ACO_ERR_INVALID_ARG = 1, /* bad size, parameter or pointer; coincident cities          */
    ACO_ERR_OOM = 2,         /* device allocation failed in aco_create_instance             */
    ACO_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed                 */
    ACO_ERR_STATE = 4,       /* call out of order (e.g. construct before build_candidates) */
    ACO_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up                          */
} aco_status;

typedef enum aco_mode {
    ACO_MODE_DENSE = 0,         /* Section 2: n x n FP64 pheromone, Eq. 1 over all unvisited */
    ACO_MODE_LBEST_PARTIAL = 1  /* Section 3 + Algorithm 1: l_best pheromone, PartialACO    */
} aco_mode;

/* Parameters of one colony (Section 2-3 notation). */
typedef struct aco_params {
    int32_t mode;         /* aco_mode                                                        */
    int32_t n;            /* cities, >= 3                                                    */
    int32_t m;            /* ants, >= 1                                                      */
    int32_t k;            /* candidate-list length, 1..min(32, n-1) (ignored in DENSE)       */
    double alpha;         /* pheromone exponent of Eq. 1                                     */
    double beta;          /* heuristic exponent of Eq. 1 (eta = 1/d); > 0 with candidate lists */
    double rho;           /* evaporation rate of Eq. 2 (DENSE only; the Section 3 form has
                             no evaporation matrix)                                          */
    double tau0;          /* initial / base pheromone, > 0                                   */
    double max_mod_frac;  /* f: at most floor(f n) cities are rebuilt (Section 3.1), (0, 1]  */
    double p_partial;     /* probability of a partial (vs full) rebuild per ant, [0, 1]      */
    uint64_t seed;        /* Philox4x32-10 key                                               */
    int32_t fallback;     /* exhausted list: 0 = argmax tau^a eta^b over unvisited (ties to the
                             lowest index), 1 = Eq. 1 over all unvisited                    */
    int32_t selection;    /* decision rule on the candidate list (LBEST only; DENSE needs 0):
                             0 = the Eq. 1 random proportional wheel;
                             1 = Independent Roulette (Section 3): argmax over unvisited
                             candidates with positive weight of tau^a eta^b * u_r, ties to the
                             lowest rank, u_r = (x + 1/2) 2^-32 from word r % 4 of the Philox
                             draw with counter (8 t + r / 4, ant, iteration, 4) at decision t;
                             no such candidate: the exhausted-list rule (fallback)           */
} aco_params;

/* Counters accumulated since creation (aco_get_stats). */
typedef struct aco_stats {
    uint64_t decisions;      /* cities chosen by Eq. 1 or the exhausted-list rule            */
    uint64_t fallbacks;      /* decisions taken by the exhausted-list rule                   */
    uint64_t exact_resolves; /* decisions re-evaluated in FP64 (FP32 screen inconclusive)    */
    uint64_t improved;       /* l_best replacements (Algorithm 1) / tours deposited (DENSE)  */
    uint64_t partial_ants;   /* partial rebuilds                                             */
    uint64_t full_ants;      /* full constructions                                           */
    double gbest;            /* length of the best tour so far (C_gbest), +inf if none       */
    int32_t gbest_ant;       /* ant holding it (lowest index among equals), -1 if none       */
    int32_t iterations;      /* completed construct + update pairs                           */
    uint64_t ls_moves;       /* 2-opt moves made by the local search                         */
    uint64_t fallback_rebuilt; /* sum over exhausted-list steps of the ant's rebuilt count M
                                  (n - 1 for a full construction)                            */
    uint64_t fallback_scanned; /* sum over exhausted-list steps of the remaining cities listed
                                  for the step (before the visited ones drop out)             */
    uint64_t fallback_fast;  /* exhausted-list steps whose nearest unvisited city was found among
                                the city's 32 nearest cities (no scan of the remaining ones)  */
} aco_stats;

typedef struct aco_instance aco_instance; /* opaque: owns all device state of one colony */

/* Create a colony on the current CUDA device.  xy_dev: n*2 FP64 coordinates (x0,y0,x1,...),
 * copied.  stream: cudaStream_t to enqueue on (NULL = the legacy default stream).  Checks the
 * parameters and that the coordinates are finite with bounding box * n < 2^30 (exact length
 * accumulation range).  Allocates every device buffer the instance will use.  Synchronises.
 * Problem statement: Section 2 (G = (V, E, d), d_ij = d_ji); parameters: Section 2-3. */
aco_status aco_create_instance(const double* xy_dev, const aco_params* p, void* stream,
                               aco_instance** out);

/* Build the candidate lists: for every city the k nearest other cities, key (d^2, index)
 * ascending with d^2 = dx*dx + dy*dy in FP64 (exact ACS-style candidate lists, Section 6), and
 * the heuristic table eta^beta of every candidate edge (Section 2).  Also initialises the
 * Eq. 1 weights to tau0^alpha eta^beta.  cand_out_dev: optional n*k int32 copy of the lists.
 * In DENSE mode builds the n x n eta^beta table and sets tau = tau0.  Synchronises; returns
 * ACO_ERR_INVALID_ARG if two cities coincide (eta = 1/d undefined). */
aco_status aco_build_candidates(aco_instance* inst, int32_t* cand_out_dev);

/* Tour construction for every ant (Section 2, Eq. 1; Algorithm 1).
 * DENSE: each ant starts at a random city and applies Eq. 1 over all unvisited cities.
 * LBEST: the first call builds full initial tours (Algorithm 1, before its iterations; tau = tau0).  Later
 * calls rebuild, per ant, a random contiguous part of at most floor(f n) cities of l_best
 * (with probability p_partial; otherwise a full tour), using Eq. 1 over the unvisited
 * candidates and the exhausted-list rule.  `iteration` keys the Philox draws (callers pass
 * 0, 1, 2, ...).  tours_out_dev: optional m*n int32 copy of the new tours (l_best layout);
 * len_out_dev: optional m FP64 lengths.  Needs aco_build_candidates first (ACO_ERR_STATE). */
aco_status aco_construct_tours(aco_instance* inst, int32_t iteration, int32_t* tours_out_dev,
                               double* len_out_dev);

/* Pheromone update after aco_construct_tours.
 * DENSE: Eq. 2 (tau <- (1 - rho) tau on every edge) then Eq. 3-5 (tau_ij += sum_k 1/C^k over
 * the tours containing edge (i,j), both directions).
 * LBEST: Algorithm 1 (an ant's l_best is replaced by its new tour when strictly
 * shorter), C_gbest = min C_lbest, then the Section 3 pheromone of every candidate edge,
 * tau_ij = tau0 + sum_a (C_gbest / C_a) [ (i,j) in l_best_a ] -- edges of replaced tours drop
 * out (evaporation) and edges of new l_best tours enter (deposit). */
aco_status aco_update_pheromone(aco_instance* inst);

/* Tour-length reduction: out_dev[c] = sum of the n edge lengths of tours_dev[c*n ..] including
 * the closing edge (Section 2), for c < count.  Exact: every edge on a 2^-96 grid, integer
 * sum, one rounding to FP64 (order-free).  Tours must be permutations of 0..n-1 (not checked
 * beyond index range; out-of-range indices give ACO_ERR_INVALID_ARG at the next
 * synchronising call). */
aco_status aco_tour_lengths(aco_instance* inst, const int32_t* tours_dev, int32_t count,
                            double* out_dev);

/* Checkpoint (Section 3 state): lbest_out_dev m*n int32 l_best tours, clen_out_dev m FP64
 * lengths; tau_out_dev n*n FP64 (DENSE only, else may be NULL).  Any pointer may be NULL.
 * Synchronises. */
aco_status aco_get_state(aco_instance* inst, int32_t* lbest_out_dev, double* clen_out_dev,
                         double* tau_out_dev);

/* Restore a checkpoint (LBEST: l_best tours, lengths recomputed exactly; DENSE: tau).
 * Philox draws are counter-based, so resuming at iteration t reproduces an uninterrupted run.
 * Synchronises. */
aco_status aco_set_state(aco_instance* inst, const int32_t* lbest_dev, const double* tau_dev);

/* Counters since creation; synchronises and reports pending device-side errors. */
aco_status aco_get_stats(aco_instance* inst, aco_stats* out_host);

/* Eq. 1 probabilities as the construction kernel sees them (FP32 weights, FP32 normaliser)
 * at city `city` for the visited bitset visited_bits_dev (ceil(n/32) uint32 words, bit j of
 * word j/32 set = visited).  probs_out_dev: k floats (LBEST, candidate ranks) or n floats
 * (DENSE).  *exhausted_out_dev = 1 when no candidate is unvisited (LBEST).  Diagnostic. */
aco_status aco_step_probs(aco_instance* inst, int32_t city, const uint32_t* visited_bits_dev,
                          float* probs_out_dev, int32_t* exhausted_out_dev);

/* Run-time schedule of the PartialACO parameters (Section 3.1; a growing f is the schedule the
 * paper proposes as future work in Section 7): from the next aco_construct_tours on, at most
 * floor(f n) cities are rebuilt, and an ant rebuilds partially with probability p_partial.
 * 0 < f <= the max_mod_frac given at creation (the per-ant lists are sized for it), 0 <= p_partial
 * <= 1; LBEST mode; not between construct and update (ACO_ERR_STATE).  Host-side only. */
aco_status aco_set_max_mod_frac(aco_instance* inst, double f);
aco_status aco_set_p_partial(aco_instance* inst, double p_partial);

/* Local search on constructed tours (Section 3.2: 2-opt applied to a tour with a given
 * probability, 0.001 in the paper; Section 5: only edges within `window` tour positions, 500 in
 * the paper).  From the next aco_construct_tours on, each ant (index order, at most 8 per
 * iteration) whose Philox draw (0, ant, iteration, 5) gives u < p applies windowed 2-opt to its new
 * tour: passes over position blocks 0, off, off + 2W, ..., n (off alternating 0 and W), each block
 * scanned first-improvement (i ascending, j = i + 2 .. i + W ascending) with FP64 gains
 * (d(a,b) + d(c,d)) - (d(a,c) + d(b,d)) > 0, until two passes in a row make no move (at most 16).
 * The tour is then committed as a whole if strictly shorter than l_best.  p in [0, 1] (0 = off,
 * the default), 2 <= window <= 4096.  LBEST mode, single colony; not between construct and
 * update.  The first call with p > 0 allocates the working tours (8 n int32). */
aco_status aco_set_local_search(aco_instance* inst, double p, int32_t window);

/* Asynchronous l_best sharing (Section 3: the paper's CPU colony runs its ants asynchronously, so
 * an ant's improved l_best, and the pheromone it implies, reach ants that are still building).
 * on = 1: from the next aco_construct_tours on, an ant whose partial rebuild is strictly shorter
 * than its l_best commits it inside the construction launch: the rebuilt l_best positions, the
 * neighbour entries of the cities they touch, the integer pheromone of those entries' candidate
 * edges (the ant keeps its deposit weight q_a of the iteration start) and the Eq. 1 weights of
 * the touched cities' candidate rows.  Ants still building read whatever value each entry holds
 * at the time (old or new).  Full constructions commit in aco_update_pheromone as before, and
 * the update recomputes every weight from C_gbest, so the state after each update is the usual
 * function of the l_best population; the tours depend on timing, so runs are not reproducible
 * and have no oracle counterpart.  on = 0 (default) restores the synchronous iteration.
 * LBEST mode, single colony (not an instance of a batch), local search off (ACO_ERR_STATE
 * otherwise); not between construct and update.  The first call with on = 1 allocates the
 * pheromone table (8 n k bytes) and fills it from the current l_best population (synchronises). */
aco_status aco_set_async_share(aco_instance* inst, int32_t on);

/* ------------------------------------------------------------------ one colony over several GPUs
 * Section 3's colony draws its pheromone from every ant's l_best, and within an iteration the
 * ants only read it (synchronous reading): the ants can be split over GPUs.  Every rank creates
 * the same instance (same coordinates and parameters) and keeps the whole colony state; it
 * constructs its own range of ants, exports the commits of its ants that improved, receives
 * every rank's records (e.g. by an all-gather), imports them and runs aco_update_pheromone.  A
 * commit touches only its own ant's l_best and neighbour entries and the pheromone sums are exact
 * integers, so each rank's state after the update equals the single colony's bit for bit.
 *
 * Records (int32 words): word 0 the number of records, word 1 zero, words 2-3 the words used (an
 * int64 counting these four), then per record: ant, s, P, M, start, L (segment length: M for a
 * partial rebuild, n for a full construction), new length (2 words, FP64 bits, low word first),
 * exact length (4 words: the 128-bit fixed-point value, low 64 bits first), then L city indices.
 * The first construction builds full tours (n cities per record). */

/* The ants this instance constructs: [ant_begin, ant_end) (default: all).  LBEST mode, not for an
 * instance of a batch, and not with local search or asynchronous sharing unless the range is the
 * whole colony (ACO_ERR_STATE).  Not between construct and update. */
aco_status aco_set_ant_range(aco_instance* inst, int32_t ant_begin, int32_t ant_end);
/* After aco_construct_tours: writes the records of the instance's own ants whose new tour is
 * strictly shorter than their l_best into buf_dev (cap_words int32 words, 8-byte aligned), in any
 * order.  *words_out = the words used (also when they exceed cap_words: then nothing usable is
 * written and ACO_ERR_INVALID_ARG is returned).  At most (ant_end - ant_begin) (12 + n) + 4 words.
 * Synchronises. */
aco_status aco_export_commits(aco_instance* inst, int32_t* buf_dev, int64_t cap_words, int64_t* words_out);
/* Before aco_update_pheromone: the records of `count` buffers laid out stride_words apart
 * (8-byte aligned, stride even), typically every rank's export; records of the instance's own
 * ants are skipped.  Ants outside the own range that have no record commit nothing this
 * iteration.  A malformed record gives ACO_ERR_INVALID_ARG at the next synchronising call.
 * Enqueued. */
aco_status aco_import_commits(aco_instance* inst, const int32_t* bufs_dev, int32_t count, int64_t stride_words);

/* ------------------------------------------------------------------ batched colonies
 * Many independent instances of uneven size solved together: the same method and parameters
 * per instance (Section 3, Algorithm 1), with all of a batch's colonies advanced by single
 * launches per step, iterations replayed as a captured CUDA graph, and the launch schedule
 * (ants per block) chosen by timing live iterations.  Results equal running every instance
 * alone with the single-colony calls above. */
typedef struct aco_batch aco_batch; /* opaque */

/* xy_dev: the instances' coordinates concatenated (sum n_i rows of 2 FP64); n_host: count sizes.
 * p: shared parameters (mode must be ACO_MODE_LBEST_PARTIAL; p->n is ignored; instance i gets
 * m_i = min(n_i, p->m) ants and seed p->seed + i).  stream: cudaStream_t for all of the batch's
 * work; NULL makes the batch create its own non-blocking stream (iterations are captured as a
 * CUDA graph, which the legacy default stream cannot be).  Allocates everything.  Synchronises. */
aco_status aco_batch_create(const double* xy_dev, const int32_t* n_host, int32_t count, const aco_params* p,
                            void* stream, aco_batch** out);
/* Candidate lists and eta^beta tables of every instance (as aco_build_candidates).  Synchronises. */
aco_status aco_batch_build_candidates(aco_batch* b);
/* Launch schedules of a batch: 0 .. 7 run an iteration as four launches over every colony
 * (construct, commit, C_gbest and weights, pheromone rebuild) replayed as a CUDA graph, with 1-4
 * ants per block and a register cap; 8 .. 11 run all iterations of a call in ONE persistent
 * cooperative launch whose resident warps pull (instance, ant) slots and city chunks from device
 * work queues, with grid-wide barriers between the phases (warps per block, register cap and
 * ants per pull vary).  Every schedule gives the same results. */
#define ACO_BATCH_SCHEDULES 12

/* `iterations` iterations of every colony, keyed first_iteration, first_iteration + 1, ...  The
 * first call builds the initial tours in its first iteration.  tune != 0 (and no schedule set by
 * aco_batch_set_schedule): the first iterations of the first tuned call (one per schedule, up to
 * twelve) are timed with every schedule and the fastest is kept.  Enqueued on the batch's stream.
 * A persistent launch whose barrier wait runs out (aco_batch_set_wait_limit) ends early; the next
 * aco_batch_get_state / aco_batch_get_best returns ACO_ERR_TIMEOUT and the batch cannot run any
 * more (ACO_ERR_STATE). */
aco_status aco_batch_run(aco_batch* b, int32_t first_iteration, int32_t iterations, int32_t tune);
/* l_best tours (instance i at offset sum_{j<i} m_j n_j, row-major m_i x n_i) and lengths
 * (offset sum_{j<i} m_j); either pointer may be NULL.  Synchronises. */
aco_status aco_batch_get_state(aco_batch* b, int32_t* lbest_out_dev, double* clen_out_dev);
/* C_gbest of every instance (count doubles).  Synchronises. */
aco_status aco_batch_get_best(aco_batch* b, double* best_len_host);
/* The schedule in use (0 .. ACO_BATCH_SCHEDULES - 1), its warps per block and minimum resident
 * blocks per SM, its ants per pull (0 for the four-launch schedules), and the tuning times
 * (ACO_BATCH_SCHEDULES floats, ms per iteration; 0 where not tuned).  Any pointer may be NULL. */
aco_status aco_batch_schedule(const aco_batch* b, int32_t* schedule_out, int32_t* warps_out,
                              int32_t* min_blocks_out, int32_t* ants_per_pull_out, float* tune_ms_out);
/* Fix the schedule (0 .. ACO_BATCH_SCHEDULES - 1) for every later call, tuning off; -1 gives the
 * choice back to the autotuner.  Host-side only. */
aco_status aco_batch_set_schedule(aco_batch* b, int32_t schedule);
/* The longest a warp of a persistent launch waits at one of its grid-wide barriers (default
 * 10 s; 0 <= seconds <= 3600; 0 gives up at once, which makes a launch of more than one block
 * end with ACO_ERR_TIMEOUT).  Host-side only. */
aco_status aco_batch_set_wait_limit(aco_batch* b, double seconds);
const char* aco_batch_last_error(const aco_batch* b);
void aco_batch_destroy(aco_batch* b);

/* Candidate lists (the same exact lists as aco_build_candidates) for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a deployment variant of the library.
 * The working memory is a fixed array inside the library (1,966,080 bytes per GPU, held until the
 * process exits); the caller passes only its input and output buffers, and nothing is allocated.
 * xy_dev: n*2 FP64 device coordinates; cand_out_dev: n*k int32 device output (row i = the k
 * nearest other cities of city i, key (d^2, index) ascending).  n <= 65536 (larger n returns
 * ACO_ERR_INVALID_ARG), 1 <= k <= min(32, n-1).  The first call on a device (and the first after
 * the device's context was reset) looks up the array's device address.  All calls share the array
 * and it keeps the last call's contents; calls that overlap on the GPU race and must be serialised
 * by the caller.  Synchronises the stream, so it cannot be captured in a CUDA graph: on a stream
 * that is capturing it returns ACO_ERR_INVALID_ARG and enqueues nothing.  Coincident or non-finite
 * cities give ACO_ERR_INVALID_ARG. */
aco_status aco_build_candidates_noalloc(const double* xy_dev, int32_t n, int32_t k, int32_t* cand_out_dev,
                                        void* stream);

/* A borrowed handle of instance i of a batch (valid until aco_batch_destroy), for the calls that
 * read or retune one colony: aco_get_state, aco_get_stats, aco_edge_features, aco_tour_labels,
 * aco_set_edge_scores.  Its work goes to the batch's stream.  Advancing it with
 * aco_construct_tours / aco_update_pheromone is not supported while it belongs to a batch. */
aco_status aco_batch_instance(aco_batch* b, int32_t i, aco_instance** out);

/* ------------------------------------------------------------------ learned edge proposal
 * An extension of the method, not in the paper: a small network scores every candidate edge
 * (i, cand[i][r]) and the score stands in for eta_ij^beta of Eq. 1 (Section 2) on candidate
 * edges; edges outside the candidate lists (the exhausted-list rule) keep eta^beta, and NULL
 * scores restore the plain heuristic everywhere.
 *
 * Features (one row of 16 BF16 values per candidate edge, rows in (city, rank) order), with
 * j = cand[i][r] and dbar_i the mean distance from i to its k candidates:
 *   x0 = d_ij / dbar_i, x1 = r / (k - 1), x2 = (x_j - x_i) / dbar_i, x3 = (y_j - y_i) / dbar_i,
 *   x4 = deg_j / 32 (deg_j = distinct neighbours of j in the l_best tours of ants 0 .. D-1),
 *   x5 = 1, x6 .. x15 = 0.
 * Network (weights as one FP32 vector of ACO_MLP_WEIGHTS entries: W1 [64][16], W2 [64][64],
 * w3 [64], row-major, used as BF16; products accumulate in FP32 on the tensor cores):
 *   h1 = relu(W1 x) with h1[63] = 1;  h2 = relu(W2 h1) with h2[63] = 1;  z = w3 . h2;
 *   score = exp(min(max(beta z, -60), 60)): exp(z) is the learned counterpart of eta, raised to
 *   the same exponent beta as eta in Eq. 1.
 * Training target: per city, the softmax of z over its k candidate edges against the
 * candidate ranks that are its neighbours in a best tour (a bitmask per city; cities without
 * such a rank are left out); cross-entropy loss, Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the
 * FP32 weights.  W1's row 63 and columns 6..15 and W2's row 63 are held at zero. */
#define ACO_MLP_WEIGHTS (64 * 16 + 64 * 64 + 64)
typedef struct aco_mlp aco_mlp; /* opaque: weights, optimiser state and training scratch */

/* w_host: ACO_MLP_WEIGHTS initial FP32 weights (finite).  max_rows: the most candidate-edge rows
 * one aco_mlp_backward call or one aco_mlp_train batch may hold (16 .. 2^30; about 350 bytes of
 * device memory per row).  stream: cudaStream_t for all of this network's work (NULL = legacy
 * default stream).  Allocates everything.  Synchronises. */
aco_status aco_mlp_create(const float* w_host, int64_t max_rows, void* stream, aco_mlp** out);
/* The FP32 weights (ACO_MLP_WEIGHTS floats).  Synchronises.  ACO_ERR_TIMEOUT if a forward or
 * backward pass on this handle gave up waiting for a tensor-core MMA (2 s; its unfinished rows or
 * gradient blocks were written NaN). */
aco_status aco_mlp_get_weights(aco_mlp* h, float* w_host);
/* z_dev and/or score_dev = exp(beta z) (rows floats each; either may be NULL, not both) for rows of
 * BF16 features X_dev (rows * 16 BF16 bit patterns).  No row limit.  On the tcgen05
 * tensor cores: 128-row tiles, accumulators in tensor memory.  Enqueued. */
aco_status aco_mlp_forward(aco_mlp* h, const uint16_t* X_dev, int64_t rows, float* z_dev, float* score_dev,
                           float beta);
/* Gradient of scale * (summed loss over `cities` cities of k rows each, k <= 32) with respect to
 * the weights into grad_dev (ACO_MLP_WEIGHTS floats, may be NULL: then kept inside for
 * aco_mlp_adam) and the scaled loss into loss_dev[0] (may be NULL).  cities * k <= max_rows.
 * Deterministic (fixed-order reductions).  Enqueued. */
aco_status aco_mlp_backward(aco_mlp* h, const uint16_t* X_dev, const uint32_t* target_dev, int32_t cities,
                            int32_t k, float scale, float* grad_dev, float* loss_dev);
/* One Adam step with grad_dev (NULL = the gradient the last aco_mlp_backward kept) and learning
 * rate lr >= 0.  Enqueued. */
aco_status aco_mlp_adam(aco_mlp* h, const float* grad_dev, float lr);
/* `steps` training steps over the data in order, batch_cities cities (batch_cities * k <= max_rows)
 * per step, wrapping around: backward with scale 1 / (cities in the step), then Adam.  Mean loss
 * of step t into loss_dev[t] (may be NULL).  Enqueued. */
aco_status aco_mlp_train(aco_mlp* h, const uint16_t* X_dev, const uint32_t* target_dev, int32_t cities, int32_t k,
                         int32_t batch_cities, int32_t steps, float lr, float* loss_dev);
const char* aco_mlp_last_error(const aco_mlp* h);
void aco_mlp_destroy(aco_mlp* h);

/* Features of the instance's candidate edges into X_dev (n * k * 16 BF16), with the degree count
 * over the l_best tours of ants 0 .. degree_ants-1 (1 <= degree_ants <= min(m, 16)).  Needs
 * candidate lists and l_best tours (ACO_ERR_STATE otherwise).  Enqueued. */
aco_status aco_edge_features(aco_instance* inst, int32_t degree_ants, uint16_t* X_dev);
/* Per city (n uint32) the bitmask of candidate ranks holding its two neighbours in the best
 * l_best tour (length C_gbest).  Needs l_best tours and k <= 32.  Enqueued. */
aco_status aco_tour_labels(aco_instance* inst, uint32_t* target_dev);
/* score_dev: n * k FP32 scores (finite, > 0) that replace eta^beta on the candidate edges from
 * now on (until the next aco_build_candidates), or NULL to restore eta^beta.  The Eq. 1 weights
 * are recomputed at once.  Not between aco_construct_tours and aco_update_pheromone
 * (ACO_ERR_STATE).  Synchronises when score_dev is given (a non-finite or non-positive score
 * gives ACO_ERR_INVALID_ARG and leaves the scores in use unchanged). */
aco_status aco_set_edge_scores(aco_instance* inst, const float* score_dev);

/* Bandwidth probe (a measurement aid, not part of the method): the roofline of the construction
 * kernel, whose working set sits in L2, needs the L2 bandwidth, which this measures on the caller's
 * buffer.  buf_dev: `bytes` bytes of device memory (16-byte aligned, bytes a multiple of 32 and
 * >= 4096; contents are read and, in mode 1, overwritten).  mode 0: one launch of reps passes that
 * read the buffer (after its first 16 bytes) with 16-byte loads cached in L2 only; mode 1: one
 * launch of reps passes that copy its first half to its second half.  One untimed pass first;
 * *ms_out = the device time of the timed launch (CUDA events on `stream`).  Changes no device
 * setting.  Synchronises. */
aco_status aco_probe_bandwidth(void* buf_dev, int64_t bytes, int32_t mode, int32_t reps, void* stream,
                               float* ms_out);

void aco_destroy_instance(aco_instance* inst);
const char* aco_status_string(aco_status s);
const char* aco_last_error(const aco_instance* inst);

#ifdef __cplusplus
}
#endif
#endif /* ACO_H */

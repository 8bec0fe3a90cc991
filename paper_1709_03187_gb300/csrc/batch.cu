// batch.cu -- many independent colonies of uneven size in single launches.
//
// A batch owns one colony per instance (same parameters, n_i cities, m_i = min(n_i, m) ants,
// seed + i).  Each iteration is four launches over every colony at once:
//   construction (ant slots ordered longest instance first; `warps` ants per block),
//   commit (one block per ant slot), C_gbest and weights (one block per colony),
//   pheromone rebuild (block map over every colony's cities),
// plus a one-thread increment of the device iteration counter, captured once as a CUDA graph and
// replayed -- or all iterations of a call in one persistent cooperative launch (construct_persist.cu:
// work queues of ant slots and city chunks, grid-wide barriers with bounded waits).  The schedule
// does not change any result (each ant's work is deterministic), so the autotuner times live
// iterations with each schedule -- for the four launches, ants per block and a register cap
// (minimum resident blocks per SM); for the persistent launch, warps per block, register cap and
// ant slots per pull -- and keeps the fastest.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"

struct LbestArgs;  // defined in construct_dev.cuh
void fill_lbest_args(const aco_instance* inst, int32_t iteration, LbestArgs& A);
size_t construct_smem_per_ant(int n, int k);
cudaError_t launch_construct_batch(const LbestArgs* args, const int2* slot, const int* iteration, int slots,
                                   int smem_per_ant, int config, cudaStream_t s);
extern const int kBatchConfigs[ACO_BATCH_CONFIGS][2];
void fill_commit_args(const aco_instance* inst, CommitArgs& C);
void fill_gbest_args(const aco_instance* inst, int keep_prev, GbestArgs& G);
void fill_rebuild_args(const aco_instance* inst, int use_ants, RebuildArgs& R);
cudaError_t launch_update_batch(const CommitArgs* cargs, const int2* slot, int slots, const GbestArgs* gargs,
                                int count, const RebuildArgs* rargs, const int4* blockmap, int rblocks, int m_cap,
                                int k, cudaStream_t s);
size_t lbest_args_size();
void fill_lbest_args_bytes(const aco_instance* inst, int32_t iteration, void* out);
cudaError_t launch_persistent_batch(PersistArgs P, int config, int num_sms, cudaStream_t s, int* grid_out);
extern const int kPersistConfigs[ACO_PERSIST_CONFIGS][3];

#define ACO_ALL_SCHEDULES (ACO_BATCH_CONFIGS + ACO_PERSIST_CONFIGS)

__global__ void bump_iteration_kernel(int* it) { *it += 1; }


struct aco_batch {
    int count = 0;
    aco_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // created by the batch (the caller passed NULL)
    std::vector<aco_instance*> inst;
    std::vector<int> n_i, m_i;
    std::vector<long long> city_off, ant_off, tour_off;
    void* d_largs = nullptr;  // LbestArgs[count]
    CommitArgs* d_cargs = nullptr;
    GbestArgs* d_gargs = nullptr;
    RebuildArgs* d_rargs = nullptr;
    int2* d_slot = nullptr;
    int4* d_rmap = nullptr;
    int* d_iter = nullptr;
    int slots = 0, rblocks = 0, smem_per_ant = 0, m_cap = 0;
    // schedule: 0 .. ACO_BATCH_CONFIGS-1 = four launches per iteration (kBatchConfigs), replayed
    // as a CUDA graph; ACO_BATCH_CONFIGS + c = one persistent launch (kPersistConfigs[c])
    int config = 0;
    int pinned = -1;  // schedule fixed by the caller (no tuning), -1 = none
    bool tuned = false;
    cudaGraphExec_t graph[ACO_BATCH_CONFIGS] = {};
    bool built = false, initialized = false, failed = false;
    int iterations = 0;
    float tune_ms[ACO_ALL_SCHEDULES] = {};
    int num_sms = 1;
    unsigned* d_queue = nullptr;  // persistent launch: work counters (4) and barrier (2)
    int* d_status = nullptr;      // bit 0: a barrier wait of a persistent launch ran out
    unsigned long long wait_ns = 10000000000ull;
    char err[512] = {0};
};

static aco_status berr(aco_batch* b, aco_status s, const char* msg) {
    if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
    return s;
}

extern "C" const char* aco_batch_last_error(const aco_batch* b) { return b ? b->err : ""; }

static void free_batch(aco_batch* b) {
    for (auto& g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    for (aco_instance* i : b->inst) aco_destroy_instance(i);
    void* ptrs[] = {b->d_largs, b->d_cargs, b->d_gargs, b->d_rargs, b->d_slot, b->d_rmap, b->d_iter, b->d_queue,
                    b->d_status};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

extern "C" aco_status aco_batch_create(const double* xy_dev, const int32_t* n_host, int32_t count, const aco_params* p,
                                       void* stream, aco_batch** out) {
    ACO_RANGE("aco_batch_create");
    if (!xy_dev || !n_host || !p || !out || count < 1) return ACO_ERR_INVALID_ARG;
    *out = nullptr;
    if (aco_misaligned(xy_dev, 8)) return ACO_ERR_INVALID_ARG;
    if (p->mode != ACO_MODE_LBEST_PARTIAL) return ACO_ERR_INVALID_ARG;
    aco_batch* b = new (std::nothrow) aco_batch();
    if (!b) return ACO_ERR_OOM;
    b->count = count;
    b->p = *p;
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {  // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return ACO_ERR_CUDA;
        }
        b->own_stream = true;
    }
    stream = b->stream;
    long long coff = 0, aoff = 0, toff = 0;
    for (int i = 0; i < count; ++i) {
        aco_params q = *p;
        q.n = n_host[i];
        q.m = p->m < n_host[i] ? p->m : n_host[i];
        q.seed = p->seed + (uint64_t)i;
        aco_instance* ins = nullptr;
        aco_status st = aco_create_instance(xy_dev + 2 * coff, &q, stream, &ins);
        if (st == ACO_OK) ins->in_batch = true;
        if (st != ACO_OK) {
            free_batch(b);
            delete b;
            return st;
        }
        b->inst.push_back(ins);
        b->n_i.push_back(q.n);
        b->m_i.push_back(q.m);
        b->city_off.push_back(coff);
        b->ant_off.push_back(aoff);
        b->tour_off.push_back(toff);
        coff += q.n;
        aoff += q.m;
        toff += (long long)q.m * q.n;
    }
    // schedule: ant slots of the largest instances first (their chains are the longest)
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->n_i[x] > b->n_i[y]; });
    std::vector<int2> slot;
    for (int i : order)
        for (int a = 0; a < b->m_i[i]; ++a) slot.push_back(make_int2(i, a));
    std::vector<int4> rmap;
    for (int i : order)
        for (int c0 = 0; c0 < b->n_i[i]; c0 += 64) rmap.push_back(make_int4(i, c0, std::min(c0 + 64, b->n_i[i]), 0));
    b->slots = (int)slot.size();
    b->rblocks = (int)rmap.size();
    for (int i = 0; i < count; ++i) {
        b->smem_per_ant = std::max(b->smem_per_ant, (int)construct_smem_per_ant(b->n_i[i], p->k));
        b->m_cap = std::max(b->m_cap, b->m_i[i]);
    }
    bool ok = cudaMalloc(&b->d_largs, lbest_args_size() * count) == cudaSuccess;
    ok &= cudaMalloc(&b->d_cargs, sizeof(CommitArgs) * count) == cudaSuccess;
    ok &= cudaMalloc(&b->d_gargs, sizeof(GbestArgs) * count) == cudaSuccess;
    ok &= cudaMalloc(&b->d_rargs, sizeof(RebuildArgs) * count) == cudaSuccess;
    ok &= cudaMalloc(&b->d_slot, sizeof(int2) * slot.size()) == cudaSuccess;
    ok &= cudaMalloc(&b->d_rmap, sizeof(int4) * rmap.size()) == cudaSuccess;
    ok &= cudaMalloc(&b->d_iter, sizeof(int)) == cudaSuccess;
    ok &= cudaMalloc(&b->d_queue, sizeof(unsigned) * 8) == cudaSuccess;
    ok &= cudaMalloc(&b->d_status, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        return ACO_ERR_OOM;
    }
    cudaMemcpy(b->d_slot, slot.data(), sizeof(int2) * slot.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_rmap, rmap.data(), sizeof(int4) * rmap.size(), cudaMemcpyHostToDevice);
    cudaMemset(b->d_queue, 0, sizeof(unsigned) * 8);
    cudaMemset(b->d_status, 0, sizeof(int));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->num_sms < 1) b->num_sms = 1;
    *out = b;
    return ACO_OK;
}

extern "C" aco_status aco_batch_build_candidates(aco_batch* b) {
    ACO_RANGE("aco_batch_build_candidates");
    if (!b) return ACO_ERR_INVALID_ARG;
    for (aco_instance* i : b->inst) {
        aco_status st = aco_build_candidates(i, nullptr);
        if (st != ACO_OK) return berr(b, st, aco_last_error(i));
    }
    b->built = true;
    return ACO_OK;
}

// Descriptors of every colony (initialized flag as the instances stand now).
static aco_status upload_args(aco_batch* b, int32_t iteration) {
    const size_t la = lbest_args_size();
    std::vector<unsigned char> L(la * b->count);
    std::vector<CommitArgs> C(b->count);
    std::vector<GbestArgs> G(b->count);
    std::vector<RebuildArgs> R(b->count);
    for (int i = 0; i < b->count; ++i) {
        fill_lbest_args_bytes(b->inst[i], iteration, L.data() + la * i);
        fill_commit_args(b->inst[i], C[i]);
        fill_gbest_args(b->inst[i], 0, G[i]);
        fill_rebuild_args(b->inst[i], 1, R[i]);
        R[i].m_cap = b->m_cap;
    }
    cudaStream_t s = b->stream;
    cudaMemcpyAsync(b->d_largs, L.data(), L.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_cargs, C.data(), sizeof(CommitArgs) * b->count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_gargs, G.data(), sizeof(GbestArgs) * b->count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_rargs, R.data(), sizeof(RebuildArgs) * b->count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_iter, &iteration, sizeof(int), cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return berr(b, ACO_ERR_CUDA, "descriptor upload failed");
    return ACO_OK;
}

static cudaError_t enqueue_iteration(aco_batch* b, int config) {
    cudaError_t e = launch_construct_batch(reinterpret_cast<const LbestArgs*>(b->d_largs), b->d_slot, b->d_iter,
                                           b->slots, b->smem_per_ant, config, b->stream);
    if (e != cudaSuccess) return e;
    e = launch_update_batch(b->d_cargs, b->d_slot, b->slots, b->d_gargs, b->count, b->d_rargs, b->d_rmap, b->rblocks,
                            b->m_cap, b->p.k, b->stream);
    if (e != cudaSuccess) return e;
    bump_iteration_kernel<<<1, 1, 0, b->stream>>>(b->d_iter);
    return cudaGetLastError();
}

// `iterations` iterations in one persistent launch (schedule ACO_BATCH_CONFIGS + pc).
static cudaError_t enqueue_persistent(aco_batch* b, int pc, int iterations) {
    cudaError_t e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned) * 5, b->stream);  // counters, arrivals
    if (e != cudaSuccess) return e;
    PersistArgs P{};
    P.largs = reinterpret_cast<const LbestArgs*>(b->d_largs);
    P.cargs = b->d_cargs;
    P.gargs = b->d_gargs;
    P.rargs = b->d_rargs;
    P.slot = b->d_slot;
    P.rmap = b->d_rmap;
    P.slots = b->slots;
    P.ritems = b->rblocks;
    P.count = b->count;
    P.iterations = iterations;
    P.smem_per_ant = b->smem_per_ant;
    P.m_cap = b->m_cap;
    P.k = b->p.k;
    P.iteration = b->d_iter;
    P.queue = b->d_queue;
    P.bar = b->d_queue + 4;
    P.wait_ns = b->wait_ns;
    P.status = b->d_status;
    return launch_persistent_batch(P, pc, b->num_sms, b->stream, nullptr);
}

// One iteration with any schedule (four launches or one persistent launch).
static cudaError_t enqueue_any(aco_batch* b, int schedule) {
    if (schedule >= ACO_BATCH_CONFIGS) return enqueue_persistent(b, schedule - ACO_BATCH_CONFIGS, 1);
    return enqueue_iteration(b, schedule);
}

static aco_status graph_for(aco_batch* b, int choice) {
    if (b->graph[choice]) return ACO_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return berr(b, ACO_ERR_CUDA, "stream capture could not begin");
    cudaError_t e = enqueue_iteration(b, choice);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return berr(b, ACO_ERR_CUDA, "iteration capture failed");
    }
    e = cudaGraphInstantiate(&b->graph[choice], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph[choice] = nullptr;
        return berr(b, ACO_ERR_CUDA, "graph instantiation failed");
    }
    return ACO_OK;
}

// The persistent launch's barrier status: ACO_ERR_TIMEOUT once a wait ran out (the batch is then
// unusable).  Synchronises.
static aco_status check_status(aco_batch* b) {
    if (b->failed) return berr(b, ACO_ERR_TIMEOUT, "a barrier wait of the persistent launch ran out");
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(b, ACO_ERR_CUDA, cudaGetErrorString(e));
    if (st & 1) {
        b->failed = true;
        return berr(b, ACO_ERR_TIMEOUT, "a barrier wait of the persistent launch ran out");
    }
    return ACO_OK;
}

extern "C" aco_status aco_batch_run(aco_batch* b, int32_t first_iteration, int32_t iterations, int32_t tune) {
    ACO_RANGE("aco_batch_run");
    if (!b || iterations < 0 || first_iteration < 0) return ACO_ERR_INVALID_ARG;
    if (!b->built) return berr(b, ACO_ERR_STATE, "run before build_candidates");
    if (b->failed) return berr(b, ACO_ERR_STATE, "the batch failed earlier (barrier wait ran out)");
    if (iterations == 0) return ACO_OK;
    if (b->pinned >= 0) b->config = b->pinned;
    if (!b->initialized) {  // initial tours (Algorithm 1, before its iterations): every ant builds a full tour
        aco_status st = upload_args(b, first_iteration);
        if (st != ACO_OK) return st;
        if (enqueue_any(b, b->config) != cudaSuccess) return berr(b, ACO_ERR_CUDA, "initial iteration failed");
        for (aco_instance* i : b->inst) {
            i->initialized = true;
            i->iterations++;
        }
        b->initialized = true;
        b->iterations++;
        ++first_iteration;
        --iterations;
        st = upload_args(b, first_iteration);  // descriptors now say "initialized"
        if (st != ACO_OK) return st;
    } else {
        cudaMemcpyAsync(b->d_iter, &first_iteration, sizeof(int), cudaMemcpyHostToDevice, b->stream);
    }
    int done = 0;
    if (tune && !b->tuned && b->pinned < 0) {  // time live iterations with each schedule, keep the fastest
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int best_choice = 0;
        for (int c = 0; c < ACO_ALL_SCHEDULES && done < iterations; ++c, ++done) {
            if (c < ACO_BATCH_CONFIGS) {
                aco_status st = graph_for(b, c);
                if (st != ACO_OK) return st;
            }
            cudaEventRecord(e0, b->stream);
            cudaError_t e = c < ACO_BATCH_CONFIGS ? cudaGraphLaunch(b->graph[c], b->stream) : enqueue_any(b, c);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            if (e != cudaSuccess) return berr(b, ACO_ERR_CUDA, cudaGetErrorString(e));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            b->tune_ms[c] = ms;
            if (ms < best) { best = ms; best_choice = c; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->config = best_choice;
        b->tuned = true;
        aco_status st = check_status(b);
        if (st != ACO_OK) return st;
    }
    const int choice = b->config;
    if (choice >= ACO_BATCH_CONFIGS) {
        if (done < iterations) {
            cudaError_t e = enqueue_persistent(b, choice - ACO_BATCH_CONFIGS, iterations - done);
            if (e != cudaSuccess) return berr(b, ACO_ERR_CUDA, cudaGetErrorString(e));
        }
    } else {
        aco_status st = graph_for(b, choice);
        if (st != ACO_OK) return st;
        for (; done < iterations; ++done)
            if (cudaGraphLaunch(b->graph[choice], b->stream) != cudaSuccess)
                return berr(b, ACO_ERR_CUDA, "graph launch failed");
    }
    for (aco_instance* i : b->inst) i->iterations += iterations;
    b->iterations += iterations;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(b, ACO_ERR_CUDA, cudaGetErrorString(e));
    return ACO_OK;
}

extern "C" aco_status aco_batch_get_state(aco_batch* b, int32_t* lbest_out_dev, double* clen_out_dev) {
    ACO_RANGE("aco_batch_get_state");
    if (!b || aco_misaligned(lbest_out_dev, 4) || aco_misaligned(clen_out_dev, 8)) return ACO_ERR_INVALID_ARG;
    aco_status st = check_status(b);
    if (st != ACO_OK) return st;
    for (int i = 0; i < b->count; ++i) {
        st = aco_get_state(b->inst[i], lbest_out_dev ? lbest_out_dev + b->tour_off[i] : nullptr,
                           clen_out_dev ? clen_out_dev + b->ant_off[i] : nullptr, nullptr);
        if (st != ACO_OK) return berr(b, st, aco_last_error(b->inst[i]));
    }
    return ACO_OK;
}

extern "C" aco_status aco_batch_get_best(aco_batch* b, double* best_len_host) {
    ACO_RANGE("aco_batch_get_best");
    if (!b || !best_len_host) return ACO_ERR_INVALID_ARG;
    aco_status st = check_status(b);
    if (st != ACO_OK) return st;
    for (int i = 0; i < b->count; ++i) {
        aco_stats s;
        st = aco_get_stats(b->inst[i], &s);
        if (st != ACO_OK) return berr(b, st, aco_last_error(b->inst[i]));
        best_len_host[i] = s.gbest;
    }
    return ACO_OK;
}

extern "C" aco_status aco_batch_schedule(const aco_batch* b, int32_t* schedule_out, int32_t* warps_out,
                                         int32_t* min_blocks_out, int32_t* persistent_out, float* tune_ms_out) {
    if (!b) return ACO_ERR_INVALID_ARG;
    const int c = b->config;
    const bool pers = c >= ACO_BATCH_CONFIGS;
    if (schedule_out) *schedule_out = c;
    if (warps_out) *warps_out = pers ? kPersistConfigs[c - ACO_BATCH_CONFIGS][0] : kBatchConfigs[c][0];
    if (min_blocks_out) *min_blocks_out = pers ? kPersistConfigs[c - ACO_BATCH_CONFIGS][1] : kBatchConfigs[c][1];
    if (persistent_out) *persistent_out = pers ? kPersistConfigs[c - ACO_BATCH_CONFIGS][2] : 0;
    if (tune_ms_out)
        for (int i = 0; i < ACO_ALL_SCHEDULES; ++i) tune_ms_out[i] = b->tune_ms[i];
    return ACO_OK;
}

extern "C" aco_status aco_batch_set_schedule(aco_batch* b, int32_t schedule) {
    if (!b || schedule < -1 || schedule >= ACO_ALL_SCHEDULES) return ACO_ERR_INVALID_ARG;
    b->pinned = schedule;
    if (schedule >= 0) b->config = schedule;
    return ACO_OK;
}

extern "C" aco_status aco_batch_set_wait_limit(aco_batch* b, double seconds) {
    if (!b || !(seconds >= 0.0 && seconds <= 3600.0)) return ACO_ERR_INVALID_ARG;
    b->wait_ns = (unsigned long long)(seconds * 1e9);
    return ACO_OK;
}

extern "C" aco_status aco_batch_instance(aco_batch* b, int32_t i, aco_instance** out) {
    if (!b || !out || i < 0 || i >= b->count) return ACO_ERR_INVALID_ARG;
    *out = b->inst[i];
    return ACO_OK;
}

extern "C" void aco_batch_destroy(aco_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

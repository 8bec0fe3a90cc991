// api.cu -- the C ABI entry points of include/aco.h: argument checks, allocation (all in
// aco_create_instance), call ordering and error reporting.  Kernels live in grid_knn.cu,
// construct_dev.cuh (launched from construct.cu and the batched units) and update.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "common.cuh"

aco_status set_err(aco_instance* inst, aco_status s, const char* fmt, ...) {
    if (inst) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(inst->err, sizeof(inst->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

aco_status check_launch(aco_instance* inst, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(inst, ACO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ACO_OK;
}

static thread_local char g_create_err[512];

extern "C" const char* aco_status_string(aco_status s) {
    switch (s) {
        case ACO_OK: return "ok";
        case ACO_ERR_INVALID_ARG: return "invalid argument";
        case ACO_ERR_OOM: return "out of device memory";
        case ACO_ERR_CUDA: return "CUDA error";
        case ACO_ERR_STATE: return "call out of order";
        case ACO_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

extern "C" const char* aco_last_error(const aco_instance* inst) { return inst ? inst->err : g_create_err; }

static void free_all(aco_instance* inst) {
    void* ptrs[] = {inst->xy, inst->grid_dev, inst->city_cell, inst->cell_start, inst->cell_city, inst->cell_xy,
                    inst->cell_fill, inst->candw, inst->cand, inst->etab, inst->W64, inst->rowflag, inst->lbest,
                    inst->nb, inst->nbrank, inst->clen, inst->cfix, inst->q, inst->gbest, inst->gbest_ant,
                    inst->seg, inst->antit, inst->accq, inst->tau, inst->etab_d, inst->W64d, inst->W32d,
                    inst->tours, inst->succ_d, inst->pred_d, inst->counters, inst->errflag, inst->xy32,
                    inst->ulist, inst->uxy, inst->bel, inst->btx, inst->btq, inst->deg, inst->ghk, inst->ghq,
                    inst->ls_buf, inst->ls_sel, inst->ls_imp, inst->fcnt, inst->ccnt, inst->csize, inst->Qt,
                    inst->rec_off, inst->nrec, inst->ext, inst->far};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// Byte limit on an instance's device buffers from the environment variable ACO_DEVICE_BYTES_LIMIT
// (unset or unparsable: none).  Creation fails with ACO_ERR_OOM, as it does when cudaMalloc
// fails, once the buffers would exceed it: a way to exercise the out-of-memory path on purpose.
static size_t device_bytes_limit() {
    const char* v = getenv("ACO_DEVICE_BYTES_LIMIT");
    if (!v || !*v) return (size_t)-1;
    char* end = nullptr;
    const unsigned long long x = strtoull(v, &end, 10);
    return (end && *end == 0) ? (size_t)x : (size_t)-1;
}

// One device buffer of `count` elements; alloc = false only counts its bytes (the dry run that
// checks the byte limit before anything touches the device).
template <typename T>
static bool dalloc(T** p, size_t count, size_t* total, bool alloc = true) {
    if (count == 0) count = 1;
    *total += count * sizeof(T);
    if (!alloc) {
        *p = nullptr;
        return true;
    }
    if (*total > device_bytes_limit()) return false;
    return cudaMalloc((void**)p, count * sizeof(T)) == cudaSuccess;
}

static bool params_ok(const aco_params* p, char* why, size_t wn) {
    if (p->mode != ACO_MODE_DENSE && p->mode != ACO_MODE_LBEST_PARTIAL) return snprintf(why, wn, "mode"), false;
    if (p->n < 3) return snprintf(why, wn, "n < 3"), false;
    if (p->m < 1 || p->m > 16384) return snprintf(why, wn, "m must be in [1, 16384]"), false;
    if (p->mode == ACO_MODE_LBEST_PARTIAL && (p->k < 1 || p->k > ACO_MAX_K || p->k > p->n - 1))
        return snprintf(why, wn, "k must be in [1, min(32, n-1)]"), false;
    if (!(isfinite(p->alpha) && p->alpha >= 0) || !(isfinite(p->beta) && p->beta >= 0))
        return snprintf(why, wn, "alpha, beta must be finite and >= 0"), false;
    if (!(isfinite(p->tau0) && p->tau0 > 0)) return snprintf(why, wn, "tau0 must be > 0"), false;
    if (p->mode == ACO_MODE_DENSE && !(p->rho >= 0 && p->rho <= 1)) return snprintf(why, wn, "rho in [0,1]"), false;
    if (p->mode == ACO_MODE_LBEST_PARTIAL && !(p->max_mod_frac > 0 && p->max_mod_frac <= 1))
        return snprintf(why, wn, "max_mod_frac in (0,1]"), false;
    if (!(p->p_partial >= 0 && p->p_partial <= 1)) return snprintf(why, wn, "p_partial in [0,1]"), false;
    if (p->fallback != 0 && p->fallback != 1) return snprintf(why, wn, "fallback must be 0 or 1"), false;
    if (p->selection != 0 && p->selection != 1) return snprintf(why, wn, "selection must be 0 or 1"), false;
    // eta^0 = 1 makes every candidate list arbitrary and the exhausted-list rule a lowest-index scan
    if (p->mode == ACO_MODE_LBEST_PARTIAL && !(p->beta > 0))
        return snprintf(why, wn, "beta must be > 0 with candidate lists"), false;
    if (p->mode == ACO_MODE_DENSE && p->selection != 0)
        return snprintf(why, wn, "Independent Roulette needs candidate lists (LBEST mode)"), false;
    if (p->mode == ACO_MODE_DENSE && p->n > 8192) return snprintf(why, wn, "DENSE mode supports n <= 8192"), false;
    // the visited bitset of one ant lives in shared memory (<= 200 KB, beside ~6 KB of buffers)
    if ((long long)(p->n + 31) / 32 * 4 > 200 * 1024) return snprintf(why, wn, "n too large for the visited bitset"), false;
    if ((long long)p->n * p->m > (1ll << 31) - 1) return snprintf(why, wn, "n*m must be < 2^31"), false;
    return true;
}

// Every device buffer an instance allocates at creation (before the grid is known), or, with
// alloc = false, only their bytes in *total.
static bool plan_buffers(aco_instance* inst, const aco_params* p, size_t* total, bool alloc) {
    const long long n = p->n, m = p->m, k = p->k;
    bool ok = true;
    ok &= dalloc(&inst->xy, 2 * n, total, alloc);
    ok &= dalloc(&inst->grid_dev, 1, total, alloc);
    ok &= dalloc(&inst->city_cell, n, total, alloc);
    inst->ncells_cap = (int32_t)(n / 2 + 16);
    ok &= dalloc(&inst->cell_start, inst->ncells_cap + 1, total, alloc);
    ok &= dalloc(&inst->cell_fill, inst->ncells_cap, total, alloc);
    ok &= dalloc(&inst->cell_city, n, total, alloc);
    ok &= dalloc(&inst->cell_xy, 2 * n, total, alloc);
    ok &= dalloc(&inst->counters, CNT_N, total, alloc);
    ok &= dalloc(&inst->errflag, 1, total, alloc);
    ok &= dalloc(&inst->clen, m, total, alloc);
    ok &= dalloc(&inst->cfix, 2 * m, total, alloc);
    ok &= dalloc(&inst->gbest, 1, total, alloc);
    ok &= dalloc(&inst->gbest_ant, 1, total, alloc);
    if (p->mode == ACO_MODE_LBEST_PARTIAL) {
        ok &= dalloc(&inst->candw, n * k, total, alloc);
        ok &= dalloc(&inst->cand, n * k, total, alloc);
        ok &= dalloc(&inst->etab, n * k, total, alloc);
        ok &= dalloc(&inst->W64, n * k, total, alloc);
        ok &= dalloc(&inst->rowflag, n, total, alloc);
        ok &= dalloc(&inst->lbest, m * n, total, alloc);
        ok &= dalloc(&inst->nb, 2 * n * m, total, alloc);
        ok &= dalloc(&inst->nbrank, 2 * n * m, total, alloc);
        ok &= dalloc(&inst->q, m, total, alloc);
        ok &= dalloc(&inst->seg, m * n, total, alloc);
        ok &= dalloc(&inst->antit, m, total, alloc);
        if (p->fallback == 1) ok &= dalloc(&inst->accq, m * n, total, alloc);
        ok &= dalloc(&inst->bel, m * 2 * m, total, alloc);
        ok &= dalloc(&inst->btx, m * 2 * m, total, alloc);
        ok &= dalloc(&inst->btq, m * 2 * m, total, alloc);
        ok &= dalloc(&inst->ghk, m * 2 * m, total, alloc);
        ok &= dalloc(&inst->ghq, m * 2 * m, total, alloc);
        long long fm = (long long)floor(p->max_mod_frac * (double)n);
        long long pmin = n - fm;
        if (pmin < 1) pmin = 1;
        if (pmin > n - 1) pmin = n - 1;
        inst->ucap = (int32_t)(n - pmin);
        inst->f_cap = p->max_mod_frac;
        inst->ls_window = 500;
        ok &= dalloc(&inst->ulist, m * inst->ucap, total, alloc);
        ok &= dalloc(&inst->uxy, m * inst->ucap, total, alloc);
        ok &= dalloc(&inst->xy32, n, total, alloc);
        ok &= dalloc(&inst->deg, n, total, alloc);
        ok &= dalloc(&inst->rec_off, m, total, alloc);
        ok &= dalloc(&inst->nrec, 1, total, alloc);
        // extended neighbour lists speed up the exhausted-list rule
        inst->kx = (int32_t)(n - 1 < ACO_KX ? n - 1 : ACO_KX);
        if (inst->kx > k) ok &= dalloc(&inst->ext, n * inst->kx, total, alloc);
        else inst->kx = 0;
        // large colonies also keep the 128 nearest: the initial tours' exhausted steps find the
        // nearest unvisited city there far more often than in the 32 nearest
        if (inst->kx > k && n > ACO_FAR_MIN_N) ok &= dalloc(&inst->far, n * ACO_KF, total, alloc);
    } else {
        ok &= dalloc(&inst->tau, n * n, total, alloc);
        ok &= dalloc(&inst->etab_d, n * n, total, alloc);
        ok &= dalloc(&inst->W64d, n * n, total, alloc);
        ok &= dalloc(&inst->W32d, n * n, total, alloc);
        ok &= dalloc(&inst->rowflag, n, total, alloc);
        ok &= dalloc(&inst->tours, m * n, total, alloc);
        ok &= dalloc(&inst->succ_d, m * n, total, alloc);
        ok &= dalloc(&inst->pred_d, m * n, total, alloc);
    }
    return ok;
}

extern "C" aco_status aco_create_instance(const double* xy_dev, const aco_params* p, void* stream,
                                          aco_instance** out) {
    ACO_RANGE("aco_create_instance");
    g_create_err[0] = 0;
    if (!out || !p || !xy_dev) {
        snprintf(g_create_err, sizeof(g_create_err), "null argument");
        return ACO_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (aco_misaligned(xy_dev, 8)) {
        snprintf(g_create_err, sizeof(g_create_err), "xy_dev not 8-byte aligned");
        return ACO_ERR_INVALID_ARG;
    }
    if (!params_ok(p, g_create_err, sizeof(g_create_err))) return ACO_ERR_INVALID_ARG;
    {
        aco_instance probe;
        memset(&probe, 0, sizeof(probe));
        size_t need = 0;
        plan_buffers(&probe, p, &need, false);
        if (need > device_bytes_limit()) {
            snprintf(g_create_err, sizeof(g_create_err), "the buffers need %zu bytes, above ACO_DEVICE_BYTES_LIMIT",
                     need);
            return ACO_ERR_OOM;
        }
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, xy_dev) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        snprintf(g_create_err, sizeof(g_create_err), "xy_dev is not a device pointer");
        return ACO_ERR_INVALID_ARG;
    }
    aco_instance* inst = new (std::nothrow) aco_instance();
    if (!inst) return ACO_ERR_OOM;
    memset(inst, 0, sizeof(*inst));
    inst->p = *p;
    inst->stream = (cudaStream_t)stream;
    inst->gbest_ant = nullptr;
    cudaGetDevice(&inst->device);
    cudaDeviceGetAttribute(&inst->num_sms, cudaDevAttrMultiProcessorCount, inst->device);

    const long long n = p->n, m = p->m;
    size_t total = 0;
    bool ok = plan_buffers(inst, p, &total, true);
    if (!ok) {
        cudaGetLastError();
        snprintf(g_create_err, sizeof(g_create_err), "device allocation of %.3f GB failed", total / 1e9);
        free_all(inst);
        delete inst;
        return ACO_ERR_OOM;
    }
    cudaStream_t s = inst->stream;
    cudaMemcpyAsync(inst->xy, xy_dev, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(inst->counters, 0, sizeof(unsigned long long) * CNT_N, s);
    cudaMemsetAsync(inst->errflag, 0, sizeof(int), s);
    if (p->mode == ACO_MODE_LBEST_PARTIAL) {
        if (inst->accq) cudaMemsetAsync(inst->accq, 0, sizeof(unsigned long long) * m * n, s);
        cudaMemsetAsync(inst->nb, 0xFF, sizeof(int32_t) * 2 * n * m, s);
        cudaMemsetAsync(inst->nbrank, 0xFF, 2 * n * m, s);
        cudaMemsetAsync(inst->ghk, 0xFF, sizeof(int32_t) * 2 * m * m, s);
        cudaMemsetAsync(inst->ghq, 0, sizeof(unsigned long long) * 2 * m * m, s);
    }
    // coordinates: finite, and bounding box * n small enough for the exact length grid
    double* hxy = (double*)malloc(sizeof(double) * 2 * n);
    cudaMemcpyAsync(hxy, xy_dev, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free(hxy);
        snprintf(g_create_err, sizeof(g_create_err), "create: %s", cudaGetErrorString(e));
        free_all(inst);
        delete inst;
        return ACO_ERR_CUDA;
    }
    double xmin = hxy[0], xmax = hxy[0], ymin = hxy[1], ymax = hxy[1];
    bool finite = true;
    for (long long i = 0; i < n; ++i) {
        const double x = hxy[2 * i], y = hxy[2 * i + 1];
        finite &= (bool)(isfinite(x) && isfinite(y));
        xmin = fmin(xmin, x); xmax = fmax(xmax, x); ymin = fmin(ymin, y); ymax = fmax(ymax, y);
    }
    free(hxy);
    const double diag = hypot(xmax - xmin, ymax - ymin);
    inst->coord_r = nextafterf((float)fmax(fmax(fabs(xmin), fabs(xmax)), fmax(fabs(ymin), fabs(ymax))), INFINITY);
    if (!finite || !(diag * (double)n < 1073741824.0)) {
        snprintf(g_create_err, sizeof(g_create_err), "coordinates must be finite with bbox diagonal * n < 2^30");
        free_all(inst);
        delete inst;
        return ACO_ERR_INVALID_ARG;
    }
    // grid over the bounding box, about two cities per cell
    GridDesc g;
    g.xmin = xmin; g.xmax = xmax; g.ymin = ymin; g.ymax = ymax;
    const double wx = fmax(xmax - xmin, 1e-300), wy = fmax(ymax - ymin, 1e-300);
    const double target_cells = fmax(1.0, (double)(n / 2));
    double h = sqrt(wx * wy / target_cells);
    if (!(h > 0)) h = fmax(wx, wy);
    h = fmax(h, fmax(wx, wy) / 4096.0);
    int gx = (int)fmin(4096.0, floor(wx / h) + 1), gy = (int)fmin(4096.0, floor(wy / h) + 1);
    while ((long long)gx * gy > inst->ncells_cap) {
        h *= 1.05;
        gx = (int)floor(wx / h) + 1;
        gy = (int)floor(wy / h) + 1;
    }
    g.h = h; g.gx = gx; g.gy = gy;
    const double mag = fabs(xmin) + fabs(xmax) + fabs(ymin) + fabs(ymax);
    g.margin = 1e-6 * h + 1e-14 * mag;
    inst->grid = g;
    cudaMemcpy(inst->grid_dev, &g, sizeof(g), cudaMemcpyHostToDevice);
    if (p->mode == ACO_MODE_LBEST_PARTIAL) {
        // per-ant unvisited counts per cell and per coarse block (full constructions)
        inst->ncells = gx * gy;
        inst->cgx = (gx + ACO_CBLK - 1) / ACO_CBLK;
        inst->cgy = (gy + ACO_CBLK - 1) / ACO_CBLK;
        inst->ncoarse = inst->cgx * inst->cgy;
        bool ok2 = dalloc(&inst->fcnt, m * inst->ncells, &total);
        ok2 &= dalloc(&inst->ccnt, m * inst->ncoarse, &total);
        ok2 &= dalloc(&inst->csize, inst->ncoarse, &total);
        if (!ok2) {
            cudaGetLastError();
            snprintf(g_create_err, sizeof(g_create_err), "device allocation of %.1f MB failed", total / 1e6);
            free_all(inst);
            delete inst;
            return ACO_ERR_OOM;
        }
    }
    inst->last_iteration = -1;
    inst->ant0 = 0;
    inst->ant1 = p->m;
    *out = inst;
    return ACO_OK;
}

extern "C" void aco_destroy_instance(aco_instance* inst) {
    if (!inst) return;
    cudaStreamSynchronize(inst->stream);
    free_all(inst);
    delete inst;
}

aco_status sync_and_check(aco_instance* inst, const char* what) {
    cudaError_t e = cudaStreamSynchronize(inst->stream);
    if (e != cudaSuccess) return set_err(inst, ACO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    int flag = 0;
    e = cudaMemcpy(&flag, inst->errflag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_err(inst, ACO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    if (flag) {
        cudaMemset(inst->errflag, 0, sizeof(int));
        if (flag & DEVERR_DUPLICATE) return set_err(inst, ACO_ERR_INVALID_ARG, "%s: coincident cities", what);
        if (flag & DEVERR_BAD_TOUR) return set_err(inst, ACO_ERR_INVALID_ARG, "%s: tour index out of range", what);
        if (flag & DEVERR_NONFINITE) return set_err(inst, ACO_ERR_INVALID_ARG, "%s: non-finite weight", what);
        if (flag & DEVERR_BAD_SCORE) return set_err(inst, ACO_ERR_INVALID_ARG, "%s: edge score not finite and > 0", what);
        if (flag & DEVERR_BAD_RECORD) return set_err(inst, ACO_ERR_INVALID_ARG, "%s: malformed commit record", what);
        return set_err(inst, ACO_ERR_CUDA, "%s: device error flag %d", what, flag);
    }
    return ACO_OK;
}

extern "C" aco_status aco_build_candidates(aco_instance* inst, int32_t* cand_out_dev) {
    ACO_RANGE("aco_build_candidates");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(cand_out_dev, 4)) return set_err(inst, ACO_ERR_INVALID_ARG, "cand_out_dev not 4-byte aligned");
    aco_status st = launch_build_grid_and_knn(inst);
    if (st != ACO_OK) return st;
    if (inst->p.mode == ACO_MODE_LBEST_PARTIAL) {
        st = launch_coarse_sizes(inst);
        if (st != ACO_OK) return st;
        st = launch_lbest_init_weights(inst);
        if (st != ACO_OK) return st;
        if (cand_out_dev)
            cudaMemcpyAsync(cand_out_dev, inst->cand, sizeof(int32_t) * (size_t)inst->p.n * inst->p.k,
                            cudaMemcpyDeviceToDevice, inst->stream);
    } else {
        st = launch_dense_init(inst);
        if (st != ACO_OK) return st;
    }
    st = sync_and_check(inst, "build_candidates");
    if (st != ACO_OK) return st;
    inst->cand_built = true;
    inst->constructed = false;
    inst->initialized = false;
    inst->scored = false;
    return ACO_OK;
}

extern "C" aco_status aco_construct_tours(aco_instance* inst, int32_t iteration, int32_t* tours_out_dev,
                                          double* len_out_dev) {
    ACO_RANGE("aco_construct_tours");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (!inst->cand_built) return set_err(inst, ACO_ERR_STATE, "construct_tours before build_candidates");
    if (iteration < 0) return set_err(inst, ACO_ERR_INVALID_ARG, "iteration must be >= 0");
    if (aco_misaligned(tours_out_dev, 4) || aco_misaligned(len_out_dev, 8))
        return set_err(inst, ACO_ERR_INVALID_ARG, "construct_tours: output not aligned to its element type");
    aco_status st = inst->p.mode == ACO_MODE_LBEST_PARTIAL ? launch_construct_lbest(inst, iteration)
                                                           : launch_construct_dense(inst, iteration);
    if (st != ACO_OK) return st;
    if (inst->p.mode == ACO_MODE_LBEST_PARTIAL && inst->ls_p > 0.0) {
        st = launch_local_search(inst, iteration);
        if (st != ACO_OK) return st;
    }
    if (tours_out_dev || len_out_dev) {
        st = launch_write_new_tours(inst, tours_out_dev, len_out_dev);
        if (st != ACO_OK) return st;
    }
    inst->constructed = true;
    inst->last_iteration = iteration;
    return ACO_OK;
}

extern "C" aco_status aco_update_pheromone(aco_instance* inst) {
    ACO_RANGE("aco_update_pheromone");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (!inst->constructed) return set_err(inst, ACO_ERR_STATE, "update_pheromone without a construction");
    aco_status st = inst->p.mode == ACO_MODE_LBEST_PARTIAL ? launch_update_lbest(inst) : launch_update_dense(inst);
    if (st != ACO_OK) return st;
    inst->constructed = false;
    inst->initialized = true;
    inst->iterations++;
    return ACO_OK;
}

extern "C" aco_status aco_tour_lengths(aco_instance* inst, const int32_t* tours_dev, int32_t count, double* out_dev) {
    ACO_RANGE("aco_tour_lengths");
    if (!inst || count < 0 || (count > 0 && (!tours_dev || !out_dev))) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(tours_dev, 4) || aco_misaligned(out_dev, 8))
        return set_err(inst, ACO_ERR_INVALID_ARG, "tour_lengths: buffer not aligned to its element type");
    if (count == 0) return ACO_OK;
    return launch_tour_lengths(inst, tours_dev, count, out_dev);
}

extern "C" aco_status aco_get_state(aco_instance* inst, int32_t* lbest_out_dev, double* clen_out_dev,
                                    double* tau_out_dev) {
    ACO_RANGE("aco_get_state");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(lbest_out_dev, 4) || aco_misaligned(clen_out_dev, 8) || aco_misaligned(tau_out_dev, 8))
        return set_err(inst, ACO_ERR_INVALID_ARG, "get_state: output not aligned to its element type");
    const size_t n = inst->p.n, m = inst->p.m;
    cudaStream_t s = inst->stream;
    if (inst->p.mode == ACO_MODE_LBEST_PARTIAL) {
        if (lbest_out_dev) cudaMemcpyAsync(lbest_out_dev, inst->lbest, sizeof(int32_t) * m * n, cudaMemcpyDeviceToDevice, s);
        if (clen_out_dev) cudaMemcpyAsync(clen_out_dev, inst->clen, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
    } else {
        if (lbest_out_dev) cudaMemcpyAsync(lbest_out_dev, inst->tours, sizeof(int32_t) * m * n, cudaMemcpyDeviceToDevice, s);
        if (clen_out_dev) cudaMemcpyAsync(clen_out_dev, inst->clen, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
        if (tau_out_dev) cudaMemcpyAsync(tau_out_dev, inst->tau, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s);
    }
    return sync_and_check(inst, "get_state");
}

aco_status launch_reweight(aco_instance* inst);

extern "C" aco_status aco_set_async_share(aco_instance* inst, int32_t on) {
    ACO_RANGE("aco_set_async_share");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "set_async_share: LBEST mode only");
    if (inst->in_batch) return set_err(inst, ACO_ERR_STATE, "set_async_share: not for an instance of a batch");
    if (inst->constructed) return set_err(inst, ACO_ERR_STATE, "set_async_share: tours constructed, update pending");
    if (on != 0 && on != 1) return set_err(inst, ACO_ERR_INVALID_ARG, "set_async_share: on must be 0 or 1");
    if (on && inst->ls_p > 0.0)
        return set_err(inst, ACO_ERR_STATE, "set_async_share: local search is on (the two exclude each other)");
    if (on && (inst->ant0 != 0 || inst->ant1 != inst->p.m))
        return set_err(inst, ACO_ERR_STATE, "set_async_share: the colony is split over ranks");
    if (on && !inst->Qt) {
        if (cudaMalloc(&inst->Qt, sizeof(unsigned long long) * (size_t)inst->p.n * inst->p.k) != cudaSuccess) {
            cudaGetLastError();
            inst->Qt = nullptr;
            return set_err(inst, ACO_ERR_OOM, "set_async_share: pheromone table allocation failed");
        }
        // the table starts as the integer pheromone of the current l_best population (zero before
        // the first update); the rebuild keeps it so from then on
        aco_status st = launch_reweight(inst);
        if (st != ACO_OK) return st;
        st = sync_and_check(inst, "set_async_share");
        if (st != ACO_OK) return st;
    }
    inst->async_share = on;
    return ACO_OK;
}

extern "C" aco_status aco_set_state(aco_instance* inst, const int32_t* lbest_dev, const double* tau_dev) {
    ACO_RANGE("aco_set_state");
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(lbest_dev, 4) || aco_misaligned(tau_dev, 8))
        return set_err(inst, ACO_ERR_INVALID_ARG, "set_state: input not aligned to its element type");
    if (!inst->cand_built) return set_err(inst, ACO_ERR_STATE, "set_state before build_candidates");
    if (inst->p.mode == ACO_MODE_LBEST_PARTIAL) {
        if (!lbest_dev) return set_err(inst, ACO_ERR_INVALID_ARG, "lbest_dev is required");
        aco_status st = launch_set_lbest(inst, lbest_dev);
        if (st != ACO_OK) return st;
    } else {
        if (!tau_dev) return set_err(inst, ACO_ERR_INVALID_ARG, "tau_dev is required");
        const size_t n = inst->p.n;
        cudaMemcpyAsync(inst->tau, tau_dev, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, inst->stream);
        aco_status st = launch_dense_init(inst);  // rebuilds the weights from tau (keeps tau)
        if (st != ACO_OK) return st;
    }
    aco_status st = sync_and_check(inst, "set_state");
    if (st != ACO_OK) return st;
    inst->initialized = true;
    inst->constructed = false;
    return ACO_OK;
}

extern "C" aco_status aco_get_stats(aco_instance* inst, aco_stats* out_host) {
    ACO_RANGE("aco_get_stats");
    if (!inst || !out_host) return ACO_ERR_INVALID_ARG;
    aco_status st = sync_and_check(inst, "get_stats");
    if (st != ACO_OK) return st;
    unsigned long long c[CNT_N];
    cudaMemcpy(c, inst->counters, sizeof(c), cudaMemcpyDeviceToHost);
    memset(out_host, 0, sizeof(*out_host));
    out_host->decisions = c[CNT_DECISIONS];
    out_host->fallbacks = c[CNT_FALLBACKS];
    out_host->exact_resolves = c[CNT_RESOLVES];
    out_host->improved = c[CNT_IMPROVED];
    out_host->partial_ants = c[CNT_PARTIAL];
    out_host->full_ants = c[CNT_FULL];
    out_host->ls_moves = c[CNT_LS_MOVES];
    out_host->fallback_rebuilt = c[CNT_FB_REBUILT];
    out_host->fallback_scanned = c[CNT_FB_SCANNED];
    out_host->fallback_fast = c[CNT_FB_FAST];
    out_host->gbest = INFINITY;
    out_host->gbest_ant = -1;
    if (inst->initialized) {
        cudaMemcpy(&out_host->gbest, inst->gbest, sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(&out_host->gbest_ant, inst->gbest_ant, sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    out_host->iterations = inst->iterations;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(inst, ACO_ERR_CUDA, "get_stats: %s", cudaGetErrorString(e));
    return ACO_OK;
}

extern "C" aco_status aco_step_probs(aco_instance* inst, int32_t city, const uint32_t* visited_bits_dev,
                                     float* probs_out_dev, int32_t* exhausted_out_dev) {
    if (!inst || !visited_bits_dev || !probs_out_dev || !exhausted_out_dev) return ACO_ERR_INVALID_ARG;
    if (aco_misaligned(visited_bits_dev, 4) || aco_misaligned(probs_out_dev, 4) || aco_misaligned(exhausted_out_dev, 4))
        return set_err(inst, ACO_ERR_INVALID_ARG, "step_probs: buffer not 4-byte aligned");
    if (city < 0 || city >= inst->p.n) return set_err(inst, ACO_ERR_INVALID_ARG, "city out of range");
    if (!inst->cand_built) return set_err(inst, ACO_ERR_STATE, "step_probs before build_candidates");
    return launch_step_probs(inst, city, visited_bits_dev, probs_out_dev, exhausted_out_dev);
}

extern "C" aco_status aco_set_max_mod_frac(aco_instance* inst, double f) {
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "set_max_mod_frac: LBEST mode only");
    if (inst->constructed) return set_err(inst, ACO_ERR_STATE, "set_max_mod_frac: tours constructed, update pending");
    if (!(f > 0.0 && f <= inst->f_cap))
        return set_err(inst, ACO_ERR_INVALID_ARG, "set_max_mod_frac: f must be in (0, f at creation = %g]", inst->f_cap);
    inst->p.max_mod_frac = f;
    return ACO_OK;
}

extern "C" aco_status aco_set_p_partial(aco_instance* inst, double p_partial) {
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "set_p_partial: LBEST mode only");
    if (inst->constructed) return set_err(inst, ACO_ERR_STATE, "set_p_partial: tours constructed, update pending");
    if (!(p_partial >= 0.0 && p_partial <= 1.0)) return set_err(inst, ACO_ERR_INVALID_ARG, "set_p_partial: p in [0, 1]");
    inst->p.p_partial = p_partial;
    return ACO_OK;
}

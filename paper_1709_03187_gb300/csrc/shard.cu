// shard.cu -- one colony split over several GPUs by ants (Section 3: a single colony whose
// pheromone comes from every ant's l_best).
//
// Every rank keeps the whole colony state (instance, candidate lists, every ant's l_best and the
// neighbour tables) and constructs only its own range of ants.  Within an iteration the
// pheromone is fixed and every commit touches only the committing ant's own l_best row and its
// own neighbour entries (Algorithm 1's replacement, read synchronously), and the pheromone
// rebuild sums integer weights, so the order of commits does not matter: once every rank has
// applied every rank's commits, each rank's update gives the state of the single colony bit for
// bit.  The exchange is a list of commit records per rank:
//
//   buffer  word 0 the number of records, word 1 zero, words 2-3 the words used (an int64,
//           including these four), then the records from word 4 on;
//   record  [0] ant, [1] s, [2] P, [3] M, [4] start, [5] segment length L (M for a partial
//           rebuild, n for a full construction), [6..7] new length (FP64 bits, low word first),
//           [8..9] and [10..11] the exact 128-bit fixed-point length (low 64 bits, high 64 bits),
//           [12 .. 12 + L) the new cities of the segment.
//
// Only ants whose new tour is strictly shorter than their l_best (the ones that commit) are
// exported.
#include <math.h>

#include "common.cuh"

#define REC_HEAD 12

__global__ void __launch_bounds__(32) export_commits_kernel(int n, int ant0, const AntIter* __restrict__ antit,
                                                            const double* __restrict__ clen,
                                                            const int* __restrict__ seg, int* __restrict__ buf,
                                                            long long cap) {
    const int a = ant0 + blockIdx.x, lane = threadIdx.x;
    const AntIter it = antit[a];
    if (!(it.newlen < clen[a])) return;
    const int L = it.s >= 0 ? it.M : n;
    long long off = 0;
    if (lane == 0) {
        off = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(buf + 2), (unsigned long long)(REC_HEAD + L));
        atomicAdd(buf, 1);
    }
    off = __shfl_sync(0xffffffffu, off, 0);
    if (off + REC_HEAD + L > cap) return;  // the host sees the words needed and reports them
    int* r = buf + off;
    if (lane < REC_HEAD) {
        const unsigned long long nl = (unsigned long long)__double_as_longlong(it.newlen);
        const int v[REC_HEAD] = {a, it.s, it.P, it.M, it.start, L, (int)(unsigned)nl, (int)(unsigned)(nl >> 32),
                                 (int)(unsigned)it.fix_lo, (int)(unsigned)(it.fix_lo >> 32),
                                 (int)(unsigned)it.fix_hi, (int)(unsigned)(it.fix_hi >> 32)};
        r[lane] = v[lane];
    }
    const int* S = seg + (size_t)a * n;
    for (int t = lane; t < L; t += 32) r[REC_HEAD + t] = S[t];
}

// Ants outside the rank's range commit nothing unless a record says so.
__global__ void clear_foreign_kernel(int m, int ant0, int ant1, AntIter* __restrict__ antit) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x)
        if (a < ant0 || a >= ant1) {
            antit[a].newlen = INFINITY;
            antit[a].s = -1;
        }
}

// One thread lists where every record starts (in buffer order); at most m records.
__global__ void index_records_kernel(const int* __restrict__ bufs, int count, long long stride, int n, int m,
                                     long long* __restrict__ rec_off, int* __restrict__ nrec,
                                     int* __restrict__ errflag) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int total = 0;
    for (int b = 0; b < count; ++b) {
        const int* B = bufs + (size_t)b * stride;
        const int recs = B[0];
        const long long used = *reinterpret_cast<const long long*>(B + 2) ;
        if (recs < 0 || used < 4 || used > stride) { atomicOr(errflag, DEVERR_BAD_RECORD); break; }
        long long pos = 4;
        for (int r = 0; r < recs; ++r) {
            if (pos + REC_HEAD > used || total >= m) { atomicOr(errflag, DEVERR_BAD_RECORD); b = count; break; }
            const int L = B[pos + 5];
            if (L < 1 || L > n || pos + REC_HEAD + L > used) { atomicOr(errflag, DEVERR_BAD_RECORD); b = count; break; }
            rec_off[total++] = (long long)b * stride + pos;
            pos += REC_HEAD + L;
        }
    }
    *nrec = total;
}

// One warp per record: the ant's iteration record and its segment.
__global__ void __launch_bounds__(32) apply_records_kernel(const int* __restrict__ bufs, const long long* __restrict__ rec_off,
                                                           const int* __restrict__ nrec, int n, int m, int ant0, int ant1,
                                                           AntIter* __restrict__ antit, int* __restrict__ seg,
                                                           int* __restrict__ errflag) {
    if ((int)blockIdx.x >= *nrec) return;
    const int* r = bufs + rec_off[blockIdx.x];
    const int a = r[0], L = r[5];
    if (a < 0 || a >= m) {
        if (threadIdx.x == 0) atomicOr(errflag, DEVERR_BAD_RECORD);
        return;
    }
    if (a >= ant0 && a < ant1) return;  // the rank's own ant: already in place
    if (threadIdx.x == 0) {
        AntIter it;
        it.s = r[1];
        it.P = r[2];
        it.M = r[3];
        it.start = r[4];
        it.newlen = __longlong_as_double((long long)(((unsigned long long)(unsigned)r[7] << 32) | (unsigned)r[6]));
        it.fix_lo = ((unsigned long long)(unsigned)r[9] << 32) | (unsigned)r[8];
        it.fix_hi = ((unsigned long long)(unsigned)r[11] << 32) | (unsigned)r[10];
        const bool ok = it.s >= 0 ? (it.M >= 1 && it.M == L && it.P == n - it.M && it.s < n) : L == n;
        if (!ok) {
            atomicOr(errflag, DEVERR_BAD_RECORD);
            it.newlen = INFINITY;
        }
        antit[a] = it;
    }
    int* S = seg + (size_t)a * n;
    for (int t = threadIdx.x; t < L; t += 32) {
        const int c = r[REC_HEAD + t];
        S[t] = (unsigned)c < (unsigned)n ? c : 0;
        if ((unsigned)c >= (unsigned)n) atomicOr(errflag, DEVERR_BAD_RECORD);
    }
}

extern "C" aco_status aco_set_ant_range(aco_instance* inst, int32_t ant_begin, int32_t ant_end) {
    if (!inst) return ACO_ERR_INVALID_ARG;
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "set_ant_range: LBEST mode only");
    if (inst->in_batch) return set_err(inst, ACO_ERR_STATE, "set_ant_range: not for an instance of a batch");
    if (inst->constructed) return set_err(inst, ACO_ERR_STATE, "set_ant_range: tours constructed, update pending");
    if (!(0 <= ant_begin && ant_begin < ant_end && ant_end <= inst->p.m))
        return set_err(inst, ACO_ERR_INVALID_ARG, "set_ant_range: need 0 <= begin < end <= m");
    const bool whole = ant_begin == 0 && ant_end == inst->p.m;
    if (!whole && (inst->ls_p > 0.0 || inst->async_share))
        return set_err(inst, ACO_ERR_STATE, "set_ant_range: local search and asynchronous sharing need the whole colony");
    inst->ant0 = ant_begin;
    inst->ant1 = ant_end;
    return ACO_OK;
}

extern "C" aco_status aco_export_commits(aco_instance* inst, int32_t* buf_dev, int64_t cap_words, int64_t* words_out) {
    ACO_RANGE("aco_export_commits");
    if (!inst || !buf_dev || !words_out || cap_words < 4) return ACO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(buf_dev) & 7) return set_err(inst, ACO_ERR_INVALID_ARG, "export_commits: buffer not 8-byte aligned");
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "export_commits: LBEST mode only");
    if (!inst->constructed) return set_err(inst, ACO_ERR_STATE, "export_commits: no construction to export");
    cudaStream_t s = inst->stream;
    const long long head[2] = {0, 4};  // records (int32 in word 0, word 1 unused), words used (int64 in words 2-3)
    cudaMemcpyAsync(buf_dev, head, sizeof(head), cudaMemcpyHostToDevice, s);
    const int ants = inst->ant1 - inst->ant0;
    export_commits_kernel<<<ants, 32, 0, s>>>(inst->p.n, inst->ant0, inst->antit, inst->clen, inst->seg, buf_dev,
                                              (long long)cap_words);
    aco_status st = check_launch(inst, "export_commits_kernel");
    if (st != ACO_OK) return st;
    long long got[2] = {0, 0};
    cudaMemcpyAsync(got, buf_dev, sizeof(got), cudaMemcpyDeviceToHost, s);
    st = sync_and_check(inst, "export_commits");
    if (st != ACO_OK) return st;
    *words_out = got[1];
    if (got[1] > cap_words)
        return set_err(inst, ACO_ERR_INVALID_ARG, "export_commits: the records need %lld words, the buffer holds %lld",
                       got[1], (long long)cap_words);
    return ACO_OK;
}

extern "C" aco_status aco_import_commits(aco_instance* inst, const int32_t* bufs_dev, int32_t count,
                                         int64_t stride_words) {
    ACO_RANGE("aco_import_commits");
    if (!inst || !bufs_dev || count < 1 || stride_words < 4) return ACO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(bufs_dev) & 7 || (stride_words & 1))
        return set_err(inst, ACO_ERR_INVALID_ARG, "import_commits: buffers must be 8-byte aligned, stride even");
    if (inst->p.mode != ACO_MODE_LBEST_PARTIAL) return set_err(inst, ACO_ERR_STATE, "import_commits: LBEST mode only");
    if (!inst->constructed) return set_err(inst, ACO_ERR_STATE, "import_commits: construct first");
    cudaStream_t s = inst->stream;
    const int m = inst->p.m;
    clear_foreign_kernel<<<ceil_div(m, 256), 256, 0, s>>>(m, inst->ant0, inst->ant1, inst->antit);
    index_records_kernel<<<1, 1, 0, s>>>(bufs_dev, count, (long long)stride_words, inst->p.n, m, inst->rec_off,
                                         inst->nrec, inst->errflag);
    apply_records_kernel<<<m, 32, 0, s>>>(bufs_dev, inst->rec_off, inst->nrec, inst->p.n, m, inst->ant0, inst->ant1,
                                          inst->antit, inst->seg, inst->errflag);
    return check_launch(inst, "import_commits");
}

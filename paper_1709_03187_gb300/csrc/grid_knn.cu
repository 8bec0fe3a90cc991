// grid_knn.cu -- uniform grid over the cities and the exact k-nearest-neighbour candidate
// lists (the ACS candidate lists cited in Section 6), fused with the heuristic table
// eta^beta = (1/d)^beta of every candidate edge (Section 2).
//
// Grid: about two cities per cell over the bounding box; cities are counting-sorted by cell
// (city ids and coordinates in cell order).  A query scans Chebyshev rings of cells around its
// own cell and stops once the k-th best key (d^2, j) lies strictly inside a conservative lower
// bound of the distance to every unscanned cell.  The result is the unique list of the k
// smallest keys, identical to a brute-force sort.
#include <float.h>
#include <math.h>

#include "common.cuh"

#define FULL 0xffffffffu


__global__ void grid_count_kernel(const double* __restrict__ xy, int n, const GridDesc* __restrict__ gd,
                                  int* __restrict__ city_cell, int* __restrict__ cell_fill) {
    const GridDesc g = *gd;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cx = cell_coord(xy[2 * i], g.xmin, g.h, g.gx);
        const int cy = cell_coord(xy[2 * i + 1], g.ymin, g.h, g.gy);
        const int c = cy * g.gx + cx;
        city_cell[i] = c;
        atomicAdd(&cell_fill[c], 1);
    }
}

// Exclusive scan of cnt[0..len) into out[0..len] with one block (len up to a few million).
__global__ void scan_single_block_kernel(const int* __restrict__ cnt, int len, int* __restrict__ out) {
    __shared__ int part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (len + T - 1) / T;
    const int b = min(len, t * chunk), e = min(len, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;  // exclusive prefix of this chunk
    for (int i = b; i < e; ++i) {
        out[i] = run;
        run += cnt[i];
    }
    if (t == T - 1) out[len] = part[T - 1];
}

__global__ void grid_scatter_kernel(const double* __restrict__ xy, int n, const int* __restrict__ city_cell,
                                    const int* __restrict__ cell_start, int* __restrict__ cell_fill,
                                    int* __restrict__ cell_city, double* __restrict__ cell_xy) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = city_cell[i];
        const int pos = cell_start[c] + atomicAdd(&cell_fill[c], 1);
        cell_city[pos] = i;
        cell_xy[2 * pos] = xy[2 * i];
        cell_xy[2 * pos + 1] = xy[2 * i + 1];
    }
}

// Cell of the `idx`-th cell on Chebyshev ring r around (cx, cy); returns -1 outside the grid.
__device__ __forceinline__ int ring_cell(const GridDesc& g, int cx, int cy, int r, int idx) {
    int x, y;
    if (r == 0) {
        x = cx; y = cy;
    } else if (idx < 2 * r + 1) {
        x = cx - r + idx; y = cy - r;
    } else if (idx < 4 * r + 2) {
        x = cx - r + (idx - 2 * r - 1); y = cy + r;
    } else if (idx < 6 * r + 1) {
        x = cx - r; y = cy - r + 1 + (idx - 4 * r - 2);
    } else {
        x = cx + r; y = cy - r + 1 + (idx - 6 * r - 1);
    }
    if (x < 0 || y < 0 || x >= g.gx || y >= g.gy) return -1;
    return y * g.gx + x;
}

// (d^2, index) order on the bit patterns of non-negative FP64 squared distances (the same order
// as the values), so that the comparisons run on the integer units.
__device__ __forceinline__ bool key_less_u(unsigned long long da, int ja, unsigned long long db, int jb) {
    return da < db || (da == db && ja < jb);
}

// One warp per query city.  LISTS_ONLY: write the candidate lists only (no weight tables).
template <bool LISTS_ONLY>
__global__ void __launch_bounds__(256) knn_kernel(const double* __restrict__ xy, const GridDesc* __restrict__ gd,
                                                  const int* __restrict__ city_cell, const int* __restrict__ cell_start,
                                                  const int* __restrict__ cell_city, const double* __restrict__ cell_xy,
                                                  int n, int k, double beta, int* __restrict__ cand,
                                                  CandW* __restrict__ candw, double* __restrict__ etab,
                                                  int* __restrict__ errflag) {
    const GridDesc g = *gd;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const double qx = xy[2 * i], qy = xy[2 * i + 1];
        const int cell = city_cell[i];
        const int cx = cell % g.gx, cy = cell / g.gx;
        // this lane's list entry (lanes < k), sorted ascending; keys are the bit patterns of the
        // non-negative FP64 squared distances (the same order), compared on the integer units
        unsigned long long ld = ~0ull;
        int lj = 0x7fffffff;
        unsigned long long kd = ~0ull;
        int kj = 0x7fffffff;
        for (int r = 0;; ++r) {
            const int ncell = r == 0 ? 1 : 8 * r;
            for (int c0 = 0; c0 < ncell; c0 += 32) {
                int pb = 0, pe = 0;
                if (c0 + lane < ncell) {
                    const int c = ring_cell(g, cx, cy, r, c0 + lane);
                    if (c >= 0) { pb = cell_start[c]; pe = cell_start[c + 1]; }
                }
                while (__any_sync(FULL, pb < pe)) {
                    unsigned long long d2 = ~0ull;
                    int j = 0x7fffffff;
                    bool cand_ok = false;
                    if (pb < pe) {
                        j = cell_city[pb];
                        d2 = (unsigned long long)__double_as_longlong(
                            dist2(qx, qy, cell_xy[2 * pb], cell_xy[2 * pb + 1]));
                        cand_ok = (j != i) && key_less_u(d2, j, kd, kj);
                        ++pb;
                    }
                    unsigned pend = __ballot_sync(FULL, cand_ok);
                    while (pend) {
                        const int src = __ffs(pend) - 1;
                        pend &= pend - 1;
                        const unsigned long long cd = __shfl_sync(FULL, d2, src);
                        const int cj = __shfl_sync(FULL, j, src);
                        if (key_less_u(cd, cj, kd, kj)) {
                            const bool before = lane < k && key_less_u(ld, lj, cd, cj);
                            const int pos = __popc(__ballot_sync(FULL, before));
                            const unsigned long long ud = __shfl_up_sync(FULL, ld, 1);
                            const int uj = __shfl_up_sync(FULL, lj, 1);
                            if (lane == pos) { ld = cd; lj = cj; }
                            else if (lane > pos) { ld = ud; lj = uj; }
                            kd = __shfl_sync(FULL, ld, k - 1);
                            kj = __shfl_sync(FULL, lj, k - 1);
                        }
                    }
                }
            }
            const double lb = ring_lower_bound(g, qx, qy, cx, cy, r);
            if (lb < 0.0) break;  // every cell scanned
            // nothing unscanned can enter the list
            if (kd != ~0ull && __longlong_as_double((long long)kd) < __dmul_rn(lb, lb)) break;
        }
        if (lane < k) {
            const double ldd = __longlong_as_double((long long)ld);
            cand[(size_t)i * k + lane] = lj;
            if (ldd == 0.0) atomicOr(errflag, DEVERR_DUPLICATE);
            if (!LISTS_ONLY) {
                candw[(size_t)i * k + lane].city = lj;
                const double e = eta_pow_from_d2(ldd, beta);
                if (!isfinite(e)) atomicOr(errflag, DEVERR_NONFINITE);
                etab[(size_t)i * k + lane] = e;
            }
        }
    }
}

// Dense mode: eta^beta for every ordered pair and tau = tau0.
// The ACO_KF nearest other cities of every city, key (d^2, index) ascending, one warp per query
// city, by the same ring scan as knn_kernel; the sorted list is spread over the lanes, entry p in
// lane p % 32 of slot p / 32, and an entry that enters it shifts the later ones up by one.
__global__ void __launch_bounds__(256) knn_far_kernel(const double* __restrict__ xy, const GridDesc* __restrict__ gd,
                                                      const int* __restrict__ city_cell,
                                                      const int* __restrict__ cell_start,
                                                      const int* __restrict__ cell_city,
                                                      const double* __restrict__ cell_xy, int n,
                                                      int* __restrict__ far) {
    constexpr int S = ACO_KF / 32;
    const GridDesc g = *gd;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const double qx = xy[2 * i], qy = xy[2 * i + 1];
        const int cell = city_cell[i];
        const int cx = cell % g.gx, cy = cell / g.gx;
        // keys are the bit patterns of the non-negative FP64 squared distances, which order as
        // the values do, so the comparisons run on the integer units
        unsigned long long ld[S];
        int lj[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            ld[s] = ~0ull;
            lj[s] = 0x7fffffff;
        }
        unsigned long long kd = ~0ull;  // the last entry of the list
        int kj = 0x7fffffff;
        for (int r = 0;; ++r) {
            const int ncell = r == 0 ? 1 : 8 * r;
            for (int c0 = 0; c0 < ncell; c0 += 32) {
                int pb = 0, pe = 0;
                if (c0 + lane < ncell) {
                    const int c = ring_cell(g, cx, cy, r, c0 + lane);
                    if (c >= 0) { pb = cell_start[c]; pe = cell_start[c + 1]; }
                }
                while (__any_sync(FULL, pb < pe)) {
                    unsigned long long d2 = ~0ull;
                    int j = 0x7fffffff;
                    bool cand_ok = false;
                    if (pb < pe) {
                        j = cell_city[pb];
                        d2 = (unsigned long long)__double_as_longlong(
                            dist2(qx, qy, cell_xy[2 * pb], cell_xy[2 * pb + 1]));
                        cand_ok = (j != i) && key_less_u(d2, j, kd, kj);
                        ++pb;
                    }
                    unsigned pend = __ballot_sync(FULL, cand_ok);
                    while (pend) {
                        const int src = __ffs(pend) - 1;
                        pend &= pend - 1;
                        const unsigned long long cd = __shfl_sync(FULL, d2, src);
                        const int cj = __shfl_sync(FULL, j, src);
                        if (!key_less_u(cd, cj, kd, kj)) continue;
                        int pos = 0;
#pragma unroll
                        for (int s = 0; s < S; ++s)
                            pos += __popc(__ballot_sync(FULL, key_less_u(ld[s], lj[s], cd, cj)));
                        // the entry before each position, read before any entry moves
                        unsigned long long ud[S];
                        int uj[S];
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            ud[s] = __shfl_up_sync(FULL, ld[s], 1);
                            uj[s] = __shfl_up_sync(FULL, lj[s], 1);
                            if (s > 0) {
                                const unsigned long long pd = __shfl_sync(FULL, ld[s - 1], 31);
                                const int pj = __shfl_sync(FULL, lj[s - 1], 31);
                                if (lane == 0) {
                                    ud[s] = pd;
                                    uj[s] = pj;
                                }
                            }
                        }
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            const int p = 32 * s + lane;
                            if (p == pos) {
                                ld[s] = cd;
                                lj[s] = cj;
                            } else if (p > pos) {
                                ld[s] = ud[s];
                                lj[s] = uj[s];
                            }
                        }
                        kd = __shfl_sync(FULL, ld[S - 1], 31);
                        kj = __shfl_sync(FULL, lj[S - 1], 31);
                    }
                }
            }
            const double lb = ring_lower_bound(g, qx, qy, cx, cy, r);
            if (lb < 0.0) break;  // every cell scanned
            // nothing unscanned can enter the list
            if (kd != ~0ull && __longlong_as_double((long long)kd) < __dmul_rn(lb, lb)) break;
        }
#pragma unroll
        for (int s = 0; s < S; ++s) far[(size_t)i * ACO_KF + 32 * s + lane] = lj[s];
    }
}

// The extended lists as the prefix of the far lists.
__global__ void ext_from_far_kernel(const int* __restrict__ far, int n, int kx, int* __restrict__ ext) {
    const long long total = (long long)n * kx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        ext[e] = far[(e / kx) * ACO_KF + e % kx];
}

__global__ void dense_eta_kernel(const double* __restrict__ xy, int n, double beta, double tau0,
                                 double* __restrict__ etab_d, double* __restrict__ tau, int* __restrict__ errflag) {
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        tau[e] = tau0;
        if (i == j) { etab_d[e] = 0.0; continue; }
        const double d2 = dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1]);
        if (d2 == 0.0) atomicOr(errflag, DEVERR_DUPLICATE);
        const double v = eta_pow_from_d2(d2, beta);
        if (!isfinite(v)) atomicOr(errflag, DEVERR_NONFINITE);
        etab_d[e] = v;
    }
}

// Candidate lists, their screen entries and eta^beta from the first k entries of the extended
// lists (the same (d^2, index) keys, so the same lists knn_kernel<false> writes).
__global__ void cand_from_ext_kernel(const double* __restrict__ xy, int n, int k, int kx, double beta,
                                     const int* __restrict__ ext, int* __restrict__ cand, CandW* __restrict__ candw,
                                     double* __restrict__ etab, int* __restrict__ errflag) {
    const long long total = (long long)n * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / k), r = (int)(e % k);
        const int j = ext[(size_t)i * kx + r];
        cand[e] = j;
        candw[e].city = j;
        const double d2 = dist2(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1]);
        if (d2 == 0.0) atomicOr(errflag, DEVERR_DUPLICATE);
        const double v = eta_pow_from_d2(d2, beta);
        if (!isfinite(v)) atomicOr(errflag, DEVERR_NONFINITE);
        etab[e] = v;
    }
}

__global__ void xy32_kernel(const double* __restrict__ xy, int n, float2* __restrict__ xy32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        xy32[i] = make_float2(__double2float_rn(xy[2 * i]), __double2float_rn(xy[2 * i + 1]));
}

aco_status launch_build_grid_and_knn(aco_instance* inst) {
    const int n = inst->p.n;
    cudaStream_t s = inst->stream;
    if (inst->p.mode == ACO_MODE_DENSE) {
        const long long total = (long long)n * n;
        const int blocks = (int)fmin(4.0 * inst->num_sms * 8, (double)ceil_div(total, 256));
        dense_eta_kernel<<<blocks, 256, 0, s>>>(inst->xy, n, inst->p.beta, inst->p.tau0, inst->etab_d, inst->tau,
                                                inst->errflag);
        return check_launch(inst, "dense_eta_kernel");
    }
    const GridDesc& g = inst->grid;
    const int ncells = g.gx * g.gy;
    cudaMemsetAsync(inst->cell_fill, 0, sizeof(int) * ncells, s);
    const int blocks = (int)fmin((double)inst->num_sms * 8, (double)ceil_div(n, 256));
    xy32_kernel<<<blocks, 256, 0, s>>>(inst->xy, n, inst->xy32);
    grid_count_kernel<<<blocks, 256, 0, s>>>(inst->xy, n, inst->grid_dev, inst->city_cell, inst->cell_fill);
    scan_single_block_kernel<<<1, 1024, 0, s>>>(inst->cell_fill, ncells, inst->cell_start);
    cudaMemsetAsync(inst->cell_fill, 0, sizeof(int) * ncells, s);
    grid_scatter_kernel<<<blocks, 256, 0, s>>>(inst->xy, n, inst->city_cell, inst->cell_start, inst->cell_fill,
                                               inst->cell_city, inst->cell_xy);
    aco_status st = check_launch(inst, "grid build");
    if (st != ACO_OK) return st;
    const int warps_per_block = 8;
    const int kblocks = (int)fmin((double)inst->num_sms * 16, (double)ceil_div(n, warps_per_block));
    if (inst->ext) {
        // the kx nearest cities once (as the prefix of the far lists when the colony keeps them);
        // the candidate lists are their first k (the same keys)
        if (inst->far) {
            knn_far_kernel<<<kblocks, 32 * warps_per_block, 0, s>>>(inst->xy, inst->grid_dev, inst->city_cell,
                                                                   inst->cell_start, inst->cell_city, inst->cell_xy, n,
                                                                   inst->far);
            const long long te = (long long)n * inst->kx;
            ext_from_far_kernel<<<(int)fmin((double)inst->num_sms * 8, (double)ceil_div(te, 256)), 256, 0, s>>>(
                inst->far, n, inst->kx, inst->ext);
        } else {
            knn_kernel<true><<<kblocks, 32 * warps_per_block, 0, s>>>(inst->xy, inst->grid_dev, inst->city_cell,
                                                                      inst->cell_start, inst->cell_city, inst->cell_xy,
                                                                      n, inst->kx, 0.0, inst->ext, nullptr, nullptr,
                                                                      inst->errflag);
        }
        const long long total = (long long)n * inst->p.k;
        cand_from_ext_kernel<<<(int)fmin((double)inst->num_sms * 8, (double)ceil_div(total, 256)), 256, 0, s>>>(
            inst->xy, n, inst->p.k, inst->kx, inst->p.beta, inst->ext, inst->cand, inst->candw, inst->etab,
            inst->errflag);
        return check_launch(inst, "knn_kernel (extended lists)");
    }
    knn_kernel<false><<<kblocks, 32 * warps_per_block, 0, s>>>(inst->xy, inst->grid_dev, inst->city_cell, inst->cell_start,
                                                       inst->cell_city, inst->cell_xy, n, inst->p.k, inst->p.beta,
                                                       inst->cand, inst->candw, inst->etab, inst->errflag);
    return check_launch(inst, "knn_kernel");
}

// ---------------------------------------------------------------- device-only set-up
// Candidate lists from caller-provided scratch, with the grid sized on the device (no host
// staging of the coordinates).  Scratch layout (all 16-byte aligned):
//   GridDesc | errflag | city_cell[n] | cell_fill[cap] | cell_start[cap + 1] | cell_city[n] | cell_xy[2n]
__global__ void bbox_desc_kernel(const double* __restrict__ xy, int n, int cap_cells, GridDesc* __restrict__ gd,
                                 int* __restrict__ errflag) {
    __shared__ double sh[4][32];
    __shared__ int bad_s;
    if (threadIdx.x == 0) bad_s = 0;
    __syncthreads();
    double xmn = 1e308, xmx = -1e308, ymn = 1e308, ymx = -1e308;
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        bad |= !(isfinite(x) && isfinite(y));
        xmn = fmin(xmn, x); xmx = fmax(xmx, x); ymn = fmin(ymn, y); ymx = fmax(ymx, y);
    }
    if (bad) atomicOr(&bad_s, 1);
    for (int o = 16; o; o >>= 1) {
        xmn = fmin(xmn, __shfl_xor_sync(FULL, xmn, o));
        xmx = fmax(xmx, __shfl_xor_sync(FULL, xmx, o));
        ymn = fmin(ymn, __shfl_xor_sync(FULL, ymn, o));
        ymx = fmax(ymx, __shfl_xor_sync(FULL, ymx, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = xmn; sh[1][w] = xmx; sh[2][w] = ymn; sh[3][w] = ymx; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
        xmn = fmin(xmn, sh[0][i]); xmx = fmax(xmx, sh[1][i]); ymn = fmin(ymn, sh[2][i]); ymx = fmax(ymx, sh[3][i]);
    }
    if (bad_s) { atomicOr(errflag, DEVERR_NONFINITE); xmn = ymn = 0.0; xmx = ymx = 1.0; }
    // about two cities per cell over the bounding box, as on the host path
    GridDesc g;
    g.xmin = xmn; g.xmax = xmx; g.ymin = ymn; g.ymax = ymx;
    const double wx = fmax(xmx - xmn, 1e-300), wy = fmax(ymx - ymn, 1e-300);
    const double target = fmax(1.0, (double)(n / 2));
    double h = sqrt(wx * wy / target);
    if (!(h > 0)) h = fmax(wx, wy);
    h = fmax(h, fmax(wx, wy) / 4096.0);
    int gx = (int)fmin(4096.0, floor(wx / h) + 1), gy = (int)fmin(4096.0, floor(wy / h) + 1);
    while ((long long)gx * gy > cap_cells) {
        h *= 1.05;
        gx = (int)floor(wx / h) + 1;
        gy = (int)floor(wy / h) + 1;
    }
    g.h = h; g.gx = gx; g.gy = gy;
    g.margin = 1e-6 * h + 1e-14 * (fabs(xmn) + fabs(xmx) + fabs(ymn) + fabs(ymx));
    *gd = g;
}

__global__ void zero_ints_kernel(int* __restrict__ v, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) v[i] = 0;
}

static inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

size_t knn_scratch_bytes(int max_n) {
    const int cap = max_n / 2 + 16;
    return align16(sizeof(GridDesc)) + 16 + align16(sizeof(int) * (size_t)max_n) + align16(sizeof(int) * (size_t)cap) +
           align16(sizeof(int) * (size_t)(cap + 1)) + align16(sizeof(int) * (size_t)max_n) +
           align16(sizeof(double) * 2 * (size_t)max_n);
}

// Runs the whole candidate-list build on `scratch` (knn_scratch_bytes(n) bytes) and leaves the
// device error flags (DEVERR_*) at scratch + align16(sizeof(GridDesc)).
cudaError_t launch_knn_on_scratch(const double* xy, int n, int k, int32_t* cand, unsigned char* scratch,
                                  int num_sms, cudaStream_t s) {
    const int cap = n / 2 + 16;
    unsigned char* p = scratch;
    GridDesc* gd = reinterpret_cast<GridDesc*>(p); p += align16(sizeof(GridDesc));
    int* errflag = reinterpret_cast<int*>(p); p += 16;
    int* city_cell = reinterpret_cast<int*>(p); p += align16(sizeof(int) * (size_t)n);
    int* cell_fill = reinterpret_cast<int*>(p); p += align16(sizeof(int) * (size_t)cap);
    int* cell_start = reinterpret_cast<int*>(p); p += align16(sizeof(int) * (size_t)(cap + 1));
    int* cell_city = reinterpret_cast<int*>(p); p += align16(sizeof(int) * (size_t)n);
    double* cell_xy = reinterpret_cast<double*>(p);
    zero_ints_kernel<<<1, 32, 0, s>>>(errflag, 1);
    bbox_desc_kernel<<<1, 1024, 0, s>>>(xy, n, cap, gd, errflag);
    const int blocks = (int)fmin((double)num_sms * 8, (double)ceil_div(n, 256));
    zero_ints_kernel<<<ceil_div(cap, 256), 256, 0, s>>>(cell_fill, cap);
    grid_count_kernel<<<blocks, 256, 0, s>>>(xy, n, gd, city_cell, cell_fill);
    scan_single_block_kernel<<<1, 1024, 0, s>>>(cell_fill, cap, cell_start);
    zero_ints_kernel<<<ceil_div(cap, 256), 256, 0, s>>>(cell_fill, cap);
    grid_scatter_kernel<<<blocks, 256, 0, s>>>(xy, n, city_cell, cell_start, cell_fill, cell_city, cell_xy);
    const int kblocks = (int)fmin((double)num_sms * 16, (double)ceil_div(n, 8));
    knn_kernel<true><<<kblocks, 256, 0, s>>>(xy, gd, city_cell, cell_start, cell_city, cell_xy, n, k, 0.0, cand,
                                              nullptr, nullptr, errflag);
    return cudaGetLastError();
}

// Cities per coarse block of ACO_CBLK x ACO_CBLK grid cells (the nearest-unvisited search of full
// constructions skips empty blocks).
__global__ void coarse_size_kernel(const int* __restrict__ cell_start, int gx, int gy, int cgx, int ncoarse,
                                   int* __restrict__ csize) {
    for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < ncoarse; C += gridDim.x * blockDim.x) {
        const int X0 = (C % cgx) * ACO_CBLK, Y0 = (C / cgx) * ACO_CBLK;
        int sum = 0;
        for (int y = Y0; y < Y0 + ACO_CBLK && y < gy; ++y)
            for (int x = X0; x < X0 + ACO_CBLK && x < gx; ++x) sum += cell_start[y * gx + x + 1] - cell_start[y * gx + x];
        csize[C] = sum;
    }
}

aco_status launch_coarse_sizes(aco_instance* inst) {
    coarse_size_kernel<<<ceil_div(inst->ncoarse, 256), 256, 0, inst->stream>>>(
        inst->cell_start, inst->grid.gx, inst->grid.gy, inst->cgx, inst->ncoarse, inst->csize);
    return check_launch(inst, "coarse_size_kernel");
}

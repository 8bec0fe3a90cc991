/* Drives the CPU oracle through every mode on small colonies, for a build with AddressSanitizer
 * and UndefinedBehaviorSanitizer (tests/test_oracle_sanitize.py compiles and runs it): a memory
 * error or undefined behaviour anywhere on these paths makes the program fail.  Test code only. */
#include "../oracle/aco_oracle.c"

#include <stdio.h>

static void fill_xy(double* xy, int n, unsigned seed) {
    uint32_t key[2] = {seed, 7u}, out[4];
    for (int i = 0; i < n; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, 0u, 9u};
        or_philox4x32_10(ctr, key, out);
        xy[2 * i] = or_u53(out[0], out[1]);
        xy[2 * i + 1] = or_u53(out[2], out[3]);
    }
}

static int run_colony(int mode, int n, int m, int k, double f, double p_partial, int fallback, int selection,
                      int iters, int threads, double ls_p) {
    double* xy = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    fill_xy(xy, n, (unsigned)(n * 31 + m));
    or_params p = {mode, n, m, k, 1.0, 2.0, 0.5, 1.0, f, p_partial, 5, fallback, selection};
    or_state* st = or_create(&p, xy);
    if (!st) return 1;
    if (ls_p > 0.0) or_set_local_search(st, ls_p, 40);
    for (int it = 0; it < iters; ++it) {
        or_construct_mt(st, it, NULL, 0, 1, threads);
        or_update(st);
    }
    int32_t* lb = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
    double* cl = (double*)malloc(sizeof(double) * (size_t)m);
    if (mode == 1) {
        or_get_lbest(st, lb);
        or_get_clen(st, cl);
        /* the exhausted-list rule at every city with a random visited set */
        unsigned char* vis = (unsigned char*)calloc((size_t)n, 1);
        double* w = (double*)malloc(sizeof(double) * (size_t)n);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) vis[j] = (unsigned char)((i * 7 + j * 3) % 5 == 0);
            vis[i] = 1;
            vis[(i + 1) % n] = 0;
            if (or_exhausted_step(st, i, vis, 0.37, w) < 0) return 2;
        }
        free(vis);
        free(w);
        double W[4096];
        uint64_t Q[4096], q[64];
        if ((size_t)n * k <= 4096 && m <= 64) or_cand_weights(st, W, Q, q);
    }
    free(lb);
    free(cl);
    or_destroy(st);
    free(xy);
    return 0;
}

int main(void) {
    int rc = 0;
    rc |= run_colony(0, 40, 12, 0, 1.0, 1.0, 0, 0, 4, 1, 0.0);    /* Section 2 dense form */
    rc |= run_colony(1, 120, 16, 8, 0.3, 1.0, 0, 0, 6, 1, 0.0);   /* PartialACO, argmax fallback */
    rc |= run_colony(1, 90, 10, 5, 0.5, 0.6, 1, 0, 5, 3, 0.0);    /* wheel fallback, full tours, threads */
    rc |= run_colony(1, 100, 8, 6, 0.4, 1.0, 0, 1, 5, 2, 0.0);    /* Independent Roulette */
    rc |= run_colony(1, 150, 8, 6, 0.5, 1.0, 0, 0, 4, 1, 0.5);    /* windowed 2-opt */
    rc |= run_colony(1, 3, 4, 2, 1.0, 1.0, 0, 0, 3, 1, 0.0);      /* the smallest instance */
    int32_t cand[200 * 8];
    double xy[400];
    fill_xy(xy, 200, 3u);
    rc |= or_knn_sweep(200, xy, 8, cand) != 0;
    printf("oracle sanitizer run: %s\n", rc ? "FAILED" : "ok");
    return rc;
}

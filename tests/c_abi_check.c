/* A C99 client of include/hylu.h, built and run by tests/test_c_abi.py: it
 * includes nothing of the library but the header, links libhylu.so and calls
 * the entry points that need no GPU (analysis, info, exports, the analysis
 * checkpoint, the empty system and error codes).  It prints one line per
 * check and exits non-zero on the first failure. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hylu.h"

#define CHECK(cond, what)                                   \
    do {                                                    \
        if (!(cond)) {                                      \
            fprintf(stderr, "FAILED: %s\n", what);          \
            return 1;                                       \
        }                                                   \
        printf("ok: %s\n", what);                           \
    } while (0)

/* k x k 5-point grid with an unsymmetric perturbation, CSR with sorted columns */
static int32_t grid(int32_t k, int64_t* rp, int32_t* ci, double* v) {
    int32_t n = k * k;
    int64_t q = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t x = i % k, y = i / k;
        rp[i] = q;
        if (y > 0) { ci[q] = i - k; v[q++] = -1.0; }
        if (x > 0) { ci[q] = i - 1; v[q++] = -1.1; }
        ci[q] = i; v[q++] = 4.05;
        if (x < k - 1) { ci[q] = i + 1; v[q++] = -0.9; }
        if (y < k - 1) { ci[q] = i + k; v[q++] = -1.0; }
    }
    rp[n] = q;
    return n;
}

int main(void) {
    enum { K = 12, N = K * K, NNZ = 5 * N };
    static int64_t rp[N + 1];
    static int32_t ci[NNZ];
    static double v[NNZ];
    const int32_t n = grid(K, rp, ci, v);

    hylu_options opt;
    CHECK(hylu_default_options(&opt) == HYLU_OK && opt.ordering == HYLU_ORDER_AMD && opt.sn_max == 256,
          "default options");
    CHECK(hylu_default_options(NULL) == HYLU_ERR_ARG, "default options refuse NULL");

    hylu_handle* h = NULL;
    CHECK(hylu_analyze(n, rp[n], rp, ci, v, NULL, &opt, &h) == HYLU_OK && h != NULL, "analyze");
    hylu_info info;
    CHECK(hylu_get_info(h, &info) == HYLU_OK && info.n == n && info.nnz_a == rp[n], "info sizes");
    CHECK(info.flops > 0.0 && info.flops_padded >= info.flops, "info flop counts");
    CHECK(info.flops_row_row + info.flops_sup_row + info.flops_sup_sup + info.flops_in_supernode ==
              info.flops_padded,
          "kernel split sums to the padded flops");
    CHECK(info.ordering == HYLU_ORDER_AMD, "info ordering");

    int32_t* rowperm = malloc(sizeof(int32_t) * n);
    int32_t* colperm = malloc(sizeof(int32_t) * n);
    int32_t* sn = malloc(sizeof(int32_t) * (info.nnodes + 1));
    int64_t* prp = malloc(sizeof(int64_t) * (n + 1));
    int32_t* pci = malloc(sizeof(int32_t) * info.nnz_store);
    CHECK(hylu_export_perm(h, rowperm, colperm, NULL, NULL, sn) == HYLU_OK, "export permutations");
    {
        char* seen = calloc(n, 1);
        int ok = 1;
        for (int32_t i = 0; i < n; ++i) {
            if (colperm[i] < 0 || colperm[i] >= n || seen[colperm[i]]) ok = 0;
            else seen[colperm[i]] = 1;
        }
        free(seen);
        CHECK(ok && sn[0] == 0 && sn[info.nnodes] == n, "column permutation and partition");
    }
    CHECK(hylu_export_pattern(h, prp, pci) == HYLU_OK && prp[n] == info.nnz_store, "export pattern");

    /* checkpoint: size query, too small a buffer, save, load, same pattern */
    int64_t bytes = 0;
    CHECK(hylu_plan_save(h, NULL, &bytes) == HYLU_OK && bytes > 0, "plan size query");
    unsigned char* img = malloc((size_t)bytes);
    int64_t small = bytes - 1;
    CHECK(hylu_plan_save(h, img, &small) == HYLU_ERR_ARG && small == bytes, "plan buffer too small");
    CHECK(hylu_plan_save(h, img, &bytes) == HYLU_OK, "plan save");
    hylu_handle* h2 = NULL;
    CHECK(hylu_plan_load(img, bytes, NULL, &h2) == HYLU_OK && h2 != NULL, "plan load");
    {
        hylu_info i2;
        int64_t* prp2 = malloc(sizeof(int64_t) * (n + 1));
        int32_t* pci2 = malloc(sizeof(int32_t) * info.nnz_store);
        CHECK(hylu_get_info(h2, &i2) == HYLU_OK && i2.nnz_store == info.nnz_store && i2.flops == info.flops,
              "loaded plan info");
        CHECK(hylu_export_pattern(h2, prp2, pci2) == HYLU_OK &&
                  memcmp(prp, prp2, sizeof(int64_t) * (n + 1)) == 0 &&
                  memcmp(pci, pci2, sizeof(int32_t) * info.nnz_store) == 0,
              "loaded plan pattern");
        free(prp2);
        free(pci2);
    }
    img[bytes / 2] ^= 0x10;
    hylu_handle* h3 = NULL;
    CHECK(hylu_plan_load(img, bytes, NULL, &h3) == HYLU_ERR_PATTERN && h3 == NULL, "damaged image refused");

    /* order of calls and arguments */
    CHECK(hylu_solve(h, NULL, NULL, 1, n, NULL) == HYLU_ERR_STATE, "solve before factor");
    CHECK(hylu_factor(NULL, NULL, NULL) == HYLU_ERR_ARG, "factor without a handle");
    opt.ordering = 9;
    hylu_handle* h4 = NULL;
    CHECK(hylu_analyze(n, rp[n], rp, ci, v, NULL, &opt, &h4) == HYLU_ERR_ARG && h4 == NULL, "bad ordering");
    opt.ordering = HYLU_ORDER_AMD;
    ci[1] = ci[0];   /* duplicate column */
    CHECK(hylu_analyze(n, rp[n], rp, ci, v, NULL, &opt, &h4) == HYLU_ERR_PATTERN, "duplicate column");

    /* the empty system needs no device */
    int64_t rp0[1] = {0};
    hylu_handle* e = NULL;
    const int64_t launches = hylu_launch_count();
    CHECK(hylu_analyze(0, 0, rp0, NULL, v, NULL, &opt, &e) == HYLU_OK, "empty analyze");
    CHECK(hylu_factor(e, NULL, NULL) == HYLU_OK && hylu_solve(e, NULL, NULL, 1, 0, NULL) == HYLU_OK &&
              hylu_solve_transpose(e, NULL, NULL, 2, 0, NULL) == HYLU_OK,
          "empty factor and solves");
    CHECK(hylu_launch_count() == launches, "no kernel launched");

    CHECK(hylu_destroy(e) == HYLU_OK && hylu_destroy(h2) == HYLU_OK && hylu_destroy(h) == HYLU_OK &&
              hylu_destroy(NULL) == HYLU_OK,
          "destroy");
    free(rowperm); free(colperm); free(sn); free(prp); free(pci); free(img);
    printf("all C ABI checks passed\n");
    return 0;
}

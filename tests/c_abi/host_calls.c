/* A plain C99 caller of the library's host entry points (no GPU calls):
 * the header must compile as C and the exported symbols must link and
 * behave as declared.  Prints one line per check; exit code 0 on success. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "slu.h"

#define CHECK(cond)                                                        \
    do {                                                                   \
        if (!(cond)) {                                                     \
            printf("FAILED %s (line %d): %s\n", #cond, __LINE__,           \
                   slu_last_error());                                      \
            return 1;                                                      \
        }                                                                  \
    } while (0)

int main(void) {
    /* 1-D Laplacian of order 50: tridiagonal, rows ascending per column */
    enum { N = 50 };
    int64_t colptr[N + 1];
    int32_t rowidx[3 * N];
    int64_t nnz = 0;
    for (int j = 0; j < N; ++j) {
        colptr[j] = nnz;
        for (int i = j - 1; i <= j + 1; ++i)
            if (i >= 0 && i < N) rowidx[nnz++] = i;
    }
    colptr[N] = nnz;

    slu_opts o;
    slu_opts_default(&o);
    CHECK(o.sample_points == 1000 && o.step == 2 && o.max_num == 3);
    o.b_min = 4;

    slu_plan *p = NULL;
    CHECK(slu_analyze(N, colptr, rowidx, &o, &p) == SLU_OK && p != NULL);
    slu_plan_info info;
    CHECK(slu_plan_query(p, &info) == SLU_OK);
    CHECK(slu_plan_check(p) == SLU_OK);
    /* no fill for a tridiagonal pattern; Algorithm 2 ends at nnz */
    CHECK(info.n == N && info.nnz_a == nnz && info.nnz_lu == nnz);
    CHECK(info.flops == 3 * (N - 1));          /* l_k = u_k = 1: 1 + 2 */
    int64_t *bp = malloc(sizeof(int64_t) * (N + 1));
    int64_t *ptr = malloc(sizeof(int64_t) * (info.nblocks_1d + 1));
    int64_t *cp = malloc(sizeof(int64_t) * (N + 1));
    int32_t *ri = malloc(sizeof(int32_t) * info.nnz_lu);
    CHECK(slu_plan_export(p, bp, ptr, cp, ri) == SLU_OK);
    for (int k = 1; k <= N; ++k) CHECK(bp[k] == 3 * k - 2);   /* closed form */
    CHECK(ptr[0] == 0 && ptr[info.nblocks_1d] == N);

    /* plan cache round trip */
    int64_t size = 0;
    CHECK(slu_plan_serialize(p, NULL, &size) == SLU_OK && size > 48);
    unsigned char *buf = malloc((size_t)size);
    int64_t small = size - 1;
    CHECK(slu_plan_serialize(p, buf, &small) == SLU_ERR_INVALID_ARG && small == size);
    CHECK(slu_plan_serialize(p, buf, &size) == SLU_OK);
    slu_plan *q = NULL;
    CHECK(slu_plan_deserialize(buf, size, &q) == SLU_OK && q != NULL);
    uint64_t d1 = 0, d2 = 0;
    CHECK(slu_plan_digest(p, &d1) == SLU_OK && slu_plan_digest(q, &d2) == SLU_OK);
    CHECK(d1 == d2);
    buf[size / 2] ^= 0x40;
    slu_plan *bad = (slu_plan *)1;
    CHECK(slu_plan_deserialize(buf, size, &bad) == SLU_ERR_INVALID_ARG && bad == NULL);

    /* the phase times add up to the analysis time */
    double sum = 0;
    for (int k = 0; k < SLU_PHASE_COUNT; ++k) {
        CHECK(info.phase_ms[k] >= 0);
        sum += info.phase_ms[k];
    }
    CHECK(sum <= info.analyze_ms * (1 + 1e-9) + 1e-6);

    /* device analysis: the plan of the host analysis, or SLU_ERR_CUDA when
     * the process has no GPU */
    slu_plan *dp = NULL;
    const slu_status ds = slu_analyze_device(N, colptr, rowidx, &o, NULL, &dp);
    CHECK(ds == SLU_OK || (ds == SLU_ERR_CUDA && dp == NULL));
    if (ds == SLU_OK) {
        uint64_t d3 = 0;
        CHECK(slu_plan_digest(dp, &d3) == SLU_OK && d3 == d1);
        slu_plan_destroy(dp);
    }

    /* errors are statuses with a message, never a crash */
    rowidx[1] = N;                              /* row out of range */
    slu_plan *dr = (slu_plan *)1;
    CHECK(slu_analyze_device(N, colptr, rowidx, &o, NULL, &dr) == SLU_ERR_INVALID_ARG &&
          dr == NULL);
    slu_plan *r = (slu_plan *)1;
    CHECK(slu_analyze(N, colptr, rowidx, &o, &r) == SLU_ERR_INVALID_ARG && r == NULL);
    CHECK(strstr(slu_last_error(), "out of range") != NULL);
    CHECK(slu_analyze(N, colptr, rowidx, &o, NULL) == SLU_ERR_INVALID_ARG);
    CHECK(slu_plan_query(NULL, &info) == SLU_ERR_INVALID_ARG);
    CHECK(slu_plan_check(NULL) == SLU_ERR_INVALID_ARG);

    slu_plan_destroy(q);
    slu_plan_destroy(p);
    slu_plan_destroy(NULL);
    free(buf); free(bp); free(ptr); free(cp); free(ri);
    printf("ok\n");
    return 0;
}

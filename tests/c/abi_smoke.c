/* A plain C11 program against include/ahs.h: create a lattice, initialise it,
 * take 20 leapfrog steps with a fused measurement every 10, read the records and
 * the fields, and exercise the error path.  Prints one line per check; exits
 * non-zero on the first failure.  Built and run by tests/test_c_abi.py. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "ahs.h"

#define CHECK(cond, what)                                                    \
    do {                                                                     \
        if (!(cond)) {                                                       \
            fprintf(stderr, "FAIL %s: %s\n", what, ahs_last_error_message()); \
            return 1;                                                        \
        }                                                                    \
        printf("ok %s\n", what);                                             \
    } while (0)

int main(void)
{
    const int N = 16;
    CHECK(ahs_sizeof_obs() == sizeof(ahs_obs_t), "record layout");
    CHECK(ahs_create(3, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, AHS_RADIATION) == NULL &&
              ahs_last_error() == AHS_EINVAL, "invalid lattice rejected");
    ahs_t *h = ahs_create(N, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, AHS_RADIATION);
    CHECK(h != NULL, "create");
    CHECK(ahs_step(h, 1) == AHS_ESTATE, "step before init refused");
    CHECK(ahs_set_option(h, AHS_OPT_MEASURE_EVERY, 10.0) == AHS_OK, "measure_every");
    CHECK(ahs_init(h, 7) == AHS_OK, "init");
    CHECK(ahs_step(h, 20) == AHS_OK, "20 steps");
    ahs_obs_t rec[4];
    int m = ahs_records(h, rec, 4);
    CHECK(m == 2 && rec[0].step == 0 && rec[1].step == 10, "two records");
    CHECK(rec[1].nonfinite == 0 && rec[1].e_total > 0.0 && rec[1].n_wind > 0, "record values");
    ahs_obs_t now;
    CHECK(ahs_measure(h, &now) == AHS_OK && now.step == 20 && isfinite(now.xi_l), "measure");
    size_t bytes = (size_t)10 * N * N * N * sizeof(float);
    float *F = (float *)malloc(bytes);
    CHECK(F != NULL && ahs_fields(h, AHS_FIELD_ALL, F, bytes) == AHS_OK, "fields");
    double m2 = 0.0;
    for (int i = 0; i < N * N * N; ++i) m2 += (double)F[i] * F[i] + (double)F[N * N * N + i] * F[N * N * N + i];
    CHECK(isfinite(m2) && m2 > 0.0 && m2 / (N * N * N) < 4.0, "|phi|^2 finite and bounded");
    CHECK(ahs_fields(h, AHS_FIELD_ALL, F, bytes - 4) == AHS_EINVAL, "wrong size refused");
    free(F);
    printf("xi_w %.6f xi_l %.6f e_total %.6f\n", now.xi_w, now.xi_l, now.e_total);
    ahs_destroy(h);

    /* a batch of two members of different size and era, run to their ends */
    const int bn[2] = {16, 12}, bera[2] = {AHS_RADIATION, AHS_MATTER};
    const uint64_t bseed[2] = {7, 8};
    const int64_t bend[2] = {20, 13};
    ahs_batch_t *b = ahs_batch_create(2, bn, bera, bseed, bend, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0);
    CHECK(b != NULL, "batch create");
    CHECK(ahs_batch_init(b) == AHS_OK, "batch init");
    CHECK(ahs_batch_run(b, 1000) == 20, "batch runs to the last member's end");
    int64_t bnow = 0, bstop = 0;
    CHECK(ahs_batch_step_info(b, 1, &bnow, &bstop) == AHS_OK && bnow == 13 && bstop == 13, "member stops at its end");
    ahs_obs_t brec[4];
    CHECK(ahs_batch_records(b, 0, brec, 4) == 2 && brec[1].step == 10, "member records");
    ahs_obs_t bm;
    CHECK(ahs_batch_measure(b, 1, &bm) == AHS_OK && bm.step == 13 && bm.nonfinite == 0, "member measure");
    CHECK(ahs_batch_records(b, 5, brec, 4) == AHS_EINVAL, "bad member refused");
    ahs_batch_destroy(b);
    return 0;
}

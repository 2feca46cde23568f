/* A plain C99 caller of the library's host-only entry points: the headers compile as C,
 * the shared library links, and a plan-only handle is built, queried and destroyed.
 * Problem: one sector (n=0, 2S_z=0, dim 2) on each side, target (0, 0), one Delta = 0
 * term with A = B = 2x2 blocks; its single contribution costs 2abc + 2acd = 32 flops
 * (a = b = c = d = 2, A-first on the tie).  Exit status 0 on success. */
#include <stdio.h>
#include <string.h>

#include "dmrg_heff.h"
#include "dmrg_profile.h"

static int fails = 0;
#define CHECK(cond)                                                 \
    do {                                                            \
        if (!(cond)) {                                              \
            fprintf(stderr, "check failed: %s (line %d)\n", #cond, __LINE__); \
            ++fails;                                                \
        }                                                           \
    } while (0)

int main(void) {
    CHECK(strlen(dmrg_strerror(DMRG_ERR_INVALID_ARG)) > 0);

    double w = 0.0; /* spin-1/2 dimer: S_L.S_R recoupling, singlet W = 1, triplet -1/3 */
    CHECK(dmrg_su2_recoupling(1, 1, 1, 1, 2, 0, &w) == DMRG_OK && w > 1.0 - 1e-14 && w < 1.0 + 1e-14);
    CHECK(dmrg_su2_recoupling(1, 1, 1, 1, 2, 2, &w) == DMRG_OK && w > -1.0 / 3 - 1e-14 && w < -1.0 / 3 + 1e-14);
    CHECK(dmrg_su2_recoupling(-1, 1, 1, 1, 2, 0, &w) == DMRG_ERR_INVALID_ARG);

    const int32_t table[3] = {0, 0, 2};
    const double coef[1] = {0.5};
    const int32_t delta[2] = {0, 0};
    const int32_t parity[1] = {0};
    const int64_t a_off[1] = {0}, b_off[1] = {4};
    const double op[8] = {1, 2, 3, 4, 5, 6, 7, 8};
    dmrg_heff_opts opts;
    memset(&opts, 0, sizeof(opts));
    opts.precision = DMRG_PREC_FP64;
    opts.max_nvec = 1;
    opts.flags = DMRG_FLAG_PLAN_ONLY;
    dmrg_heff_t h = NULL;
    CHECK(dmrg_heff_create(table, 1, table, 1, 0, 0, coef, delta, parity, a_off, b_off, 1, op, 8, &opts, &h) == DMRG_OK);
    CHECK(h != NULL);
    if (h) {
        int64_t flops = -1, rows = 0, plan[5];
        CHECK(dmrg_heff_dim(h) == 4);
        CHECK(dmrg_heff_flops(h, &flops) == DMRG_OK && flops == 32);
        CHECK(dmrg_heff_plan_dump(h, NULL, &rows) == DMRG_OK && rows == 1);
        CHECK(dmrg_heff_plan_dump(h, plan, &rows) == DMRG_OK && plan[0] == 0 && plan[1] == 0 && plan[2] == 0 &&
              plan[3] == 0 && plan[4] == 32);
        dmrg_heff_destroy(h);
    }
    /* a block offset past the end of op_data is refused, with a message */
    const int64_t bad_off[1] = {6};
    h = NULL;
    CHECK(dmrg_heff_create(table, 1, table, 1, 0, 0, coef, delta, parity, a_off, bad_off, 1, op, 8, &opts, &h) ==
          DMRG_ERR_INVALID_ARG);
    CHECK(h == NULL && strlen(dmrg_last_error()) > 0);
    if (fails == 0) printf("c abi ok\n");
    return fails == 0 ? 0 : 1;
}

/* A plain C99 program written against include/rlb.h and linked to librlb:
 * the boundary is usable from C, with no C++ or torch on the caller's side.
 * It makes only host-side calls (no GPU is needed): state layout and
 * workspace sizes, parameter validation before any CUDA call, status strings
 * and the last-error text.  Prints "ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "rlb.h"

static int fails = 0;
#define CHECK(c)                                                     \
    do {                                                             \
        if (!(c)) {                                                  \
            printf("FAIL line %d: %s\n", __LINE__, #c);              \
            ++fails;                                                 \
        }                                                            \
    } while (0)

int main(void) {
    rlb_params p;
    memset(&p, 0, sizeof p);
    /* the 3D shock on a sphere: 200 x 100 x 100, inflow beta_x = 0.5 */
    p.nx = 200;
    p.ny = 100;
    p.nz = 100;
    p.prec = RLB_FP32_DEV;
    p.xbc = RLB_BC_INFLOW_OUTFLOW;
    p.eos = RLB_EOS_ULTRA;
    p.tau = 0.8;
    p.c_l = 1.0;
    p.n_in = 1.0;
    p.eps_in = 1.0;
    p.beta_in[0] = 0.5;
    p.n_ref = 0.46;
    p.eps_ref = 1.0;

    int64_t stride = 0;
    int32_t elem = 0;
    size_t bytes = 0, ws = 0;
    CHECK(rlb_state_layout(&p, &stride, &elem, &bytes) == RLB_OK);
    CHECK(stride >= 2000000 && stride % 64 == 0 && elem == 4);
    CHECK(bytes == (size_t)38 * (size_t)stride * 4u);
    CHECK(rlb_workspace_bytes(&p, &ws) == RLB_OK && ws >= 2 * bytes);
    p.prec = RLB_FP64;
    CHECK(rlb_state_layout(&p, &stride, &elem, &bytes) == RLB_OK && elem == 8);
    CHECK(bytes == (size_t)38 * (size_t)stride * 8u);

    /* invalid parameters are refused before any CUDA call */
    rlb_ctx* ctx = NULL;
    p.tau = 0.5; /* tau > 1/2 */
    CHECK(rlb_create(&p, NULL, NULL, 0, &ctx) == RLB_ERR_ARG && ctx == NULL);
    CHECK(strlen(rlb_last_error(NULL)) > 0);
    p.tau = 0.8;
    p.nx = 2; /* a non-periodic lattice needs nx >= 3 */
    CHECK(rlb_create(&p, NULL, NULL, 0, &ctx) == RLB_ERR_ARG && ctx == NULL);
    p.nx = 200;
    p.prec = RLB_FP32_DEV;
    p.eos = RLB_EOS_GAMMA_LAW; /* the general equation of state is FP64 only */
    p.eos_gamma = 5.0 / 3.0;
    CHECK(rlb_create(&p, NULL, NULL, 0, &ctx) == RLB_ERR_ARG && ctx == NULL);
    CHECK(rlb_state_layout(NULL, &stride, &elem, &bytes) == RLB_ERR_ARG);

    /* sizes at the limit N <= 2^31 - 2^21 (all arithmetic in 64 bits) */
    p.eos = RLB_EOS_ULTRA;
    p.xbc = RLB_BC_PERIODIC;
    p.prec = RLB_FP64;
    p.nx = 2145386496; /* 2^31 - 2^21 */
    p.ny = 1;
    p.nz = 1;
    CHECK(rlb_state_layout(&p, &stride, &elem, &bytes) == RLB_OK);
    CHECK(stride == 2145386496LL && bytes == (size_t)38 * 2145386496ULL * 8u);
    CHECK(rlb_workspace_bytes(&p, &ws) == RLB_OK && ws > 2 * bytes);
    p.nx = 2145386497; /* 2^31 - 2^21 + 1 */
    CHECK(rlb_state_layout(&p, &stride, &elem, &bytes) == RLB_ERR_ARG);
    p.nx = 65536;
    p.ny = 65536; /* N = 2^32: the product is formed in 64 bits */
    CHECK(rlb_workspace_bytes(&p, &ws) == RLB_ERR_ARG);
    p.nx = 0;
    CHECK(rlb_create(&p, NULL, NULL, 0, &ctx) == RLB_ERR_ARG && ctx == NULL);

    CHECK(strcmp(rlb_status_str(RLB_OK), rlb_status_str(RLB_ERR_ARG)) != 0);
    CHECK(rlb_destroy(NULL) == RLB_OK);
    int64_t count = 0;
    const rlb_status s = rlb_debug_bounds_violations(&count);
    CHECK(s == RLB_ERR_STATE && count == -1); /* the release library */

    if (fails) return 1;
    printf("ok\n");
    return 0;
}

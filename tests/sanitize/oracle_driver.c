/*
 * Exercises the FP64 oracle (oracle/rlb_oracle.c) on small lattices of every
 * boundary kind, with solid cells and both equations of state, so that the
 * oracle can be run under AddressSanitizer and UndefinedBehaviorSanitizer
 * (tests/test_oracle_sanitize.py builds it with -fsanitize=address,undefined).
 * Test infrastructure only.  Exit status 0 when every call returned normally.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    int32_t xbc;
    double tau, c_l;
    double n_in, eps_in, beta_in[3];
    int32_t eos, pad;
    double eos_gamma, eos_mass;
} orc_params;

typedef struct {
    int64_t steps, n_unphysical, first_bad, n_nonpositive_eq;
} orc_stats;

int orc_init(const orc_params*, const double*, const double*, const double*, const uint8_t*, double*);
int orc_run(const orc_params*, const uint8_t*, double*, double*, int64_t, int64_t, orc_stats*);
int64_t orc_macro(const orc_params*, const uint8_t*, const double*, double*, double*, double*);
int orc_adjoint_step(const orc_params*, const uint8_t*, const double*, const double*, double*, double*, double*);
int orc_adjoint_macro(const orc_params*, const uint8_t*, const double*, const double*, const double*, const double*,
                      double*);
int orc_adjoint_fields(const orc_params*, const uint8_t*, const double*, const double*, const double*,
                       const double*, double*, double*, double*, double*);

static double urand(uint64_t* s) {
    *s = *s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(*s >> 11) / 9007199254740992.0;
}

static int run_case(int nx, int ny, int nz, int xbc, int with_solid, int eos) {
    orc_params p;
    memset(&p, 0, sizeof p);
    p.nx = nx, p.ny = ny, p.nz = nz, p.xbc = xbc, p.tau = 0.8, p.c_l = 1.0;
    p.n_in = 1.0, p.eps_in = 1.1, p.beta_in[0] = 0.2;
    p.eos = eos, p.eos_gamma = eos ? 1.2 : 4.0 / 3.0, p.eos_mass = eos ? 0.3 : 0.0;
    const int64_t N = (int64_t)nx * ny * nz;
    double* n = calloc(N, sizeof(double));
    double* eps = calloc(N, sizeof(double));
    double* beta = calloc(3 * N, sizeof(double));
    double* a = calloc(N * 38, sizeof(double));
    double* b = calloc(N * 38, sizeof(double));
    double* lam = calloc(N * 38, sizeof(double));
    double* lam2 = calloc(N * 38, sizeof(double));
    double* d3 = calloc(3 * N, sizeof(double));
    uint8_t* solid = calloc(N, 1);
    uint64_t seed = 12345u + (uint64_t)(nx * 100 + ny * 10 + nz);
    for (int64_t c = 0; c < N; ++c) {
        n[c] = 0.9 + 0.2 * urand(&seed);
        eps[c] = 1.0 + 0.2 * urand(&seed);
        for (int k = 0; k < 3; ++k) beta[k * N + c] = 0.1 * (urand(&seed) - 0.5);
    }
    if (with_solid && nx >= 7) solid[(int64_t)(nz / 2) * ny * nx + (ny / 2) * nx + nx / 2] = 1;
    orc_stats st = {0, 0, -1, 0};
    orc_init(&p, n, eps, beta, with_solid ? solid : NULL, a);
    orc_run(&p, with_solid ? solid : NULL, a, b, 5, 0, &st);
    orc_macro(&p, with_solid ? solid : NULL, a, n, eps, beta);
    if (eos == 0) {
        for (int64_t k = 0; k < N * 38; ++k) lam[k] = urand(&seed) - 0.5;
        double dtau = 0.0, dbin[3] = {0, 0, 0};
        orc_adjoint_step(&p, with_solid ? solid : NULL, a, lam, lam2, &dtau, dbin);
        orc_adjoint_macro(&p, with_solid ? solid : NULL, a, n, eps, beta, lam);
        for (int64_t c = 0; c < N; ++c)
            if (!(n[c] == n[c])) n[c] = 1.0, eps[c] = 1.0;  /* solid cells: NaN from macro */
        for (int64_t k = 0; k < 3 * N; ++k)
            if (!(beta[k] == beta[k])) beta[k] = 0.0;
        orc_adjoint_fields(&p, with_solid ? solid : NULL, n, eps, beta, lam2, b, lam, d3, dbin);
    }
    free(n), free(eps), free(beta), free(a), free(b), free(lam), free(lam2), free(d3), free(solid);
    return (int)st.steps == 5 ? 0 : 1;
}

int main(void) {
    int bad = 0;
    const int shapes[][3] = {{1, 1, 1}, {2, 3, 4}, {3, 3, 3}, {9, 5, 4}, {12, 1, 1}};
    for (int s = 0; s < 5; ++s)
        for (int xbc = 0; xbc < 3; ++xbc)
            for (int eos = 0; eos < 2; ++eos) {
                if (xbc != 0 && shapes[s][0] < 3) continue;
                bad |= run_case(shapes[s][0], shapes[s][1], shapes[s][2], xbc, 1, eos);
            }
    printf("oracle sanitizer driver: %s\n", bad ? "FAILED" : "ok");
    return bad;
}

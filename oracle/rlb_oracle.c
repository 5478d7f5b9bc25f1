/*
 * rlb_oracle.c -- plain, slow FP64 reference of the relativistic lattice
 * Boltzmann (RLB) scheme of Mendoza, Boghosian, Herrmann and Succi,
 * "Lattice Boltzmann scheme for relativistic fluids" (arXiv:0912.2913).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA library; the D3Q19 table below is written out here on its own.
 *
 * Arithmetic: IEEE binary64, compiled with -ffp-contract=off, every sum taken
 * in the fixed order i = 0..18.  No blocking, no fusion, no reordering beyond
 * what the equations state.  Cells are independent inside one step, so the
 * OpenMP loop over z planes gives bit-identical results for any thread count.
 *
 * Layout (oracle-private): state[cell*38 + s*19 + i], s = 0 for the number
 * populations f_i and s = 1 for the energy-momentum populations g_i, with
 * cell = (z*ny + y)*nx + x.
 *
 * Readings of the paper that the code takes (the paper is silent on them):
 *  - velocity ordering: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the twelve
 *    (+-1,+-1,0)-type diagonals in opposite pairs (Fig. 2 is not available);
 *  - c_i = c_l e_i with integer e_i, one cell per step; u = beta (c = 1);
 *  - the stored populations are the post-collision ones, the step is
 *    "gather from x - e_i, then collide" (Eqs. lbe1/lbe2 read as a pull);
 *  - solid cells: half-way link bounce-back, h_i(x) = A_opp(i)(x) when x - e_i
 *    is solid; solid cells are never updated;
 *  - x boundaries: periodic, or an inflow ghost plane x = 0 held at
 *    equilibrium of (n_in, eps_in, beta_in) with an outflow ghost x = nx-1
 *    copied from x = nx-2 after each step, or outflow copies at both ends;
 *    y and z are always periodic;
 *  - macroscopic recovery: the positive root of the quadratic obtained from
 *    the three moment constraints with eps = 3P (derived in orc_recover);
 *  - general equation of state (eos = 1): an ideal gas with rest mass,
 *    P = (Gamma - 1)(eps - n m), with the equilibria of Eqs. (equil1),
 *    (equil2a), (equil2b) and a Newton iteration on P for the recovery
 *    (orc_recover_general).  Gamma = 4/3, m = 0 is the eps = 3P case.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define NPOP 38

/* D3Q19 cell configuration (Fig. 2): integer directions e_i, weights w_i
 * (w_0 = 1/3, 1/18 for |c_i| = c_l, 1/36 for |c_i| = sqrt(2) c_l), opposites. */
static const int EV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight(int i) {
    int s = EV[i][0] * EV[i][0] + EV[i][1] * EV[i][1] + EV[i][2] * EV[i][2];
    if (s == 0) return 1.0 / 3.0;
    if (s == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int i) {
    for (int j = 0; j < Q; ++j)
        if (EV[j][0] == -EV[i][0] && EV[j][1] == -EV[i][1] && EV[j][2] == -EV[i][2]) return j;
    return -1;
}

enum { XBC_PERIODIC = 0, XBC_INFLOW_OUTFLOW = 1, XBC_OUTFLOW_BOTH = 2 };

enum { EOS_ULTRA = 0, EOS_GAMMA_LAW = 1 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t xbc;
    double tau, c_l;
    double n_in, eps_in, beta_in[3];
    int32_t eos, pad;
    double eos_gamma, eos_mass;
} orc_params;

typedef struct {
    int64_t steps;
    int64_t n_unphysical;
    int64_t first_bad;
    int64_t n_nonpositive_eq;
} orc_stats;

void orc_lattice(int32_t* e, double* w, int32_t* opp) {
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = EV[i][a];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

static int omp_threads_wanted = 0;
void orc_set_threads(int n) { omp_threads_wanted = n; }
int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_threads_wanted > 0 ? omp_threads_wanted : omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Equilibria for the ultra-relativistic equation of state eps = 3P,          */
/* Eqs. (equil1s), (equil2as), (equil2bs), with (c_i . u)/c_l^2 = e_i.beta/c_l */
/* and |u|^2/c_l^2 = |beta|^2/c_l^2.                                          */
/* ------------------------------------------------------------------------ */
void orc_equilibrium(double n, double eps, const double* beta, double c_l, double* feq, double* geq) {
    double b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    double gam2 = 1.0 / (1.0 - b2);
    double gam = sqrt(gam2);
    double cl2 = c_l * c_l;
    for (int i = 0; i < Q; ++i) {
        double cu = (EV[i][0] * beta[0] + EV[i][1] * beta[1] + EV[i][2] * beta[2]) * c_l; /* c_i . u */
        double w = weight(i);
        /* Eq. (equil1s): f_i = w_i n gamma [1 + 3 (c_i.u)/c_l^2] */
        feq[i] = w * n * gam * (1.0 + 3.0 * cu / cl2);
        if (i == 0) {
            /* Eq. (equil2bs): g_0 = w_0 eps gamma^2 [4 - (2 + c_l^2)/(gamma^2 c_l^2) - 2|u|^2/c_l^2] */
            geq[i] = w * eps * gam2 * (4.0 - (2.0 + cl2) / (gam2 * cl2) - 2.0 * b2 / cl2);
        } else {
            /* Eq. (equil2as): g_i = w_i eps gamma^2 [1/(gamma^2 c_l^2) + 4 (c_i.u)/c_l^2
             *                  + 6 (c_i.u)^2/c_l^4 - 2 |u|^2/c_l^2] */
            geq[i] = w * eps * gam2 *
                     (1.0 / (gam2 * cl2) + 4.0 * cu / cl2 + 6.0 * cu * cu / (cl2 * cl2) - 2.0 * b2 / cl2);
        }
    }
}

/* Macroscopic constraints (the three sums after Fig. 2, and their eps = 3P
 * form after Eq. equil2bs): m[0] = sum f_i = n gamma, m[1] = sum g_i = T^00,
 * m[2..4] = sum g_i c_i = T^0i.                                             */
void orc_moments(const double* h, double c_l, double* m) {
    const double* f = h;
    const double* g = h + Q;
    double sf = 0.0, e = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int i = 0; i < Q; ++i) {
        sf += f[i];
        e += g[i];
        mx += g[i] * (c_l * EV[i][0]);
        my += g[i] * (c_l * EV[i][1]);
        mz += g[i] * (c_l * EV[i][2]);
    }
    m[0] = sf;
    m[1] = e;
    m[2] = mx;
    m[3] = my;
    m[4] = mz;
}

/* Recovery of n, eps, beta from the five moments with eps = 3P.
 * With E = T^00 and M = |T^0i|: E = (4/3) eps gamma^2 - eps/3 and
 * M = (4/3) eps gamma^2 |beta| give E + P = (4/3) eps gamma^2, so
 * beta = M/(E + P) and eps = E - M |beta|.  Eliminating beta:
 *     eps^2 + 2 E eps - 3 E^2 + 3 M^2 = 0,
 * whose non-negative root is eps = -E + sqrt(4 E^2 - 3 M^2).  Then
 * beta = 3 T^0i / (3E + eps) and n = (n gamma) / gamma.
 * Returns 1 when the state is unphysical (sum f <= 0, E <= 0,
 * 4E^2 < 3M^2, eps <= 0, |beta| >= 1, or a non-finite value); the values are
 * still written as computed (no clamping).                                  */
int orc_recover(const double* m, double c_l, double* n, double* eps, double* beta) {
    (void)c_l;
    double sf = m[0], e = m[1];
    double m2 = m[2] * m[2] + m[3] * m[3] + m[4] * m[4];
    double disc = 4.0 * e * e - 3.0 * m2;
    double ep = -e + sqrt(disc);
    double d = 3.0 * e + ep;
    double b[3];
    for (int a = 0; a < 3; ++a) b[a] = 3.0 * m[2 + a] / d;
    double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double nn = sf * sqrt(1.0 - b2);
    *n = nn;
    *eps = ep;
    for (int a = 0; a < 3; ++a) beta[a] = b[a];
    int bad = 0;
    if (!(sf > 0.0)) bad = 1;
    if (!(e > 0.0)) bad = 1;
    if (!(disc >= 0.0)) bad = 1;
    if (!(ep > 0.0)) bad = 1;
    if (!(b2 < 1.0)) bad = 1;
    if (!isfinite(nn) || !isfinite(ep) || !isfinite(b[0]) || !isfinite(b[1]) || !isfinite(b[2])) bad = 1;
    return bad;
}

/* ------------------------------------------------------------------------ */
/* General equation of state (the macroscopic constraints after Fig. 2 and   */
/* Eqs. equil1, equil2a, equil2b): an ideal gas with rest mass m,             */
/*     P = (Gamma - 1) (eps - n m).                                           */
/* ------------------------------------------------------------------------ */
double orc_eos_pressure(double gamma_ad, double mass, double n, double eps) {
    return (gamma_ad - 1.0) * (eps - n * mass);
}

/* Eqs. (equil1), (equil2a), (equil2b) with pressure P. */
void orc_equilibrium_general(double n, double eps, double P, const double* beta, double c_l, double* feq,
                             double* geq) {
    double b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    double gam2 = 1.0 / (1.0 - b2);
    double gam = sqrt(gam2);
    double cl2 = c_l * c_l;
    double h = (eps + P) * gam2; /* (eps + P) gamma^2 */
    for (int i = 0; i < Q; ++i) {
        double cu = (EV[i][0] * beta[0] + EV[i][1] * beta[1] + EV[i][2] * beta[2]) * c_l; /* c_i . u */
        double w = weight(i);
        /* Eq. (equil1): f_i = w_i n gamma [1 + 3 (c_i.u)/c_l^2] */
        feq[i] = w * n * gam * (1.0 + 3.0 * cu / cl2);
        if (i == 0) {
            /* Eq. (equil2b): g_0 = w_0 (eps+P) gamma^2 [3 - 3P(2 + c_l^2)/((P+eps) gamma^2 c_l^2)
             *                                            - (3/2)|u|^2/c_l^2] */
            geq[i] = w * h * (3.0 - 3.0 * P * (2.0 + cl2) / ((P + eps) * gam2 * cl2) - 1.5 * b2 / cl2);
        } else {
            /* Eq. (equil2a): g_i = w_i (eps+P) gamma^2 [3P/((P+eps) gamma^2 c_l^2) + 3 (c_i.u)/c_l^2
             *                      + (9/2)(c_i.u)^2/c_l^4 - (3/2)|u|^2/c_l^2] */
            geq[i] = w * h *
                     (3.0 * P / ((P + eps) * gam2 * cl2) + 3.0 * cu / cl2 + 4.5 * cu * cu / (cl2 * cl2) -
                      1.5 * b2 / cl2);
        }
    }
}

/* Recovery of n, eps, P, beta from the moments m = (n gamma, T^00, T^0i)
 * with P = (Gamma - 1)(eps - n m).  The constraints give, for a trial P,
 *     beta = T^0i / (T^00 + P),   eps = T^00 - |T^0i|^2 / (T^00 + P),
 *     n = (n gamma) sqrt(1 - beta^2),
 * and P solves r(P) = (Gamma - 1)(eps(P) - m n(P)) - P = 0 with
 *     r'(P) = (Gamma - 1)(beta^2 - m n beta^2 / ((T^00 + P)(1 - beta^2))) - 1.
 * Newton from P = (Gamma - 1)(T^00 - m n gamma) (the value at rest), raised
 * above |T^0i| - T^00 so that |beta| < 1, until |dP| <= 1e-14 (P + T^00)
 * (eps(P) is formed by cancellation at high |beta|, so the last steps move P
 * by rounding noise of T^00; at most 100 iterations).  Returns 1 when the state is unphysical
 * (n gamma <= 0, T^00 <= 0, no convergence, P <= 0, |beta| >= 1, a
 * non-finite value); *iters receives the iteration count.                   */
int orc_recover_general(const double* m, double c_l, double gamma_ad, double mass, double* n, double* eps,
                        double* P, double* beta, int* iters) {
    (void)c_l;
    double D = m[0], E = m[1];
    double M2 = m[2] * m[2] + m[3] * m[3] + m[4] * m[4];
    double M = sqrt(M2);
    double g1 = gamma_ad - 1.0;
    double p = g1 * (E - mass * D);
    double lo = M - E;
    if (!(p > lo)) p = lo + 1e-3 * (E > 0.0 ? E : 1.0);
    int it = 0, conv = 0;
    for (it = 0; it < 100; ++it) {
        double W = E + p;
        double b2 = M2 / (W * W);
        double nn = D * sqrt(1.0 - b2);
        double ep = E - M2 / W;
        double r = g1 * (ep - mass * nn) - p;
        double dr = g1 * (b2 - mass * nn * b2 / (W * (1.0 - b2))) - 1.0;
        double dp = -r / dr;
        p = p + dp;
        if (fabs(dp) <= 1e-14 * (fabs(p) + fabs(E))) {
            conv = 1;
            ++it;
            break;
        }
    }
    double W = E + p;
    double b[3];
    for (int a = 0; a < 3; ++a) b[a] = m[2 + a] / W;
    double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double nn = D * sqrt(1.0 - b2);
    double ep = E - M2 / W;
    *n = nn;
    *eps = ep;
    *P = p;
    for (int a = 0; a < 3; ++a) beta[a] = b[a];
    if (iters) *iters = it;
    int bad = 0;
    if (!(D > 0.0)) bad = 1;
    if (!(E > 0.0)) bad = 1;
    if (!conv) bad = 1;
    if (!(p > 0.0)) bad = 1;
    if (!(b2 < 1.0)) bad = 1;
    if (!isfinite(nn) || !isfinite(ep) || !isfinite(p) || !isfinite(b[0]) || !isfinite(b[1]) || !isfinite(b[2]))
        bad = 1;
    return bad;
}

/* Equilibria of a cell's fields under the run's equation of state. */
static void equilibrium_of(const orc_params* p, double n, double eps, const double* beta, double* feq,
                           double* geq) {
    if (p->eos == EOS_GAMMA_LAW)
        orc_equilibrium_general(n, eps, orc_eos_pressure(p->eos_gamma, p->eos_mass, n, eps), beta, p->c_l, feq,
                                geq);
    else
        orc_equilibrium(n, eps, beta, p->c_l, feq, geq);
}

/* Positivity diagnostic (the condition stated after the tachyon paragraph:
 * f_i^eq > 0 requires c_i . u < c_l^2/3).  The decision is taken in binary32
 * on beta rounded to binary32, as the CUDA kernels take it:
 *   q_p  = e_p . beta over the nine direction pairs (pair sums in float),
 *   f-bracket at -|q|:  c_l - 3|q|           <= 0  -> flag,
 *   g-bracket at -|q|:  (1 - 3 b2) + |q| (6|q| - 4 c_l) <= 0 -> flag,
 * with b2 = (bx*bx + by*by) + bz*bz.  Both brackets are the Eq. (equil1s) and
 * Eq. (equil2as) brackets multiplied by positive factors; the rest-particle
 * bracket of Eq. (equil2bs) is positive for |beta| < 1 and is not tested.   */
static int positivity_flag(const double* beta, double c_l) {
    float bx = (float)beta[0], by = (float)beta[1], bz = (float)beta[2];
    float cl = (float)c_l;
    float q[9];
    q[0] = bx;
    q[1] = by;
    q[2] = bz;
    q[3] = bx + by;
    q[4] = bx - by;
    q[5] = bx + bz;
    q[6] = bx - bz;
    q[7] = by + bz;
    q[8] = by - bz;
    float t0 = bx * bx;
    float t1 = by * by;
    float t2 = bz * bz;
    float t01 = t0 + t1;
    float b2 = t01 + t2;
    float three_b2 = 3.0f * b2;
    float c0 = 1.0f - three_b2;
    int flag = 0;
    for (int p = 0; p < 9; ++p) {
        float aq = fabsf(q[p]);
        float three_aq = 3.0f * aq;
        float fb = cl - three_aq;
        float six_aq = 6.0f * aq;
        float four_cl = 4.0f * cl;
        float inner = six_aq - four_cl;
        float prod = aq * inner;
        float gb = c0 + prod;
        if (fb <= 0.0f) flag = 1;
        if (gb <= 0.0f) flag = 1;
    }
    return flag;
}

static inline int64_t cell_index(const orc_params* p, int x, int y, int z) {
    return ((int64_t)z * p->ny + y) * p->nx + x;
}

static int is_ghost(const orc_params* p, int x) {
    if (p->xbc == XBC_PERIODIC) return 0;
    return x == 0 || x == p->nx - 1;
}

/* Initial condition: every cell in equilibrium with its initial fields
 * ("thermodynamically equilibrated matter" on both sides of the membrane).
 * Under the inflow/outflow condition the inflow plane x = 0 takes the inflow
 * state instead.  beta is three planes of N values (x, y, z components).   */
int orc_init(const orc_params* p, const double* n, const double* eps, const double* beta, const uint8_t* solid,
             double* state) {
    (void)solid;
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t c = 0; c < N; ++c) {
        double b[3] = {beta[c], beta[N + c], beta[2 * N + c]};
        int x = (int)(c % p->nx);
        double* h = state + c * NPOP;
        if (p->xbc == XBC_INFLOW_OUTFLOW && x == 0)
            equilibrium_of(p, p->n_in, p->eps_in, p->beta_in, h, h + Q);
        else
            equilibrium_of(p, n[c], eps[c], b, h, h + Q);
    }
    return 0;
}

/* Gather (pull streaming) for one cell: h_i(x) = A_i(x - e_i), or the link
 * bounce-back h_i(x) = A_opp(i)(x) when x - e_i is solid.  Eqs. (lbe1) and
 * (lbe2) move f_i from x to x + c_i dt; read backwards, x receives from
 * x - e_i.  The x index of a non-periodic lattice never leaves [0, nx) for
 * the interior cells that are gathered.                                     */
static void gather(const orc_params* p, const uint8_t* solid, const double* in, int x, int y, int z, double* h) {
    int64_t self = cell_index(p, x, y, z);
    for (int i = 0; i < Q; ++i) {
        int sx = x - EV[i][0], sy = y - EV[i][1], sz = z - EV[i][2];
        sx = (sx % p->nx + p->nx) % p->nx;
        sy = (sy % p->ny + p->ny) % p->ny;
        sz = (sz % p->nz + p->nz) % p->nz;
        int64_t src = cell_index(p, sx, sy, sz);
        if (solid && solid[src]) {
            int o = opposite(i);
            h[i] = in[self * NPOP + o];
            h[Q + i] = in[self * NPOP + Q + o];
        } else {
            h[i] = in[src * NPOP + i];
            h[Q + i] = in[src * NPOP + Q + i];
        }
    }
}

/* One time step of Eqs. (lbe1), (lbe2): gather, moments, recovery,
 * equilibria, BGK relaxation with delta t = 1:
 *     out_i = h_i - (h_i - eq_i) / tau,
 * then the boundary planes.  step_index numbers the update for first_bad.  */
int orc_step(const orc_params* p, const uint8_t* solid, const double* in, double* out, int64_t step_index,
             orc_stats* st) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    int64_t N = (int64_t)nx * ny * nz;
    int64_t n_unph = 0, n_pos = 0;
    int64_t first = -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(orc_get_threads()) reduction(+ : n_unph, n_pos)
#endif
    for (int z = 0; z < nz; ++z) {
        int64_t first_local = -1;
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell_index(p, x, y, z);
                if ((solid && solid[c]) || is_ghost(p, x)) {
                    memcpy(out + c * NPOP, in + c * NPOP, sizeof(double) * NPOP);
                    continue;
                }
                double h[NPOP], m[5], feq[Q], geq[Q], beta[3], n, eps;
                gather(p, solid, in, x, y, z, h);
                orc_moments(h, p->c_l, m);
                int bad, pos;
                if (p->eos == EOS_GAMMA_LAW) {
                    /* general EOS: the positivity counter flags any equilibrium <= 0 */
                    double P;
                    bad = orc_recover_general(m, p->c_l, p->eos_gamma, p->eos_mass, &n, &eps, &P, beta, NULL);
                    orc_equilibrium_general(n, eps, P, beta, p->c_l, feq, geq);
                    pos = 0;
                    for (int i = 0; i < Q; ++i)
                        if (!(feq[i] > 0.0) || !(geq[i] > 0.0)) pos = 1;
                } else {
                    bad = orc_recover(m, p->c_l, &n, &eps, beta);
                    pos = positivity_flag(beta, p->c_l);
                    orc_equilibrium(n, eps, beta, p->c_l, feq, geq);
                }
                double* o = out + c * NPOP;
                for (int i = 0; i < Q; ++i) {
                    o[i] = h[i] - (h[i] - feq[i]) / p->tau;
                    o[Q + i] = h[Q + i] - (h[Q + i] - geq[i]) / p->tau;
                }
                if (bad) {
                    n_unph += 1;
                    int64_t id = step_index * N + c;
                    if (first_local < 0 || id < first_local) first_local = id;
                }
                if (pos) n_pos += 1;
            }
        }
        if (first_local >= 0) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (first < 0 || first_local < first) first = first_local;
            }
        }
    }
    /* boundary planes, after the collision of the whole lattice */
    if (p->xbc != XBC_PERIODIC) {
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y) {
                int64_t g1 = cell_index(p, nx - 1, y, z), s1 = cell_index(p, nx - 2, y, z);
                if (!(solid && solid[g1])) memcpy(out + g1 * NPOP, out + s1 * NPOP, sizeof(double) * NPOP);
                int64_t g0 = cell_index(p, 0, y, z), s0 = cell_index(p, 1, y, z);
                if (solid && solid[g0]) continue;
                if (p->xbc == XBC_OUTFLOW_BOTH)
                    memcpy(out + g0 * NPOP, out + s0 * NPOP, sizeof(double) * NPOP);
                else
                    equilibrium_of(p, p->n_in, p->eps_in, p->beta_in, out + g0 * NPOP, out + g0 * NPOP + Q);
            }
    }
    if (st) {
        st->steps += 1;
        st->n_unphysical += n_unph;
        st->n_nonpositive_eq += n_pos;
        if (first >= 0 && (st->first_bad < 0 || first < st->first_bad)) st->first_bad = first;
    }
    return 0;
}

/* nsteps steps; state holds the result, scratch is a second buffer of the
 * same size.  step0 is the index of the first step (for first_bad).        */
int orc_run(const orc_params* p, const uint8_t* solid, double* state, double* scratch, int64_t nsteps, int64_t step0,
            orc_stats* st) {
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double* a = state;
    double* b = scratch;
    for (int64_t t = 0; t < nsteps; ++t) {
        orc_step(p, solid, a, b, step0 + t, st);
        double* tmp = a;
        a = b;
        b = tmp;
    }
    if (a != state) memcpy(state, a, sizeof(double) * NPOP * N);
    return 0;
}

/* Macroscopic output: n, eps, beta from the moments of the stored
 * populations at every cell; NaN at solid cells.  Returns the number of
 * non-solid cells whose recovery is unphysical.                             */
int64_t orc_macro(const orc_params* p, const uint8_t* solid, const double* state, double* n, double* eps,
                  double* beta) {
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    int64_t bad = 0;
    for (int64_t c = 0; c < N; ++c) {
        if (solid && solid[c]) {
            n[c] = eps[c] = beta[c] = beta[N + c] = beta[2 * N + c] = NAN;
            continue;
        }
        double m[5], b[3], nn, ep, P;
        orc_moments(state + c * NPOP, p->c_l, m);
        if (p->eos == EOS_GAMMA_LAW)
            bad += orc_recover_general(m, p->c_l, p->eos_gamma, p->eos_mass, &nn, &ep, &P, b, NULL);
        else
            bad += orc_recover(m, p->c_l, &nn, &ep, b);
        n[c] = nn;
        eps[c] = ep;
        beta[c] = b[0];
        beta[N + c] = b[1];
        beta[2 * N + c] = b[2];
    }
    return bad;
}

/* ======================================================================== */
/* Discrete adjoint (transpose of the exact Jacobian of one step).          */
/* Partial derivatives below are taken by hand from Eqs. (equil1s),          */
/* (equil2as), (equil2bs) and from the closed-form recovery above.           */
/* ======================================================================== */

/* d(feq, geq)/d(n, eps, beta_a) at a field point: out[38][5], columns
 * (n, eps, beta_x, beta_y, beta_z).  Eq. (equil1s) depends on n gamma and
 * beta, Eqs. (equil2as, equil2bs) on eps and beta.                          */
static void deq_dfields(double n, double eps, const double* beta, double c_l, double out[NPOP][5]) {
    double b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    double gam2 = 1.0 / (1.0 - b2);
    double gam = sqrt(gam2);
    double cl2 = c_l * c_l;
    for (int i = 0; i < Q; ++i) {
        double w = weight(i);
        double q = EV[i][0] * beta[0] + EV[i][1] * beta[1] + EV[i][2] * beta[2]; /* e_i . beta */
        double fb = 1.0 + 3.0 * q / c_l;
        /* f_i = w n gamma fb;  d gamma / d beta_a = gamma^3 beta_a */
        out[i][0] = w * gam * fb;
        out[i][1] = 0.0;
        for (int a = 0; a < 3; ++a)
            out[i][2 + a] = w * n * (gam * gam2 * beta[a] * fb + gam * 3.0 * EV[i][a] / c_l);
        /* g: d gamma^2 / d beta_a = 2 gamma^4 beta_a */
        double dg2[3];
        for (int a = 0; a < 3; ++a) dg2[a] = 2.0 * gam2 * gam2 * beta[a];
        out[Q + i][0] = 0.0;
        if (i == 0) {
            /* g_0 = w0 eps [4 gamma^2 - (2 + c_l^2)/c_l^2 - 2 gamma^2 b2 / c_l^2] */
            out[Q + i][1] = w * (4.0 * gam2 - (2.0 + cl2) / cl2 - 2.0 * gam2 * b2 / cl2);
            for (int a = 0; a < 3; ++a)
                out[Q + i][2 + a] = w * eps * (4.0 * dg2[a] - 2.0 * (dg2[a] * b2 + gam2 * 2.0 * beta[a]) / cl2);
        } else {
            /* g_i = w eps [1/c_l^2 + gamma^2 (4q/c_l + 6 q^2/c_l^2 - 2 b2/c_l^2)] */
            double br = 4.0 * q / c_l + 6.0 * q * q / cl2 - 2.0 * b2 / cl2;
            out[Q + i][1] = w * (1.0 / cl2 + gam2 * br);
            for (int a = 0; a < 3; ++a) {
                double dbr = 4.0 * EV[i][a] / c_l + 12.0 * q * EV[i][a] / cl2 - 4.0 * beta[a] / cl2;
                out[Q + i][2 + a] = w * eps * (dg2[a] * br + gam2 * dbr);
            }
        }
    }
}

/* Jacobian of the recovery: J[r][k] = d(out_r)/d(m_k) with outputs
 * r = (n gamma = sum f, eps, beta_x, beta_y, beta_z) and moments
 * k = (sum f, E, Mx, My, Mz).  Also returns the recovered fields.           */
static void drecover(const double* m, double c_l, double J[5][5], double* sf, double* eps, double* beta) {
    double n;
    orc_recover(m, c_l, &n, eps, beta);
    *sf = m[0];
    double E = m[1];
    double M[3] = {m[2], m[3], m[4]};
    double m2 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    double s = sqrt(4.0 * E * E - 3.0 * m2);
    double D = 3.0 * E + *eps;
    double deps_dE = 4.0 * E / s - 1.0;
    double deps_dM[3];
    for (int b = 0; b < 3; ++b) deps_dM[b] = -3.0 * M[b] / s;
    memset(J, 0, sizeof(double) * 25);
    J[0][0] = 1.0;
    J[1][1] = deps_dE;
    for (int b = 0; b < 3; ++b) J[1][2 + b] = deps_dM[b];
    double dD_dE = 3.0 + deps_dE;
    for (int a = 0; a < 3; ++a) {
        J[2 + a][1] = -3.0 * M[a] * dD_dE / (D * D);
        for (int b = 0; b < 3; ++b)
            J[2 + a][2 + b] = (a == b ? 3.0 / D : 0.0) - 3.0 * M[a] * deps_dM[b] / (D * D);
    }
}

/* d(moment k)/d(population j): P[k][j]. */
static double dmoment(int k, int j, double c_l) {
    int s = j / Q, i = j % Q;
    if (k == 0) return s == 0 ? 1.0 : 0.0;
    if (s == 0) return 0.0;
    if (k == 1) return 1.0;
    return c_l * EV[i][k - 2];
}

/* nu = J_C(h)^T mu for the collision C(h) = h - (h - eq(h))/tau, with
 * eq(h) = eq(S_f, eps(m), beta(m)), m = P h (f^eq taken as w S_f [...] since
 * n gamma = S_f).  The full 38x38 Jacobian is formed explicitly.
 * Also returns sum_i mu_i (h_i - eq_i)/tau^2 = mu . dC/dtau.                */
static double collision_adjoint(const double* h, const double* mu, double tau, double c_l, double* nu) {
    double m[5], J[5][5], sf, eps, beta[3];
    orc_moments(h, c_l, m);
    drecover(m, c_l, J, &sf, &eps, beta);
    /* eq as a function of (S_f, eps, beta): Eq. (equil1s) with n gamma = S_f */
    double b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    double gam = sqrt(1.0 / (1.0 - b2));
    double feq[Q], geq[Q];
    orc_equilibrium(sf / gam, eps, beta, c_l, feq, geq);
    double dF[NPOP][5]; /* columns: (n, eps, beta) at n = S_f / gamma */
    deq_dfields(sf / gam, eps, beta, c_l, dF);
    /* convert the n-column and beta-columns to the (S_f, eps, beta) variables:
     * f_i = w S_f fb  ->  d/dS_f = w fb,  d/dbeta_a at fixed S_f = w S_f 3 e_a / c_l */
    double dE[NPOP][5];
    for (int j = 0; j < NPOP; ++j) {
        int s = j / Q, i = j % Q;
        if (s == 0) {
            double q = EV[i][0] * beta[0] + EV[i][1] * beta[1] + EV[i][2] * beta[2];
            dE[j][0] = weight(i) * (1.0 + 3.0 * q / c_l);
            dE[j][1] = 0.0;
            for (int a = 0; a < 3; ++a) dE[j][2 + a] = weight(i) * sf * 3.0 * EV[i][a] / c_l;
        } else {
            for (int r = 0; r < 5; ++r) dE[j][r] = dF[j][r];
        }
    }
    /* Jfull[j][l] = (1 - 1/tau) delta_jl + (1/tau) sum_r sum_k dE[j][r] J[r][k] P[k][l] */
    double A[NPOP][5]; /* A = dE J : d eq_j / d m_k */
    for (int j = 0; j < NPOP; ++j)
        for (int k = 0; k < 5; ++k) {
            double acc = 0.0;
            for (int r = 0; r < 5; ++r) acc += dE[j][r] * J[r][k];
            A[j][k] = acc;
        }
    double om = 1.0 / tau;
    for (int l = 0; l < NPOP; ++l) {
        double acc = 0.0;
        for (int j = 0; j < NPOP; ++j) {
            double deq = 0.0;
            for (int k = 0; k < 5; ++k) deq += A[j][k] * dmoment(k, l, c_l);
            double Jjl = (j == l ? 1.0 - om : 0.0) + om * deq;
            acc += Jjl * mu[j];
        }
        nu[l] = acc;
    }
    double dtau = 0.0;
    for (int i = 0; i < Q; ++i) {
        dtau += mu[i] * (h[i] - feq[i]) / (tau * tau);
        dtau += mu[Q + i] * (h[Q + i] - geq[i]) / (tau * tau);
    }
    return dtau;
}

/* Adjoint of one step.  in_t is the state A_t the forward step started
 * from; lam_in = dL/dA_{t+1}; lam_out = dL/dA_t (overwritten).  Adds the
 * step's contributions to *dtau and dbeta_in[3].                            */
int orc_adjoint_step(const orc_params* p, const uint8_t* solid, const double* in_t, const double* lam_in,
                     double* lam_out, double* dtau, double* dbeta_in) {
    if (p->eos != EOS_ULTRA) return -1; /* the adjoint covers eps = 3P */
    int nx = p->nx, ny = p->ny, nz = p->nz;
    int64_t N = (int64_t)nx * ny * nz;
    memset(lam_out, 0, sizeof(double) * NPOP * N);
    double tsum = 0.0;
    double bsum[3] = {0.0, 0.0, 0.0};
    double dIn[NPOP][5];
    if (p->xbc == XBC_INFLOW_OUTFLOW) deq_dfields(p->n_in, p->eps_in, p->beta_in, p->c_l, dIn);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell_index(p, x, y, z);
                if (solid && solid[c]) { /* never updated: identity */
                    for (int j = 0; j < NPOP; ++j) lam_out[c * NPOP + j] += lam_in[c * NPOP + j];
                    continue;
                }
                if (is_ghost(p, x)) {
                    /* inflow ghost: A_{t+1}(x) = eq(n_in, eps_in, beta_in) */
                    if (p->xbc == XBC_INFLOW_OUTFLOW && x == 0)
                        for (int j = 0; j < NPOP; ++j)
                            for (int a = 0; a < 3; ++a) bsum[a] += lam_in[c * NPOP + j] * dIn[j][2 + a];
                    continue; /* outflow ghosts: handled by their copy source */
                }
                double h[NPOP], mu[NPOP], nu[NPOP];
                gather(p, solid, in_t, x, y, z, h);
                for (int j = 0; j < NPOP; ++j) mu[j] = lam_in[c * NPOP + j];
                if (p->xbc != XBC_PERIODIC && x == nx - 2) {
                    int64_t g = cell_index(p, nx - 1, y, z);
                    if (!(solid && solid[g]))
                        for (int j = 0; j < NPOP; ++j) mu[j] += lam_in[g * NPOP + j];
                }
                if (p->xbc == XBC_OUTFLOW_BOTH && x == 1) {
                    int64_t g = cell_index(p, 0, y, z);
                    if (!(solid && solid[g]))
                        for (int j = 0; j < NPOP; ++j) mu[j] += lam_in[g * NPOP + j];
                }
                tsum += collision_adjoint(h, mu, p->tau, p->c_l, nu);
                /* transpose of the gather */
                for (int i = 0; i < Q; ++i) {
                    int sx = ((x - EV[i][0]) % nx + nx) % nx;
                    int sy = ((y - EV[i][1]) % ny + ny) % ny;
                    int sz = ((z - EV[i][2]) % nz + nz) % nz;
                    int64_t src = cell_index(p, sx, sy, sz);
                    if (solid && solid[src]) {
                        int o = opposite(i);
                        lam_out[c * NPOP + o] += nu[i];
                        lam_out[c * NPOP + Q + o] += nu[Q + i];
                    } else {
                        lam_out[src * NPOP + i] += nu[i];
                        lam_out[src * NPOP + Q + i] += nu[Q + i];
                    }
                }
            }
    if (dtau) *dtau += tsum;
    if (dbeta_in)
        for (int a = 0; a < 3; ++a) dbeta_in[a] += bsum[a];
    return 0;
}

/* Adjoint of the macroscopic output: lam = (d macro / d state)^T g, where
 * g = (dL/dn, dL/deps, dL/dbeta) per cell (beta as three planes).  n = S_f
 * sqrt(1 - |beta|^2).  Solid cells get zero.                               */
int orc_adjoint_macro(const orc_params* p, const uint8_t* solid, const double* state, const double* dn,
                      const double* deps, const double* dbeta, double* lam) {
    if (p->eos != EOS_ULTRA) return -1; /* the adjoint covers eps = 3P */
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t c = 0; c < N; ++c) {
        double* l = lam + c * NPOP;
        if (solid && solid[c]) {
            for (int j = 0; j < NPOP; ++j) l[j] = 0.0;
            continue;
        }
        double m[5], J[5][5], sf, eps, beta[3];
        orc_moments(state + c * NPOP, p->c_l, m);
        drecover(m, p->c_l, J, &sf, &eps, beta);
        double b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
        double rt = sqrt(1.0 - b2);
        /* outputs (n, eps, beta) as functions of r = (S_f, eps, beta) */
        double gr[5];
        gr[0] = dn[c] * rt;
        gr[1] = deps[c];
        for (int a = 0; a < 3; ++a) gr[2 + a] = dbeta[a * N + c] + dn[c] * (-sf * beta[a] / rt);
        double gm[5];
        for (int k = 0; k < 5; ++k) {
            double acc = 0.0;
            for (int r = 0; r < 5; ++r) acc += gr[r] * J[r][k];
            gm[k] = acc;
        }
        for (int j = 0; j < NPOP; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += gm[k] * dmoment(k, j, p->c_l);
            l[j] = acc;
        }
    }
    return 0;
}

/* Adjoint of orc_init: gradients of L with respect to the initial fields
 * n0, eps0, beta0 (beta as three planes), given lam0 = dL/dA_0.  The inflow
 * plane of the inflow/outflow condition adds to dbeta_in instead; solid cells
 * give zero.                                                               */
int orc_adjoint_fields(const orc_params* p, const uint8_t* solid, const double* n, const double* eps,
                       const double* beta, const double* lam0, double* dn, double* deps, double* dbeta,
                       double* dbeta_in) {
    if (p->eos != EOS_ULTRA) return -1; /* the adjoint covers eps = 3P */
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double dIn[NPOP][5];
    if (p->xbc == XBC_INFLOW_OUTFLOW) deq_dfields(p->n_in, p->eps_in, p->beta_in, p->c_l, dIn);
    double bsum[3] = {0.0, 0.0, 0.0};
    for (int64_t c = 0; c < N; ++c) {
        int x = (int)(c % p->nx);
        double out[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        const double* l = lam0 + c * NPOP;
        if (solid && solid[c]) {
        } else if (p->xbc == XBC_INFLOW_OUTFLOW && x == 0) {
            for (int j = 0; j < NPOP; ++j)
                for (int a = 0; a < 3; ++a) bsum[a] += l[j] * dIn[j][2 + a];
        } else {
            double b[3] = {beta[c], beta[N + c], beta[2 * N + c]};
            double d[NPOP][5];
            deq_dfields(n[c], eps[c], b, p->c_l, d);
            for (int r = 0; r < 5; ++r) {
                double acc = 0.0;
                for (int j = 0; j < NPOP; ++j) acc += l[j] * d[j][r];
                out[r] = acc;
            }
        }
        dn[c] = out[0];
        deps[c] = out[1];
        for (int a = 0; a < 3; ++a) dbeta[a * N + c] = out[2 + a];
    }
    if (dbeta_in)
        for (int a = 0; a < 3; ++a) dbeta_in[a] += bsum[a];
    return 0;
}

/* Scalar building blocks exposed for the pin tests. */
void orc_deq_dfields(double n, double eps, const double* beta, double c_l, double* out /* 38*5 */) {
    double d[NPOP][5];
    deq_dfields(n, eps, beta, c_l, d);
    memcpy(out, d, sizeof(d));
}

double orc_collision_adjoint(const double* h, const double* mu, double tau, double c_l, double* nu) {
    return collision_adjoint(h, mu, tau, c_l, nu);
}

void orc_collide(const double* h, double tau, double c_l, double* out) {
    double m[5], beta[3], n, eps, feq[Q], geq[Q];
    orc_moments(h, c_l, m);
    orc_recover(m, c_l, &n, &eps, beta);
    orc_equilibrium(n, eps, beta, c_l, feq, geq);
    for (int i = 0; i < Q; ++i) {
        out[i] = h[i] - (h[i] - feq[i]) / tau;
        out[Q + i] = h[Q + i] - (h[Q + i] - geq[i]) / tau;
    }
}

int orc_positivity_flag(const double* beta, double c_l) { return positivity_flag(beta, c_l); }

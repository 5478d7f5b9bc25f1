// rlb_eos.cu -- the relativistic lattice Boltzmann step with a general
// equation of state (an ideal gas with rest mass m,
//     P = (Gamma - 1)(eps - n m)):
// the equilibria of Eqs. (equil1), (equil2a), (equil2b), the macroscopic
// constraints n gamma = sum f, (eps + P) gamma^2 - P = sum g,
// (eps + P) gamma^2 u = sum g c, and their inversion by a Newton iteration on
// P.  Gamma = 4/3, m = 0 is the eps = 3P scheme.  FP64 states only.
//
// Recovery: with D = sum f, E = sum g, M = sum g c and a trial P,
//     beta = M / (E + P),   eps = E - |M|^2 / (E + P),   n = D sqrt(1 - beta^2);
// P solves r(P) = (Gamma - 1)(eps(P) - m n(P)) - P = 0, with
//     r'(P) = (Gamma - 1)(beta^2 - m n beta^2 / ((E + P)(1 - beta^2))) - 1,
// started from the massless solution (the positive root of
// X^2 - Gamma E X + (Gamma - 1)|M|^2 = 0 for X = E + P, then
// P = (Gamma - 1)(eps - m n) at its eps and n) and iterated until
// |dP| <= 1e-14 (P + E), at most 100 iterations.  Reciprocals and inverse
// square roots are binary32 seeds refined by two FP64 Newton-Raphson steps
// (x -> x (2 - a x) and y -> y (3 - a y^2)/2), which are far cheaper than the
// IEEE FP64 sequences on this GPU's FP64 pipe.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rlb_device.cuh"

namespace rlb {

namespace {

__device__ __forceinline__ double rcp64(double a) {
    double x = rcp_seed(a);
    x = fma(x, fma(-a, x, 1.0), x);
    x = fma(x, fma(-a, x, 1.0), x);
    return x;
}

__device__ __forceinline__ double rsqrt64(double a) {
    double y, half_y;
    rsqrt_seed(a, y, half_y);
    (void)half_y;
    y = y * fma(-0.5 * a * y, y, 1.5);
    y = y * fma(-0.5 * a * y, y, 1.5);
    return y;
}

__device__ __forceinline__ double eos_pressure(const Phys& ph, double n, double eps) {
    return (ph.eos_gamma - 1.0) * (eps - n * ph.eos_mass);
}

// Eqs. (equil1), (equil2a), (equil2b) in pair form: q_p = e_p . beta, so
// (c_i . u)/c_l^2 = +-q_p/c_l and (c_i . u)^2/c_l^4 = q_p^2/c_l^2.
__device__ __forceinline__ void equilibrium_general(double n, double eps, double P, double bx, double by, double bz,
                                                    const Phys& ph, double* f, double* g) {
    const double b2 = bx * bx + by * by + bz * bz;
    const double gam = rsqrt64(1.0 - b2);
    const double gam2 = gam * gam;
    const double h = (eps + P) * gam2;
    const double pr = P * rcp64(h);  // P / ((P + eps) gamma^2)
    const double rest = 3.0 * pr * ph.inv_cl2;
    const double ng = n * gam;
    f[0] = kW0 * ng;
    g[0] = kW0 * h * (3.0 - 3.0 * pr * (2.0 + ph.c_l * ph.c_l) * ph.inv_cl2 - 1.5 * b2 * ph.inv_cl2);
    const double q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const double w = pair_w(p);
        const double fa = 3.0 * q[p] * ph.inv_cl;
        f[2 * p + 1] = w * ng * (1.0 + fa);
        f[2 * p + 2] = w * ng * (1.0 - fa);
        const double gs = w * h * (rest + 4.5 * q[p] * q[p] * ph.inv_cl2 - 1.5 * b2 * ph.inv_cl2);
        const double ga = w * h * 3.0 * q[p] * ph.inv_cl;
        g[2 * p + 1] = gs + ga;
        g[2 * p + 2] = gs - ga;
    }
}

// Returns true when the state is unphysical (see the file header).
__device__ __forceinline__ bool recover_general(double D, double E, double mx, double my, double mz, const Phys& ph,
                                                double& n, double& eps, double& P, double& bx, double& by,
                                                double& bz) {
    const double M2 = mx * mx + my * my + mz * mz;
    const double g1 = ph.eos_gamma - 1.0;
    const double mass = ph.eos_mass;
    double p;
    {
        // massless solution: X = E + P, X^2 - Gamma E X + (Gamma - 1) M^2 = 0
        const double ge = ph.eos_gamma * E;
        const double disc = fma(ge, ge, -4.0 * g1 * M2);
        const double X = 0.5 * (ge + disc * rsqrt64(disc));
        const double rX = rcp64(X);
        const double b2 = M2 * rX * rX;
        const double omb = 1.0 - b2;
        p = g1 * ((E - M2 * rX) - mass * D * (omb * rsqrt64(omb)));
        const double lo = sqrt(M2) - E;
        if (!(p > lo)) p = lo + 1e-3 * (E > 0.0 ? E : 1.0);
    }
    bool conv = false;
    for (int it = 0; it < 100; ++it) {
        const double rW = rcp64(E + p);
        const double b2 = M2 * rW * rW;
        const double rs = rsqrt64(1.0 - b2);
        const double nn = D * ((1.0 - b2) * rs);
        const double ep = E - M2 * rW;
        const double r = g1 * (ep - mass * nn) - p;
        const double dr = g1 * (b2 - mass * D * rs * b2 * rW) - 1.0;  // n / (1 - b2) = D rs
        const double dp = -r * rcp64(dr);
        p = p + dp;
        if (fabs(dp) <= 1e-14 * (fabs(p) + fabs(E))) {
            conv = true;
            break;
        }
    }
    const double rW = rcp64(E + p);
    bx = mx * rW;
    by = my * rW;
    bz = mz * rW;
    const double b2 = bx * bx + by * by + bz * bz;
    n = D * ((1.0 - b2) * rsqrt64(1.0 - b2));
    eps = E - M2 * rW;
    P = p;
    return !(conv && pos_finite(D) && pos_finite(E) && pos_finite(p) && below_one(b2) && isfinite(n) &&
             isfinite(eps) && isfinite(bx) && isfinite(by) && isfinite(bz));
}

template <int XBC>
__global__ void __launch_bounds__(128) k_step_eos(const double* __restrict__ A, double* __restrict__ B, Geom g,
                                                  Phys ph, Counters cnt, int count, long long step_index) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int x, y, z;
    cell_coords(g, idx, x, y, z);
    const long long S = g.S;
    if (XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1)) {
        // ghost planes are not collided (the inflow plane is copied so that
        // every cell of B is written; outflow ghosts are written below)
        if (XBC == XBC_INFLOW_OUTFLOW && x == 0) {
            for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = A[RLB_CHK(q * S + idx, 38ll * S)];
        }
        return;
    }
    const PullOffsets o(g, x, y, z);
    double f[19], gg[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int s = idx + o.src(i);
        f[i] = A[RLB_CHK(i * S + s, 38ll * S)];
        gg[i] = A[RLB_CHK((19 + i) * S + s, 38ll * S)];
    }
    if (is_solid(f[0])) {  // the cell itself is solid: keep the marker
        const double m = solid_marker_d();
        for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = m;
        return;
    }
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (is_solid(f[i])) {  // link bounce-back
            f[i] = A[RLB_CHK(opp(i) * S + idx, 38ll * S)];
            gg[i] = A[RLB_CHK((19 + opp(i)) * S + idx, 38ll * S)];
        }
    }
    double sf, E, mx, my, mz;
    moments_pairs(f, gg, sf, E, mx, my, mz);
    mx *= ph.c_l;
    my *= ph.c_l;
    mz *= ph.c_l;
    double n, eps, P, bx, by, bz;
    const bool unphys = recover_general(sf, E, mx, my, mz, ph, n, eps, P, bx, by, bz);
    double feq[19], geq[19];
    equilibrium_general(n, eps, P, bx, by, bz, ph, feq, geq);
    bool nonpos = false;
    const double om = ph.omega, omw = 1.0 - ph.omega;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        nonpos |= !(feq[i] > 0.0) || !(geq[i] > 0.0);
        f[i] = fma(omw, f[i], om * feq[i]);
        gg[i] = fma(omw, gg[i], om * geq[i]);
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        B[RLB_CHK(i * S + idx, 38ll * S)] = f[i];
        B[RLB_CHK((19 + i) * S + idx, 38ll * S)] = gg[i];
    }
    if (XBC != XBC_PERIODIC && x == g.nx - 2) {  // outflow ghost x = nx-1 copies x = nx-2
        for (int i = 0; i < 19; ++i) {
            B[RLB_CHK(i * S + idx + 1, 38ll * S)] = f[i];
            B[RLB_CHK((19 + i) * S + idx + 1, 38ll * S)] = gg[i];
        }
    }
    if (XBC == XBC_OUTFLOW_BOTH && x == 1) {  // outflow ghost x = 0 copies x = 1
        for (int i = 0; i < 19; ++i) {
            B[RLB_CHK(i * S + idx - 1, 38ll * S)] = f[i];
            B[RLB_CHK((19 + i) * S + idx - 1, 38ll * S)] = gg[i];
        }
    }
    if (count) count_flags(cnt, unphys, nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
}

__global__ void __launch_bounds__(128) k_init_eos(const double* __restrict__ n, const double* __restrict__ eps,
                                                  const double* __restrict__ beta, const uint8_t* __restrict__ solid,
                                                  double* __restrict__ A, double* __restrict__ B, Geom g, Phys ph) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long S = g.S;
    if (solid && solid[idx]) {
        const double m = solid_marker_d();
        for (int q = 0; q < 38; ++q) A[RLB_CHK(q * S + idx, 38ll * S)] = B[RLB_CHK(q * S + idx, 38ll * S)] = m;
        return;
    }
    const int x = idx % g.nx;
    double f[19], gg[19];
    if (g.xbc == XBC_INFLOW_OUTFLOW && x == 0)
        equilibrium_general(ph.n_in, ph.eps_in, eos_pressure(ph, ph.n_in, ph.eps_in), ph.beta_in[0], ph.beta_in[1],
                            ph.beta_in[2], ph, f, gg);
    else
        equilibrium_general(n[idx], eps[idx], eos_pressure(ph, n[idx], eps[idx]), beta[idx], beta[g.N + idx],
                            beta[2 * (long long)g.N + idx], ph, f, gg);
    for (int i = 0; i < 19; ++i) {
        A[RLB_CHK(i * S + idx, 38ll * S)] = B[RLB_CHK(i * S + idx, 38ll * S)] = f[i];
        A[RLB_CHK((19 + i) * S + idx, 38ll * S)] = B[RLB_CHK((19 + i) * S + idx, 38ll * S)] = gg[i];
    }
}

__global__ void __launch_bounds__(128) k_macro_eos(const double* __restrict__ A, double* __restrict__ n,
                                                   double* __restrict__ eps, double* __restrict__ beta, Geom g,
                                                   Phys ph, unsigned long long* bad_count) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long S = g.S;
    if (is_solid(A[RLB_CHK(idx, 38ll * S)])) {
        const double nan = __longlong_as_double(0x7FF8000000000000ll);
        n[idx] = eps[idx] = beta[idx] = beta[g.N + idx] = beta[2 * (long long)g.N + idx] = nan;
        return;
    }
    double f[19], gg[19];
    for (int i = 0; i < 19; ++i) {
        f[i] = A[RLB_CHK(i * S + idx, 38ll * S)];
        gg[i] = A[RLB_CHK((19 + i) * S + idx, 38ll * S)];
    }
    double sf, E, mx, my, mz;
    moments_pairs(f, gg, sf, E, mx, my, mz);
    mx *= ph.c_l;
    my *= ph.c_l;
    mz *= ph.c_l;
    double nn, e, P, bx, by, bz;
    const bool bad = recover_general(sf, E, mx, my, mz, ph, nn, e, P, bx, by, bz);
    n[idx] = nn;
    eps[idx] = e;
    beta[idx] = bx;
    beta[g.N + idx] = by;
    beta[2 * (long long)g.N + idx] = bz;
    if (bad) atomicAdd(bad_count, 1ull);
}

inline unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_init_eos(const Geom& g, const Phys& ph, const double* n, const double* eps, const double* beta,
                            const uint8_t* solid, void* A, void* B, cudaStream_t st) {
    set_last_launch_count(1);
    k_init_eos<<<nblocks(g.N, 128), 128, 0, st>>>(n, eps, beta, solid, (double*)A, (double*)B, g, ph);
    return cudaGetLastError();
}

cudaError_t launch_step_eos(const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt, bool count,
                            long long step_index, cudaStream_t st) {
    set_last_launch_count(1);
    const unsigned nb = nblocks(g.N, 128);
    const int cs = count ? 1 : 0;
    switch (g.xbc) {
        case XBC_PERIODIC:
            k_step_eos<XBC_PERIODIC><<<nb, 128, 0, st>>>((const double*)A, (double*)B, g, ph, cnt, cs, step_index);
            break;
        case XBC_INFLOW_OUTFLOW:
            k_step_eos<XBC_INFLOW_OUTFLOW><<<nb, 128, 0, st>>>((const double*)A, (double*)B, g, ph, cnt, cs,
                                                               step_index);
            break;
        default:
            k_step_eos<XBC_OUTFLOW_BOTH><<<nb, 128, 0, st>>>((const double*)A, (double*)B, g, ph, cnt, cs,
                                                             step_index);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_macro_eos(const Geom& g, const Phys& ph, const void* A, double* n, double* eps, double* beta,
                             Counters cnt, cudaStream_t st) {
    set_last_launch_count(1);
    k_macro_eos<<<nblocks(g.N, 128), 128, 0, st>>>((const double*)A, n, eps, beta, g, ph, cnt.macro_bad);
    return cudaGetLastError();
}

// Bounds-check count of this translation unit (0 in the release build).
RLB_OOB_TAKE_FN(oob_take_eos)

}  // namespace rlb

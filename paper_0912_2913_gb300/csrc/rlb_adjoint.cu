// rlb_adjoint.cu -- discrete adjoint of the relativistic lattice Boltzmann
// step (the transpose of the exact Jacobian of Eqs. lbe1/lbe2 with the
// eps = 3P equilibria Eqs. equil1s, equil2as, equil2bs and the closed-form
// recovery), the adjoint of the macroscopic output and of the equilibrium
// initialisation.
//
// Step adjoint, push form.  With lambda_{t+1} = dL/dA_{t+1}, one thread per
// interior fluid cell x
//   1. gathers h(x) from A_t exactly as the forward step does,
//   2. takes mu(x) = lambda_{t+1}(x) (+ lambda_{t+1} of the outflow ghost that
//      copies x),
//   3. forms nu = J_C(h)^T mu, where C(h) = h + (eq(m(h)) - h)/tau:
//        nu = (1 - 1/tau) mu + (1/tau) P^T (d eq / d m)^T mu,
//      m = P h the five moments, by the chain rule through the equilibria and
//      the recovery (the partial derivatives are written out below),
//   4. scatters nu_i to lambda_t(x - e_i, i), or to lambda_t(x, opp(i)) when
//      x - e_i is solid (transpose of the pull with bounce-back).
// Every element of lambda_t has exactly one writer: the scatter above, or
// the owner cell writing 0 where nobody reads the population (a neighbour
// that is a ghost plane), or the identity at solid cells (never updated).
// dL/dtau = sum mu_i (h_i - eq_i)/tau^2 and, at the inflow plane (held at
// eq(n_in, eps_in, beta_in)), dL/dbeta_in = sum lambda_{t+1} d eq/d beta_in
// are summed per warp (binary32 for the FP32 path, binary64 otherwise) and
// then over the warp partials in a fixed order (k_finalize).
#include <cuda.h>  // CUcontext type only; cuCtxGetCurrent is taken through the runtime
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "rlb_device.cuh"

namespace rlb {

// ---------------------------------------------------------------------------
// Adjoint of the g equilibria (Eqs. equil2as, equil2bs) with respect to
// (eps, beta) at fixed mu:   a_eps = sum mu_i d g_i / d eps,
//                            a_beta = sum mu_i d g_i / d beta.
// g_{+-p} = w_p [eps/c_l^2 + eps gamma^2 (6 q_p^2 - 2 b2)/c_l^2] +- w_p eps gamma^2 4 q_p / c_l
// g_0     = w_0 [4 eps gamma^2 - eps (2 + c_l^2)/c_l^2 - 2 eps gamma^2 b2 / c_l^2]
// with q_p = e_p . beta, b2 = |beta|^2, d gamma^2 / d beta = 2 gamma^4 beta.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void g_eq_adjoint(const T* mug, T eps, T bx, T by, T bz, T b2, T gam2, T inv_cl,
                                             T inv_cl2, T& a_eps, T& abx, T& aby, T& abz) {
    const T q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    T ae = 0, gg2 = 0, gb2 = 0;  // d/d eps, d/d gamma^2, d/d b2 (explicit)
    T Qp[9];
    T sw = 0;  // sum_p w_p sigma_p
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const T w = (T)pair_w(p);
        const T sig = mug[2 * p + 1] + mug[2 * p + 2];
        const T del = mug[2 * p + 1] - mug[2 * p + 2];
        const T sym = (6 * q[p] * q[p] - 2 * b2) * inv_cl2;
        const T asy = 4 * q[p] * inv_cl;
        ae += w * (sig * (inv_cl2 + gam2 * sym) + del * gam2 * asy);
        gg2 += w * (sig * sym + del * asy);
        sw += w * sig;
        // d/dq_p: w eps gamma^2 (sigma 12 q / c_l^2 + delta 4 / c_l)
        Qp[p] = w * (sig * 12 * q[p] * inv_cl2 + del * 4 * inv_cl);
    }
    const T w0 = (T)kW0;
    const T m0 = mug[0];
    ae += w0 * m0 * (4 * gam2 - (2 * inv_cl2 + 1) - 2 * gam2 * b2 * inv_cl2);
    gg2 += w0 * m0 * (4 - 2 * b2 * inv_cl2);
    gb2 = -2 * gam2 * inv_cl2 * (sw + w0 * m0);
    // chain: gamma^2 (factor eps), b2 (factor eps), q_p (factor eps gamma^2)
    const T eg = eps * gam2;
    const T rad = 2 * eps * (gb2 + gam2 * gam2 * gg2);  // coefficient of beta_a
    a_eps = ae;
    abx = eg * (Qp[0] + Qp[3] + Qp[4] + Qp[5] + Qp[6]) + rad * bx;
    aby = eg * (Qp[1] + Qp[3] - Qp[4] + Qp[7] + Qp[8]) + rad * by;
    abz = eg * (Qp[2] + Qp[5] - Qp[6] + Qp[7] - Qp[8]) + rad * bz;
}

// Adjoint of the f equilibria written as f_i = w_i S (1 + 3 q_i / c_l) with
// S = n gamma held fixed: a_S = sum mu_i w_i (1 + 3 q_i/c_l),
// a_beta = (3 S / c_l) sum_i mu_i w_i e_i.
template <typename T>
__device__ __forceinline__ void f_eq_adjoint_S(const T* muf, T S, T bx, T by, T bz, T inv_cl, T& aS, T& abx, T& aby,
                                               T& abz) {
    const T q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    T s0 = (T)kW0 * muf[0], s1 = 0;
    T d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const T w = (T)pair_w(p);
        s0 += w * (muf[2 * p + 1] + muf[2 * p + 2]);
        d[p] = w * (muf[2 * p + 1] - muf[2 * p + 2]);
        s1 += d[p] * q[p];
    }
    aS = s0 + 3 * inv_cl * s1;
    const T c = 3 * S * inv_cl;
    abx = c * (d[0] + d[3] + d[4] + d[5] + d[6]);
    aby = c * (d[1] + d[3] - d[4] + d[7] + d[8]);
    abz = c * (d[2] + d[5] - d[6] + d[7] - d[8]);
}

// Adjoint of the closed-form recovery: given adjoints (a_eps, a_beta) of
// eps = s - E and beta = 3M/D (s = sqrt(4E^2 - 3M^2), D = 3E + eps), the
// adjoints of E and M:
//   d eps/dE = 4E/s - 1,          d eps/dM_b = -3 M_b / s,
//   d beta_a/dE = -(beta_a/D)(3 + d eps/dE),
//   d beta_a/dM_b = 3 delta_ab / D + 3 beta_a M_b / (D s).
template <typename T>
__device__ __forceinline__ void recovery_adjoint(T a_eps, T abx, T aby, T abz, T E, T s, T D, T bx, T by, T bz, T Mx,
                                                 T My, T Mz, T& vE, T& vx, T& vy, T& vz) {
    const T ab_b = abx * bx + aby * by + abz * bz;
    const T rD = 1 / D;
    const T rs = 1 / s;
    const T depsdE = 4 * E * rs - 1;
    vE = a_eps * depsdE - ab_b * rD * (3 + depsdE);
    const T c = 3 * rs * (ab_b * rD - a_eps);
    vx = 3 * abx * rD + c * Mx;
    vy = 3 * aby * rD + c * My;
    vz = 3 * abz * rD + c * Mz;
}

// Warp partial sums written to red[(global warp)*4 + k], no block barrier:
// tau in binary32 across the warp for the FP32 path (the per-cell terms are
// binary32 already), the beta_in terms only when a lane has one.
template <typename T>
__device__ __forceinline__ void warp_partials(double tau, double b0, double b1, double b2, bool has_b, double* red) {
    const unsigned full = 0xffffffffu;
    double v0;
    if constexpr (sizeof(T) == 4) {
        float t = (float)tau;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(full, t, off);
        v0 = (double)t;
    } else {
        v0 = tau;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v0 += __shfl_xor_sync(full, v0, off);
    }
    double v1 = b0, v2 = b1, v3 = b2;
    if (__any_sync(full, has_b)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v1 += __shfl_xor_sync(full, v1, off);
            v2 += __shfl_xor_sync(full, v2, off);
            v3 += __shfl_xor_sync(full, v3, off);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        red[wg * 4 + 0] = v0;
        red[wg * 4 + 1] = v1;
        red[wg * 4 + 2] = v2;
        red[wg * 4 + 3] = v3;
    }
}

// Block reduction of four doubles into red[blockIdx.x*4 + k].
__device__ __forceinline__ void block_reduce4(double v0, double v1, double v2, double v3, double* red) {
    __shared__ double sm[4][32];
    double v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sm[k][warp] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double t = lane < nw ? sm[k][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
            if (lane == 0) red[blockIdx.x * 4 + k] = t;
        }
    }
}

// Sum the partial-sum slots (one per warp or per block, 4 doubles each) and
// add them to the accumulators.  256 threads per component; thread t sums
// slots t, t+256, ... in a fixed grouping, then a fixed tree combines the 256
// sums: the result does not depend on scheduling.
__global__ void __launch_bounds__(1024) k_finalize(const double* __restrict__ red, int nslots, double* dtau,
                                                   double* dbeta_in) {
    __shared__ double sm[4][256];
    const int k = threadIdx.x >> 8, t = threadIdx.x & 255;
    // eight independent partial sums so that eight loads are in flight; the
    // grouping depends only on nslots (deterministic)
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int b = t;
    for (; b + 7 * 256 < nslots; b += 8 * 256) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] += red[(b + j * 256) * 4 + k];
    }
#pragma unroll
    for (int j = 0; j < 7; ++j)
        if (b + j * 256 < nslots) a[j] += red[(b + j * 256) * 4 + k];
    sm[k][t] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) sm[k][t] += sm[k][t + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (dtau) *dtau += sm[0][0];
        if (dbeta_in) {
            dbeta_in[0] += sm[1][0];
            dbeta_in[1] += sm[2][0];
            dbeta_in[2] += sm[3][0];
        }
    }
}

// Adjoint of eq(n, eps, beta) with respect to the fields (f with n gamma,
// gamma = (1 - b2)^-1/2, d gamma / d beta = gamma^3 beta).
__device__ __noinline__ void eq_fields_adjoint(const double* muf, const double* mug, double n, double eps, double bx, double by,
                                  double bz, const Phys& ph, double& an, double& ae, double& abx, double& aby,
                                  double& abz) {
    const double b2 = bx * bx + by * by + bz * bz;
    const double gam2 = 1.0 / (1.0 - b2);
    const double gam = sqrt(gam2);
    double aS, fbx, fby, fbz;
    f_eq_adjoint_S(muf, n * gam, bx, by, bz, ph.inv_cl, aS, fbx, fby, fbz);
    // S = n gamma: dS/dn = gamma, dS/dbeta = n gamma^3 beta
    an = aS * gam;
    const double cS = aS * n * gam * gam2;
    double gbx, gby, gbz;
    g_eq_adjoint(mug, eps, bx, by, bz, b2, gam2, ph.inv_cl, ph.inv_cl2, ae, gbx, gby, gbz);
    abx = fbx + gbx + cS * bx;
    aby = fby + gby + cS * by;
    abz = fbz + gbz + cS * bz;
}

// ---------------------------------------------------------------------------
// Step adjoint.  T = double: FP64 states and arithmetic.  T = float: FP32
// deviation states, binary32 arithmetic throughout (the recovery in the
// cancellation-free deviation form of cell_g).  Per cell two phases, g then
// f.  The per-cell mathematics (cell_g, cell_f, scatter_cell) is shared by
// the register kernel and the shared-memory staged kernel.
// ---------------------------------------------------------------------------
template <typename T>
struct AdjConst {
    T om, omw, c_l, inv_cl, inv_cl2, n_ref, g0a, g0b, eps_ref_t, inv_tau2_t;
    double inv_tau2;
    // per-run products for the binary64 cell functions (cell_g64 and after);
    // the _36 ones divided by 36, for the pair sums carried times 36
    double c2, c2p1;                  // 2/c_l^2, 2/c_l^2 + 1
    double i2_36, c2_36, c3_36, c4_36, c6_36, c12_36;  // 1/c_l^2, 2/c_l^2, 3/c_l, 4/c_l, 6/c_l^2, 12/c_l^2
    double three_cl, m3cl2, om_cl;    // 3 c_l, -3 c_l^2, omega c_l
    double g0_eg, g0_e, g0_egb2;      // g_0^eq = eg g0_eg + eps g0_e + eg b2 g0_egb2
};

template <typename T>
static AdjConst<T> make_adj_const(const Phys& ph) {
    AdjConst<T> c;
    c.om = (T)ph.omega;
    c.omw = (T)(1.0 - ph.omega);
    c.c_l = (T)ph.c_l;
    c.inv_cl = (T)ph.inv_cl;
    c.inv_cl2 = (T)ph.inv_cl2;
    c.n_ref = (T)ph.n_ref;
    c.g0a = (T)(3.0 - 2.0 * ph.inv_cl2);
    c.g0b = (T)(4.0 - 2.0 * ph.inv_cl2);
    c.eps_ref_t = (T)ph.eps_ref;
    c.inv_tau2 = ph.omega * ph.omega;
    c.inv_tau2_t = (T)c.inv_tau2;
    c.c2 = 2.0 * ph.inv_cl2;
    c.i2_36 = ph.inv_cl2 / 36.0;
    c.c2_36 = 2.0 * ph.inv_cl2 / 36.0;
    c.c3_36 = 3.0 * ph.inv_cl / 36.0;
    c.c4_36 = 4.0 * ph.inv_cl / 36.0;
    c.c6_36 = 6.0 * ph.inv_cl2 / 36.0;
    c.c12_36 = 12.0 * ph.inv_cl2 / 36.0;
    c.three_cl = 3.0 * ph.c_l;
    c.m3cl2 = -3.0 * ph.c_l * ph.c_l;
    c.om_cl = ph.omega * ph.c_l;
    c.g0_eg = 4.0 * kW0;
    c.g0_e = -kW0 * (2.0 * ph.inv_cl2 + 1.0);
    c.g0_egb2 = -2.0 * kW0 * ph.inv_cl2;
    c.c2p1 = 2.0 * ph.inv_cl2 + 1.0;
    return c;
}

// Sums over the 19 populations as shallow trees (independent partial sums
// instead of one 18-deep dependency chain).
template <typename T>
__device__ __forceinline__ T sum19(const T* h) {
    const T a0 = h[0] + h[1], a1 = h[2] + h[3], a2 = h[4] + h[5], a3 = h[6] + h[7], a4 = h[8] + h[9];
    const T a5 = h[10] + h[11], a6 = h[12] + h[13], a7 = h[14] + h[15], a8 = h[16] + h[17];
    return ((a0 + a1) + (a2 + a3)) + (((a4 + a5) + (a6 + a7)) + (a8 + h[18]));
}
template <typename T>
__device__ __forceinline__ T dot19(const T* a, const T* b) {
    T s0 = a[0] * b[0], s1 = a[1] * b[1], s2 = a[2] * b[2], s3 = a[3] * b[3];
#pragma unroll
    for (int i = 4; i < 16; i += 4) {
        s0 += a[i] * b[i];
        s1 += a[i + 1] * b[i + 1];
        s2 += a[i + 2] * b[i + 2];
        s3 += a[i + 3] * b[i + 3];
    }
    s0 += a[16] * b[16];
    s1 += a[17] * b[17];
    s2 += a[18] * b[18];
    return (s0 + s1) + (s2 + s3);
}

// What the g phase leaves for the f phase and the recovery adjoint.
template <typename T>
struct CellG {
    T mx, my, mz, Et, sqt, Dt, bx, by, bz;  // moments (cell_g64: M / c_l), recovery
    T tacc, ae, gbx, gby, gbz;              // sum mu_g (h - eq), d/d eps, d/d beta
    T rD, rs;                               // 1/D, 1/s (cell_g64)
};

// Moments and recovery from the 19 g populations h, then the g part of the
// collision adjoint at mu = mug.
template <typename T>
__device__ __forceinline__ void cell_g(const T* h, const T* mug, const AdjConst<T>& c, CellG<T>& r) {
    const T dE = sum19(h);
    T dd[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) dd[p] = h[2 * p + 1] - h[2 * p + 2];
    const T mx = c.c_l * (dd[0] + dd[3] + dd[4] + dd[5] + dd[6]);
    const T my = c.c_l * (dd[1] + dd[3] - dd[4] + dd[7] + dd[8]);
    const T mz = c.c_l * (dd[2] + dd[5] - dd[6] + dd[7] - dd[8]);
    T Et, sqt, Dt, epst, e0, bx, by, bz, b2, gam2;
    if constexpr (sizeof(T) == 8) {
        const double E = dE;
        const double sq = sqrt(4.0 * E * E - 3.0 * (mx * mx + my * my + mz * mz));
        const double eps = sq - E;
        const double D = 3.0 * E + eps;
        const double r3 = 3.0 / D;
        bx = mx * r3;
        by = my * r3;
        bz = mz * r3;
        b2 = bx * bx + by * by + bz * bz;
        gam2 = 1.0 / (1.0 - b2);
        Et = E;
        sqt = sq;
        Dt = D;
        epst = eps;
        e0 = eps;
    } else {
        // binary32 in deviation form (the coefficients of the adjoint need
        // no FP64): E = eps_ref + dE, s = sqrt(E^2 - 3/4 M^2), eps = 2 s - E,
        // and the deviation eps - eps_ref = 2 (s - eps_ref) - dE with
        // s - eps_ref = (dE (2 eps_ref + dE) - 3/4 M^2) / (s + eps_ref),
        // free of the cancellation of eps - eps_ref.
        const float er = c.eps_ref_t;
        const float m34 = 0.75f * fmaf(mx, mx, fmaf(my, my, mz * mz));
        const float num = fmaf(dE, fmaf(2.0f, er, dE), -m34);
        const float sr = sqrtf(fmaf(er, er, num));
        e0 = fmaf(2.0f, __fdividef(num, sr + er), -dE);
        epst = er + e0;
        Et = er + dE;
        sqt = 2.0f * sr;
        Dt = fmaf(3.0f, Et, epst);
        const float r3 = __fdividef(3.0f, Dt);
        bx = mx * r3;
        by = my * r3;
        bz = mz * r3;
        b2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
        gam2 = __fdividef(1.0f, 1.0f - b2);
    }
    const T q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    const T eg = epst * gam2;
    // Everything the collision adjoint needs from mu reduces to a few
    // weighted pair sums (sigma_p = mu_{+p} + mu_{-p}, delta_p = mu_{+p} -
    // mu_{-p}, weight w_p, q_p = e_p . beta):
    //   S1 = sum w sigma,  Sq2 = sum w sigma q^2,  Sdq = sum w delta q,
    //   Vq = sum w sigma q e_p,  Vd = sum w delta e_p.
    // With them (Eqs. equil2as/equil2bs and their derivatives):
    //   sum mu_i geq_i = mu_0 geq_0 + k1 S1 + k2 Sq2 + k3 Sdq,
    //   d/d eps = S1/c_l^2 + gamma^2 (SYM + ASY) + rest-particle term,
    //   d/d gamma^2 = eps (SYM + ASY + rest term), d/d b2 = -2 eps gamma^2 (S1 + w0 mu_0)/c_l^2,
    //   d/d beta = eps gamma^2 (12 Vq / c_l^2 + 4 Vd / c_l) + (chain through gamma^2 and b2) beta,
    // SYM = (6 Sq2 - 2 b2 S1)/c_l^2, ASY = 4 Sdq / c_l; and likewise for f.
    const T muh = dot19(mug, h);
    T S1 = 0, Sq2 = 0, Sdq = 0, Vq[3] = {0, 0, 0}, Vd[3] = {0, 0, 0};
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const T w = (T)pair_w(p);
        const T ws = w * (mug[2 * p + 1] + mug[2 * p + 2]);
        const T wd = w * (mug[2 * p + 1] - mug[2 * p + 2]);
        S1 += ws;
        const T wsq = ws * q[p];
        Sq2 += wsq * q[p];
        Sdq += wd * q[p];
        const int ex = pair_ex(p), ey = pair_ey(p), ez = pair_ez(p);
        if (ex) { Vq[0] += wsq; Vd[0] += wd; }
        if (ey > 0) { Vq[1] += wsq; Vd[1] += wd; }
        if (ey < 0) { Vq[1] -= wsq; Vd[1] -= wd; }
        if (ez > 0) { Vq[2] += wsq; Vd[2] += wd; }
        if (ez < 0) { Vq[2] -= wsq; Vd[2] -= wd; }
    }
    const T m0 = mug[0], w0 = (T)kW0;
    const T k1 = (e0 - 2 * eg * b2) * c.inv_cl2, k2 = 6 * eg * c.inv_cl2, k3 = 4 * eg * c.inv_cl;
    const T geq0 = (sizeof(T) == 8) ? w0 * (4 * eg - epst * (2 * c.inv_cl2 + 1) - 2 * eg * b2 * c.inv_cl2)
                                    : w0 * (e0 * c.g0a + eg * b2 * c.g0b);
    r.tacc = muh - (m0 * geq0 + k1 * S1 + k2 * Sq2 + k3 * Sdq);
    const T SYM = (6 * Sq2 - 2 * b2 * S1) * c.inv_cl2;
    const T ASY = 4 * c.inv_cl * Sdq;
    r.ae = c.inv_cl2 * S1 + gam2 * (SYM + ASY) + w0 * m0 * (4 * gam2 - (2 * c.inv_cl2 + 1) - 2 * gam2 * b2 * c.inv_cl2);
    const T gg2 = SYM + ASY + w0 * m0 * (4 - 2 * b2 * c.inv_cl2);
    const T gb2 = -2 * gam2 * c.inv_cl2 * (S1 + w0 * m0);
    const T rad = 2 * epst * (gb2 + gam2 * gam2 * gg2);
    const T cq = eg * 12 * c.inv_cl2, cd = eg * 4 * c.inv_cl;
    r.gbx = cq * Vq[0] + cd * Vd[0] + rad * bx;
    r.gby = cq * Vq[1] + cd * Vd[1] + rad * by;
    r.gbz = cq * Vq[2] + cd * Vd[2] + rad * bz;
    r.mx = mx;
    r.my = my;
    r.mz = mz;
    r.Et = Et;
    r.sqt = sqt;
    r.Dt = Dt;
    r.bx = bx;
    r.by = by;
    r.bz = bz;
}

// The f part: sum mu_f (h - eq) and the adjoints of S = n gamma and beta.
template <typename T>
__device__ __forceinline__ void cell_f(const T* h, const T* muf, const CellG<T>& r, const AdjConst<T>& c, T& tacc,
                                       T& aS, T& fbx, T& fby, T& fbz) {
    const T q[9] = {r.bx, r.by, r.bz, r.bx + r.by, r.bx - r.by, r.bx + r.bz, r.bx - r.bz, r.by + r.bz, r.by - r.bz};
    const T dS = sum19(h);
    const T Sfull = (sizeof(T) == 8) ? dS : dS + c.n_ref;
    const T muh = dot19(muf, h);
    T F1 = 0, Fdq = 0, Vf[3] = {0, 0, 0};
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const T w = (T)pair_w(p);
        const T ws = w * (muf[2 * p + 1] + muf[2 * p + 2]);
        const T wd = w * (muf[2 * p + 1] - muf[2 * p + 2]);
        F1 += ws;
        Fdq += wd * q[p];
        const int ex = pair_ex(p), ey = pair_ey(p), ez = pair_ez(p);
        if (ex) Vf[0] += wd;
        if (ey > 0) Vf[1] += wd;
        if (ey < 0) Vf[1] -= wd;
        if (ez > 0) Vf[2] += wd;
        if (ez < 0) Vf[2] -= wd;
    }
    const T w0 = (T)kW0;
    const T fa = 3 * Sfull * c.inv_cl;
    // f^eq_{+-p} = w_p (fb +- fa q_p), fb = S (values) or dS (deviations)
    tacc = muh - (muf[0] * w0 * dS + dS * F1 + fa * Fdq);
    aS = w0 * muf[0] + F1 + 3 * c.inv_cl * Fdq;
    fbx = fa * Vf[0];
    fby = fa * Vf[1];
    fbz = fa * Vf[2];
}

// nu = (1 - 1/tau) mu + (1/tau) P^T v for the 38 populations of the cell,
// handed to put(plane, velocity, value) (the transpose of the pull).
template <typename T, typename PUT>
__device__ __forceinline__ void scatter_cell(const T* muf, const T* mug, T aS, T vE, T vx, T vy, T vz,
                                             const AdjConst<T>& c, PUT put) {
    const T nuS = c.om * aS, nuE = c.om * vE;
#pragma unroll
    for (int i = 0; i < 19; ++i) put(i, i, c.omw * muf[i] + nuS);
    put(19, 0, c.omw * mug[0] + nuE);
    const T pm[9] = {vx, vy, vz, vx + vy, vx - vy, vx + vz, vx - vz, vy + vz, vy - vz};
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const T t = c.om * c.c_l * pm[p];
        put(20 + 2 * p, 2 * p + 1, c.omw * mug[2 * p + 1] + nuE + t);
        put(21 + 2 * p, 2 * p + 2, c.omw * mug[2 * p + 2] + nuE - t);
    }
}

// ---------------------------------------------------------------------------
// The same per-cell mathematics in binary64 with fewer FP64 instructions
// (the FP64 pipe bounds the FP64 adjoint):
//  * the square root and the reciprocals 1/D, 1/(1 - b2), 1/s from binary32
//    seeds and two Newton steps each (the forward step's recovery), 1/D and
//    1/s computed once for the recovery and its adjoint;
//  * the per-run products of 1/c_l, the weights and omega folded (AdjConst);
//    the weighted pair sums are carried times 36 (weights 2 and 1), the
//    1/36 folded into their coefficients;
//  * the pair sums that depend on beta formed from beta-free moments of mu:
//    with q_p = e_p . beta,
//      Sdq = sum w delta_p q_p = beta . Vd,     Vd = sum w delta_p e_p,
//      Vq  = sum w sigma_p q_p e_p = T beta,    T  = sum w sigma_p e_p e_p^T,
//      Sq2 = sum w sigma_p q_p^2 = beta . Vq.
// ---------------------------------------------------------------------------

// x = 1/a from a binary32 seed and two Newton steps
__device__ __forceinline__ double rcp_newton(double a) {
    double x = rcp_seed(a);
    x = fma(x, fma(-a, x, 1.0), x);
    return fma(x, fma(-a, x, 1.0), x);
}

// 36 sum w s_p (36 w = 2 for the axis pairs, 1 for the diagonal ones)
__device__ __forceinline__ double wsum9(const double* s) {
    return fma(2.0, (s[0] + s[1]) + s[2], ((s[3] + s[4]) + (s[5] + s[6])) + (s[7] + s[8]));
}
// 36 sum w d_p e_p (three components)
__device__ __forceinline__ void wvec9(const double* d, double& vx, double& vy, double& vz) {
    vx = fma(2.0, d[0], (d[3] + d[4]) + (d[5] + d[6]));
    vy = fma(2.0, d[1], (d[3] - d[4]) + (d[7] + d[8]));
    vz = fma(2.0, d[2], (d[5] - d[6]) + (d[7] - d[8]));
}

__device__ __forceinline__ void cell_g64(const double* h, const double* mug, const AdjConst<double>& c,
                                         CellG<double>& r) {
    const double E = sum19(h);
    double dd[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) dd[p] = h[2 * p + 1] - h[2 * p + 2];
    double dx, dy, dz;  // M / c_l
    dx = dd[0] + dd[3] + dd[4] + dd[5] + dd[6];
    dy = dd[1] + dd[3] - dd[4] + dd[7] + dd[8];
    dz = dd[2] + dd[5] - dd[6] + dd[7] - dd[8];
    const double m2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double disc = fma(4.0 * E, E, c.m3cl2 * m2);  // 4 E^2 - 3 M^2
    double ys, hs;
    rsqrt_seed(disc, ys, hs);
    double sq = disc * ys;
    sq = fma(fma(-sq, sq, disc), hs, sq);
    sq = fma(fma(-sq, sq, disc), hs, sq);
    const double eps = sq - E;
    const double D = fma(3.0, E, eps);
    const double rD = rcp_newton(D);
    const double r3 = c.three_cl * rD;  // beta = 3 M / D
    const double bx = dx * r3, by = dy * r3, bz = dz * r3;
    const double b2 = (r3 * r3) * m2;
    const double gam2 = rcp_newton(1.0 - b2);
    // beta-free moments of mu_g (all times 36)
    double sg[9], dg[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        sg[p] = mug[2 * p + 1] + mug[2 * p + 2];
        dg[p] = mug[2 * p + 1] - mug[2 * p + 2];
    }
    const double s34 = sg[3] + sg[4], s56 = sg[5] + sg[6], s78 = sg[7] + sg[8];
    const double S1 = fma(2.0, (sg[0] + sg[1]) + sg[2], (s34 + s56) + s78);
    const double Txx = fma(2.0, sg[0], s34 + s56);
    const double Tyy = fma(2.0, sg[1], s34 + s78);
    const double Tzz = fma(2.0, sg[2], s56 + s78);
    const double Txy = sg[3] - sg[4], Txz = sg[5] - sg[6], Tyz = sg[7] - sg[8];
    double Vdx, Vdy, Vdz;
    wvec9(dg, Vdx, Vdy, Vdz);
    const double Vqx = fma(Txx, bx, fma(Txy, by, Txz * bz));
    const double Vqy = fma(Txy, bx, fma(Tyy, by, Tyz * bz));
    const double Vqz = fma(Txz, bx, fma(Tyz, by, Tzz * bz));
    const double Sq2 = fma(Vqx, bx, fma(Vqy, by, Vqz * bz));
    const double Sdq = fma(Vdx, bx, fma(Vdy, by, Vdz * bz));
    // the coefficients (Eqs. equil2as/equil2bs and their derivatives), the
    // 1/36 of the sums folded into them
    const double eg = eps * gam2, egb2 = eg * b2;
    const double m0 = mug[0], w0m0 = kW0 * m0;
    const double k1 = fma(-2.0, egb2, eps) * c.i2_36, k2 = eg * c.c6_36, k3 = eg * c.c4_36;
    const double geq0 = fma(eg, c.g0_eg, fma(eps, c.g0_e, egb2 * c.g0_egb2));
    r.tacc = dot19(mug, h) - fma(m0, geq0, fma(k1, S1, fma(k2, Sq2, k3 * Sdq)));
    const double SA = fma(c.c6_36, Sq2, fma(-c.c2_36 * b2, S1, c.c4_36 * Sdq));  // SYM + ASY
    const double t4 = fma(-c.c2, b2, 4.0);                                          // 4 - 2 b2 / c_l^2
    r.ae = fma(c.i2_36, S1, fma(gam2, SA, w0m0 * fma(gam2, t4, -c.c2p1)));
    const double gg2 = fma(w0m0, t4, SA);
    const double gb2 = -(c.c2 * gam2) * fma(S1, 1.0 / 36.0, w0m0);
    const double rad = (2.0 * eps) * fma(gam2 * gam2, gg2, gb2);
    const double cq = eg * c.c12_36;  // the Vd coefficient is k3
    r.gbx = fma(cq, Vqx, fma(k3, Vdx, rad * bx));
    r.gby = fma(cq, Vqy, fma(k3, Vdy, rad * by));
    r.gbz = fma(cq, Vqz, fma(k3, Vdz, rad * bz));
    r.mx = dx;
    r.my = dy;
    r.mz = dz;
    r.Et = E;
    r.sqt = sq;
    r.Dt = D;
    r.rD = rD;
    r.rs = rcp_newton(sq);
    r.bx = bx;
    r.by = by;
    r.bz = bz;
}

__device__ __forceinline__ void cell_f64(const double* h, const double* muf, const CellG<double>& r,
                                         const AdjConst<double>& c, double& tacc, double& aS, double& fbx,
                                         double& fby, double& fbz) {
    const double dS = sum19(h);
    double sf[9], df[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        sf[p] = muf[2 * p + 1] + muf[2 * p + 2];
        df[p] = muf[2 * p + 1] - muf[2 * p + 2];
    }
    const double F1 = wsum9(sf);  // sums times 36
    double Vx, Vy, Vz;
    wvec9(df, Vx, Vy, Vz);
    const double Fdq = fma(Vx, r.bx, fma(Vy, r.by, Vz * r.bz));
    const double fa = c.c3_36 * dS;  // (3 S / c_l) / 36
    // f^eq_{+-p} = w_p (S +- 3 S q_p / c_l)
    tacc = dot19(muf, h) - fma(kW0 * muf[0], dS, fma(dS * (1.0 / 36.0), F1, fa * Fdq));
    aS = fma(F1, 1.0 / 36.0, fma(c.c3_36, Fdq, kW0 * muf[0]));
    fbx = fa * Vx;
    fby = fa * Vy;
    fbz = fa * Vz;
}

// recovery_adjoint with 1/D and 1/s given and d = M / c_l
__device__ __forceinline__ void recovery_adjoint64(double a_eps, double abx, double aby, double abz,
                                                   const CellG<double>& r, const AdjConst<double>& c, double& vE,
                                                   double& vx, double& vy, double& vz) {
    const double abD = fma(abx, r.bx, fma(aby, r.by, abz * r.bz)) * r.rD;
    const double depsdE = fma(4.0 * r.Et, r.rs, -1.0);
    vE = fma(a_eps, depsdE, -abD * (3.0 + depsdE));
    const double cc = (c.three_cl * r.rs) * (abD - a_eps);  // 3 (ab.beta / D - a_eps) / s, times c_l
    const double rD3 = 3.0 * r.rD;
    vx = fma(cc, r.mx, abx * rD3);
    vy = fma(cc, r.my, aby * rD3);
    vz = fma(cc, r.mz, abz * rD3);
}

template <typename PUT>
__device__ __forceinline__ void scatter_cell64(const double* muf, const double* mug, double aS, double vE, double vx,
                                               double vy, double vz, const AdjConst<double>& c, PUT put) {
    const double nuS = c.om * aS, nuE = c.om * vE;
#pragma unroll
    for (int i = 0; i < 19; ++i) put(i, i, fma(c.omw, muf[i], nuS));
    put(19, 0, fma(c.omw, mug[0], nuE));
    const double ux = c.om_cl * vx, uy = c.om_cl * vy, uz = c.om_cl * vz;
    const double t[9] = {ux, uy, uz, ux + uy, ux - uy, ux + uz, ux - uz, uy + uz, uy - uz};
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        put(20 + 2 * p, 2 * p + 1, fma(c.omw, mug[2 * p + 1], nuE) + t[p]);
        put(21 + 2 * p, 2 * p + 2, fma(c.omw, mug[2 * p + 2], nuE) - t[p]);
    }
}

// A ghost plane cell (non-periodic x): nobody reads its populations that do
// not point into the lattice; the others are written by the scatter of x +- 1.
// At the inflow plane (held at eq(n_in, eps_in, beta_in)) its adjoint adds
// lambda_{t+1} . d eq_in / d beta_in (a per-context table).
// TERMS = false: only the zeros (the dL/dbeta_in terms taken elsewhere).
template <typename T, int XBC, bool TERMS = true>
__device__ __forceinline__ void ghost_cell(int x, int idx, long long S, const T* __restrict__ A,
                                           const T* __restrict__ Lin, T* __restrict__ Lout,
                                           const T* __restrict__ inflow_t, double& bin0, double& bin1,
                                           double& bin2, bool& has_b) {
    const int inward = (x == 0) ? 1 : -1;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (vel_x(i) != inward) {
            Lout[RLB_CHK(i * S + idx, 38ll * S)] = (T)0;
            Lout[RLB_CHK((19 + i) * S + idx, 38ll * S)] = (T)0;
        }
    }
    if (TERMS && XBC == XBC_INFLOW_OUTFLOW && x == 0 && !is_solid(A[RLB_CHK(idx, 38ll * S)])) {
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 2
        for (int q = 0; q < 38; ++q) {
            const T l = Lin[RLB_CHK(q * S + idx, 38ll * S)];
            a0 += l * inflow_t[3 * q + 0];
            a1 += l * inflow_t[3 * q + 1];
            a2 += l * inflow_t[3 * q + 2];
        }
        bin0 += (double)a0;
        bin1 += (double)a1;
        bin2 += (double)a2;
        has_b = true;
    }
}

// Populations of x that a ghost plane would pull: nobody reads them.
template <typename T, int XBC>
__device__ __forceinline__ void zero_to_ghost(int x, int nx, int idx, long long S, T* __restrict__ Lout) {
    if (XBC != XBC_PERIODIC && (x == 1 || x == nx - 2)) {
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const bool to_ghost = (x == 1 && vel_x(i) == -1) || (x == nx - 2 && vel_x(i) == 1);
            if (to_ghost) {
                Lout[RLB_CHK(i * S + idx, 38ll * S)] = (T)0;
                Lout[RLB_CHK((19 + i) * S + idx, 38ll * S)] = (T)0;
            }
        }
    }
}

// mu offset of the outflow ghost that copies x (0 if none)
template <int XBC>
__device__ __forceinline__ int dup_of(int x, int nx) {
    return (XBC != XBC_PERIODIC && x == nx - 2) ? 1 : ((XBC == XBC_OUTFLOW_BOTH && x == 1) ? -1 : 0);
}

// Register kernel.  PIPE: persistent grid-stride loop over the cells;
// otherwise one cell per thread.
template <typename T, int XBC, int MINB, bool PIPE>
__global__ void __launch_bounds__(128, MINB)
    k_adjoint_step(const T* __restrict__ A, const T* __restrict__ Lin, T* __restrict__ Lout, Geom g, Phys ph,
                   AdjConst<T> c, double* red, const T* __restrict__ inflow_t) {
    const long long S = g.S;
    T tau_acc = 0;
    double bin0 = 0.0, bin1 = 0.0, bin2 = 0.0;
    bool has_b = false;
    const long long stride = PIPE ? (long long)gridDim.x * blockDim.x : (long long)g.N;
    // the loop ends for every thread before the warp reduction ('continue'
    // skips to the next cell); the counter is 64-bit so that the last
    // stride cannot wrap
    for (long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x; li < g.N; li += stride) {
        const int idx = (int)li;
        int x, y, z;
        cell_coords(g, idx, x, y, z);
        if constexpr (sizeof(T) == 8 && XBC == XBC_INFLOW_OUTFLOW) {
            // dL/dbeta_in at the fluid inflow ghosts of this warp, their 38
            // products with the table spread over the active lanes (one lane
            // issuing all 114 would take a full FP64 warp slot for each)
            const unsigned act = __activemask();
            unsigned m = __ballot_sync(act, x == 0 && !is_solid(A[RLB_CHK(idx, 38ll * S)]));
            if (m) {
                const int lane = threadIdx.x & 31;
                const int rank = __popc(act & ((1u << lane) - 1u)), cnt = __popc(act);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const int gidx = __shfl_sync(act, idx, src);
                    for (int q = rank; q < 38; q += cnt) {
                        const T l = Lin[RLB_CHK((long long)q * S + gidx, 38ll * S)];
                        bin0 = fma(l, inflow_t[3 * q + 0], bin0);
                        bin1 = fma(l, inflow_t[3 * q + 1], bin1);
                        bin2 = fma(l, inflow_t[3 * q + 2], bin2);
                    }
                    has_b = true;
                }
            }
        }
        if ((XBC != XBC_PERIODIC) && (x == 0 || x == g.nx - 1)) {
            if constexpr (sizeof(T) == 8 && XBC == XBC_INFLOW_OUTFLOW)
                ghost_cell<T, XBC, false>(x, idx, S, A, Lin, Lout, inflow_t, bin0, bin1, bin2, has_b);
            else
                ghost_cell<T, XBC>(x, idx, S, A, Lin, Lout, inflow_t, bin0, bin1, bin2, has_b);
            continue;
        }
        if (is_solid(A[RLB_CHK(19 * S + idx, 38ll * S)])) {  // never updated: identity
#pragma unroll
            for (int q = 0; q < 38; ++q) Lout[RLB_CHK(q * S + idx, 38ll * S)] = Lin[RLB_CHK(q * S + idx, 38ll * S)];
            continue;
        }
        const PullOffsets o(g, x, y, z);
        // mu = lambda_{t+1}(x), plus the outflow ghost that copies x
        const int dup = dup_of<XBC>(x, g.nx);
        // rare cases (a cell copied by an outflow ghost, links to solid cells)
        // take branches, so the common cell runs straight-line loads/stores
        auto load_mu = [&](T* mu, int base) {
#pragma unroll
            for (int i = 0; i < 19; ++i) mu[i] = Lin[RLB_CHK((base + i) * S + idx, 38ll * S)];
            if (dup) {
#pragma unroll
                for (int i = 0; i < 19; ++i) mu[i] += Lin[RLB_CHK((base + i) * S + idx + dup, 38ll * S)];
            }
        };
        if (!PIPE) {
            // f-phase populations and adjoints: start their trip from HBM into L2 now
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(RLB_CHK_PTR(A, i * S + idx + o.src(i), 38ll * S)));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(RLB_CHK_PTR(Lin, i * S + idx, 38ll * S)));
            }
        }
        // ---- g phase: gather, moments, recovery, g part of the adjoint
        unsigned bounced = 0u;
        T h[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) h[i] = A[RLB_CHK((19 + i) * S + idx + o.src(i), 38ll * S)];
        {
            // a pulled solid marker is a NaN: test the per-value markers only
            // when the sum of the gathered values is NaN
            if (isnan(sum19(h))) {
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    if (is_solid(h[i])) {
                        bounced |= 1u << i;
                        h[i] = A[RLB_CHK((19 + opp(i)) * S + idx, 38ll * S)];
                    }
                }
            }
        }
        T mug[19];
        load_mu(mug, 19);
        CellG<T> r;
        if constexpr (sizeof(T) == 8)
            cell_g64(h, mug, c, r);
        else
            cell_g(h, mug, c, r);
        // ---- f phase
#pragma unroll
        for (int i = 0; i < 19; ++i) h[i] = A[RLB_CHK(i * S + idx + o.src(i), 38ll * S)];
        if (bounced) {
#pragma unroll
            for (int i = 1; i < 19; ++i)
                if ((bounced >> i) & 1u) h[i] = A[RLB_CHK(opp(i) * S + idx, 38ll * S)];
        }
        T muf[19];
        load_mu(muf, 0);
        T tf, aS, fbx, fby, fbz;
        if constexpr (sizeof(T) == 8)
            cell_f64(h, muf, r, c, tf, aS, fbx, fby, fbz);
        else
            cell_f(h, muf, r, c, tf, aS, fbx, fby, fbz);
        tau_acc += (r.tacc + tf) * c.inv_tau2_t;
        T vE, vx, vy, vz;
        if constexpr (sizeof(T) == 8)
            recovery_adjoint64(r.ae, fbx + r.gbx, fby + r.gby, fbz + r.gbz, r, c, vE, vx, vy, vz);
        else
            recovery_adjoint<T>(r.ae, fbx + r.gbx, fby + r.gby, fbz + r.gbz, r.Et, r.sqt, r.Dt, r.bx, r.by, r.bz,
                                r.mx, r.my, r.mz, vE, vx, vy, vz);
        auto put = [&](int q, int i, T v) {
            if ((bounced >> i) & 1u)
                Lout[RLB_CHK((q - i + opp(i)) * S + idx, 38ll * S)] = v;
            else
                Lout[RLB_CHK(q * S + idx + o.src(i), 38ll * S)] = v;
        };
        if constexpr (sizeof(T) == 8)
            scatter_cell64(muf, mug, aS, vE, vx, vy, vz, c, put);
        else
            scatter_cell(muf, mug, aS, vE, vx, vy, vz, c, put);
        zero_to_ghost<T, XBC>(x, g.nx, idx, S, Lout);
    }
    warp_partials<T>((double)tau_acc, bin0, bin1, bin2, has_b, red);
}

// ---------------------------------------------------------------------------
// Shared-memory staged FP32 kernel.  Persistent grid-stride loop; every
// thread stages the 38 values of each phase of its cells (19 pulled
// populations + 19 lambda_{t+1}) in its own column of a three-slot ring with
// 4-byte cp.async copies, one phase ahead of the arithmetic:
//
//     issue F_k | wait G_k, compute G_k | issue G_k+1 | wait F_k, compute F_k, scatter
//
// so the loads of the next phase are in flight during the arithmetic of the
// current one without holding registers.  Slots: G_k, F_k, G_k+1 (the G slot
// stays valid through F_k, whose scatter reads mu_g).  Each thread reads only
// the slots it wrote, so cp.async.wait_group alone orders the accesses.
// ---------------------------------------------------------------------------
constexpr int kStageThreads = 128;
constexpr int kStageSlots = 3;
constexpr size_t kStageSmemBytes = sizeof(float) * kStageSlots * 38 * kStageThreads;

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Base address of each of the 38 planes of the three buffers, a kernel
// parameter: with every plane number a compile-time constant after
// unrolling, an address is a 32-bit cell offset added to a uniform base.
struct PlaneTab {
    const float* a[38];
    const float* l[38];
    float* o[38];
};

// Every address of a cell's populations is its plane's base from the table
// plus a 32-bit cell offset (N < 2^31): the fewest address instructions at any
// accepted lattice size.
template <int XBC>
__global__ void __launch_bounds__(kStageThreads, 3)
    k_adjoint_step_staged(const float* __restrict__ A, const float* __restrict__ Lin, float* __restrict__ Lout,
                          Geom g, Phys ph, AdjConst<float> c, double* red, const float* __restrict__ inflow_t,
                          const __grid_constant__ PlaneTab tab) {
    extern __shared__ float stage[];  // [slot][value 0..37][thread]
    const long long S = g.S;
    // element q S + off of A, Lin, Lout (off a cell index, q a constant)
    auto pa = [&](int q, int off) -> const float* { return RLB_CHK_PTR(tab.a[q], off, S); };
    auto pl = [&](int q, int off) -> const float* { return RLB_CHK_PTR(tab.l[q], off, S); };
    auto po = [&](int q, int off) -> float* { return RLB_CHK_PTR(tab.o[q], off, S); };
    const int tid = threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const uint32_t scol = (uint32_t)__cvta_generic_to_shared(stage) + 4u * tid;
    auto sval = [&](int slot, int q) -> float { return stage[(slot * 38 + q) * kStageThreads + tid]; };
    auto is_ghost = [&](int x) { return XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1); };
    // one phase (base 19: g, base 0: f) of a cell (pull offsets o) into a slot
    auto issue = [&](int cidx, const PullOffsets& o, int base, int slot) {
        const uint32_t s0 = scol + 4u * (uint32_t)(slot * 38 * kStageThreads);
#pragma unroll
        for (int i = 0; i < 19; ++i) cp_async4(s0 + 4u * (uint32_t)(i * kStageThreads), pa(base + i, cidx + o.src(i)));
#pragma unroll
        for (int i = 0; i < 19; ++i) cp_async4(s0 + 4u * (uint32_t)((19 + i) * kStageThreads), pl(base + i, cidx));
    };

    float tau_acc = 0.0f;
    double bin0 = 0.0, bin1 = 0.0, bin2 = 0.0;
    bool has_b = false;
    // 64-bit loop counter: li + stride cannot wrap for any accepted N
    long long li = (long long)blockIdx.x * blockDim.x + tid;
    int idx = li < g.N ? (int)li : 0;
    int x = 0, y = 0, z = 0;
    PullOffsets o{};
    if (li < g.N) {
        cell_coords(g, idx, x, y, z);
        o = PullOffsets(g, x, y, z);
        if (!is_ghost(x)) issue(idx, o, 19, 0);
    }
    cp_async_commit();
    int sg = 0;
    for (; li < g.N; li += stride) {
        idx = (int)li;
        const int sf = sg == kStageSlots - 1 ? 0 : sg + 1;
        const int sn = sf == kStageSlots - 1 ? 0 : sf + 1;
        const bool ghost = is_ghost(x);
        if (!ghost) issue(idx, o, 0, sf);
        cp_async_commit();
        const long long nl = (long long)idx + stride;  // 64-bit: cannot wrap
        const int nidx = nl < g.N ? (int)nl : 0;
        int xn = 0, yn = 0, zn = 0;
        PullOffsets on{};
        if (nl < g.N) {
            cell_coords(g, nidx, xn, yn, zn);
            on = PullOffsets(g, xn, yn, zn);
        }
        cp_async_wait<1>();  // G_k has landed
        // ---- g phase
        unsigned bounced = 0u;
        bool solid = false;
        const int dup = dup_of<XBC>(x, g.nx);
        float mug[19];
        CellG<float> r;
        if (!ghost) {
            float h[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) h[i] = sval(sg, i);
            solid = is_solid(h[0]);  // the cell's own g_0 (pull offset 0)
            if (!solid) {
                if (isnan(sum19(h))) {
#pragma unroll
                    for (int i = 1; i < 19; ++i) {
                        if (is_solid(h[i])) {
                            bounced |= 1u << i;
                            h[i] = *pa(19 + opp(i), idx);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 19; ++i) mug[i] = sval(sg, 19 + i);
                if (dup) {
#pragma unroll
                    for (int i = 0; i < 19; ++i) mug[i] += *pl(19 + i, idx + dup);
                }
                cell_g(h, mug, c, r);
            }
        }
        if (nl < g.N && !is_ghost(xn)) issue(nidx, on, 19, sn);
        cp_async_commit();
        cp_async_wait<1>();  // F_k has landed
        // ---- f phase, scatter
        if (ghost) {
            ghost_cell<float, XBC>(x, idx, S, A, Lin, Lout, inflow_t, bin0, bin1, bin2, has_b);
        } else if (solid) {  // never updated: identity
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                *po(i, idx) = sval(sf, 19 + i);
                *po(19 + i, idx) = sval(sg, 19 + i);
            }
        } else {
            float h[19], muf[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) h[i] = sval(sf, i);
            if (bounced) {
#pragma unroll
                for (int i = 1; i < 19; ++i)
                    if ((bounced >> i) & 1u) h[i] = *pa(opp(i), idx);
            }
#pragma unroll
            for (int i = 0; i < 19; ++i) muf[i] = sval(sf, 19 + i);
            if (dup) {
#pragma unroll
                for (int i = 0; i < 19; ++i) muf[i] += *pl(i, idx + dup);
            }
            float tf, aS, fbx, fby, fbz;
            cell_f(h, muf, r, c, tf, aS, fbx, fby, fbz);
            tau_acc += (r.tacc + tf) * c.inv_tau2_t;
            float vE, vx, vy, vz;
            recovery_adjoint<float>(r.ae, fbx + r.gbx, fby + r.gby, fbz + r.gbz, r.Et, r.sqt, r.Dt, r.bx, r.by,
                                    r.bz, r.mx, r.my, r.mz, vE, vx, vy, vz);
            scatter_cell(muf, mug, aS, vE, vx, vy, vz, c, [&](int q, int i, float v) {
                if ((bounced >> i) & 1u)
                    *po(q - i + opp(i), idx) = v;
                else
                    *po(q, idx + o.src(i)) = v;
            });
            zero_to_ghost<float, XBC>(x, g.nx, idx, S, Lout);
        }
        sg = sn;
        x = xn;
        o = on;
    }
    cp_async_wait<0>();
    warp_partials<float>((double)tau_acc, bin0, bin1, bin2, has_b, red);
}

// Cooperative form of the staged kernel (the default FP32 adjoint kernel).
// The pulled populations are staged per thread as above; lambda_t+1, read at
// the cell's own index, is copied by the whole block in 16-byte chunks (a
// quarter of the copy instructions), so the block meets at two barriers per
// cell: after the G phase has landed (then every thread is past the f phase
// of the previous cell, and its slots can be refilled) and after the F phase
// has landed.  Because every cell's lambda_t+1 is in the ring, the ghost
// planes and the outflow-copy cells read theirs from it instead of from HBM
// (a lane that waits on HBM would hold the whole block at the next barrier).
template <int XBC>
__global__ void __launch_bounds__(kStageThreads, 3)
    k_adjoint_step_coop(const float* __restrict__ A, const float* __restrict__ Lin, float* __restrict__ Lout,
                          Geom g, Phys ph, AdjConst<float> c, double* red, const float* __restrict__ inflow_t,
                          const __grid_constant__ PlaneTab tab) {
    extern __shared__ float stage[];  // [slot][value 0..37][thread]
    const long long S = g.S;
    // element q S + off of A, Lin, Lout (off a cell index, q a constant)
    auto pa = [&](int q, int off) -> const float* { return RLB_CHK_PTR(tab.a[q], off, S); };
    auto pl = [&](int q, int off) -> const float* { return RLB_CHK_PTR(tab.l[q], off, S); };
    auto po = [&](int q, int off) -> float* { return RLB_CHK_PTR(tab.o[q], off, S); };
    const int tid = threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const uint32_t scol = (uint32_t)__cvta_generic_to_shared(stage) + 4u * tid;
    auto sval = [&](int slot, int q) -> float { return stage[(slot * 38 + q) * kStageThreads + tid]; };
    // another thread's column (lambda_t+1 of every cell of the block is staged)
    auto sval_c = [&](int slot, int q, int col) -> float { return stage[(slot * 38 + q) * kStageThreads + col]; };
    auto is_ghost = [&](int x) { return XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1); };
    // the pulled values of one phase (base 19: g, base 0: f) of this thread's
    // cell (pull offsets o) into its column of a slot
    auto issue = [&](int cidx, const PullOffsets& o, int base, int slot) {
        const uint32_t s0 = scol + 4u * (uint32_t)(slot * 38 * kStageThreads);
#pragma unroll
        for (int i = 0; i < 19; ++i) cp_async4(s0 + 4u * (uint32_t)(i * kStageThreads), pa(base + i, cidx + o.src(i)));
    };
    // lambda_t+1 of one phase for the block's cells [cb, cb + 128): warp w
    // copies planes w, w + 4, ..., lane l the 16 bytes of cells cb + 4l .. + 3
    // (S is a multiple of 4: a chunk lies wholly inside or outside a plane)
    const int wq = tid >> 5, lane4 = 4 * (tid & 31);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage);
    auto issue_lam = [&](long long cb, int base, int slot) {
        const long long cell = cb + lane4;
        if (cell >= S) return;
        const uint32_t s0 = sbase + 4u * (uint32_t)((slot * 38 + 19) * kStageThreads + lane4);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const int q = wq + 4 * m;
            if (q < 19) cp_async16(s0 + 4u * (uint32_t)(q * kStageThreads), RLB_CHK_PTR(Lin, (long long)(base + q) * S + cell, 38ll * S));
        }
    };

    float tau_acc = 0.0f;
    float ga0 = 0.0f, ga1 = 0.0f, ga2 = 0.0f;  // this lane's share of the inflow plane's terms
    double bin0 = 0.0, bin1 = 0.0, bin2 = 0.0;
    bool has_b = false;
    // block-uniform loop over the block's cells [cb, cb + 128) (every thread
    // reaches every barrier); 64-bit: cb + stride cannot wrap
    long long cb = (long long)blockIdx.x * blockDim.x;
    long long li = cb + tid;
    int idx = li < g.N ? (int)li : 0;
    int x = 0, y = 0, z = 0;
    PullOffsets o{};
    if (li < g.N) {
        cell_coords(g, idx, x, y, z);
        o = PullOffsets(g, x, y, z);
        if (!is_ghost(x)) issue(idx, o, 19, 0);
    }
    if (cb < g.N) issue_lam(cb, 19, 0);
    cp_async_commit();
    int sg = 0;
    for (; cb < g.N; cb += stride) {
        li = cb + tid;
        const bool act = li < g.N;
        idx = act ? (int)li : 0;
        const int sf = sg == kStageSlots - 1 ? 0 : sg + 1;
        const int sn = sf == kStageSlots - 1 ? 0 : sf + 1;
        const bool ghost = !act || is_ghost(x);
        // the inflow ghost's own f_0 (solid marker), loaded early
        const float own0 = (XBC == XBC_INFLOW_OUTFLOW && act && x == 0) ? *pa(0, idx) : 0.0f;
        const long long nl = li + stride;
        const int nidx = nl < g.N ? (int)nl : 0;
        int xn = 0, yn = 0, zn = 0;
        PullOffsets on{};
        if (nl < g.N) {
            cell_coords(g, nidx, xn, yn, zn);
            on = PullOffsets(g, xn, yn, zn);
        }
        cp_async_wait<0>();  // G_k has landed (this thread's copies)
        __syncthreads();     // ... and every thread's; all are past f phase k-1
        if (!ghost) issue(idx, o, 0, sf);
        issue_lam(cb, 0, sf);
        cp_async_commit();
        // ---- g phase
        unsigned bounced = 0u;
        bool solid = false;
        const int dup = dup_of<XBC>(x, g.nx);
        const int dcol = tid + dup;  // the copying ghost's column, when in this block
        const bool dup_in = dcol >= 0 && dcol < kStageThreads;
        float mug[19];
        CellG<float> r;
        if (!ghost) {
            float h[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) h[i] = sval(sg, i);
            solid = is_solid(h[0]);  // the cell's own g_0 (pull offset 0)
            if (!solid) {
                if (isnan(sum19(h))) {
#pragma unroll
                    for (int i = 1; i < 19; ++i) {
                        if (is_solid(h[i])) {
                            bounced |= 1u << i;
                            h[i] = *pa(19 + opp(i), idx);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 19; ++i) mug[i] = sval(sg, 19 + i);
                if (dup) {
                    if (dup_in) {
#pragma unroll
                        for (int i = 0; i < 19; ++i) mug[i] += sval_c(sg, 19 + i, dcol);
                    } else {
#pragma unroll
                        for (int i = 0; i < 19; ++i) mug[i] += *pl(19 + i, idx + dup);
                    }
                }
                cell_g(h, mug, c, r);
            }
        }
        if (nl < g.N && !is_ghost(xn)) issue(nidx, on, 19, sn);
        if (cb + stride < g.N) issue_lam(cb + stride, 19, sn);
        cp_async_commit();
        cp_async_wait<1>();  // F_k has landed (this thread's copies)
        __syncthreads();     // ... and every thread's
        // ---- f phase, scatter
        if (!act) {
        } else if (ghost) {
            // ghost_cell: its zeros and the inflow plane's dL/dbeta_in terms
            // are written below by the whole warp
        } else if (solid) {  // never updated: identity
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                *po(i, idx) = sval(sf, 19 + i);
                *po(19 + i, idx) = sval(sg, 19 + i);
            }
        } else {
            float h[19], muf[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) h[i] = sval(sf, i);
            if (bounced) {
#pragma unroll
                for (int i = 1; i < 19; ++i)
                    if ((bounced >> i) & 1u) h[i] = *pa(opp(i), idx);
            }
#pragma unroll
            for (int i = 0; i < 19; ++i) muf[i] = sval(sf, 19 + i);
            if (dup) {
                if (dup_in) {
#pragma unroll
                    for (int i = 0; i < 19; ++i) muf[i] += sval_c(sf, 19 + i, dcol);
                } else {
#pragma unroll
                    for (int i = 0; i < 19; ++i) muf[i] += *pl(i, idx + dup);
                }
            }
            float tf, aS, fbx, fby, fbz;
            cell_f(h, muf, r, c, tf, aS, fbx, fby, fbz);
            tau_acc += (r.tacc + tf) * c.inv_tau2_t;
            float vE, vx, vy, vz;
            recovery_adjoint<float>(r.ae, fbx + r.gbx, fby + r.gby, fbz + r.gbz, r.Et, r.sqt, r.Dt, r.bx, r.by,
                                    r.bz, r.mx, r.my, r.mz, vE, vx, vy, vz);
            scatter_cell(muf, mug, aS, vE, vx, vy, vz, c, [&](int q, int i, float v) {
                if ((bounced >> i) & 1u)
                    *po(q - i + opp(i), idx) = v;
                else
                    *po(q, idx + o.src(i)) = v;
            });
        }
        if constexpr (XBC != XBC_PERIODIC) {
            // The zeros next to the ghost planes, spread over the warp (one
            // lane storing 28 or 10 of them would hold its block at the next
            // barrier): for each lane that is a ghost cell, lane q zeroes
            // population q of it where nobody reads it (velocity not pointing
            // inward); for each fluid cell at x = 1 or nx - 2, lane q zeroes
            // population q of it where the ghost would have pulled it.
            const int lane = tid & 31;
            const int vq = lane < 19 ? vel_x(lane) : 0;
            unsigned m = __ballot_sync(0xffffffffu, act && (ghost || (!solid && (x == 1 || x == g.nx - 2))));
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const int cx = __shfl_sync(0xffffffffu, x, src);
                const int cidx = __shfl_sync(0xffffffffu, idx, src);
                bool z;
                if (cx == 0 || cx == g.nx - 1)
                    z = vq != (cx == 0 ? 1 : -1);  // a ghost cell
                else  // next to a ghost (both, when nx = 3)
                    z = (cx == 1 && vq == -1) || (cx == g.nx - 2 && vq == 1);
                if (lane < 19 && z) {
                    Lout[RLB_CHK((long long)lane * S + cidx, 38ll * S)] = 0.0f;
                    Lout[RLB_CHK((long long)(19 + lane) * S + cidx, 38ll * S)] = 0.0f;
                }
            }
        }
        if constexpr (XBC == XBC_INFLOW_OUTFLOW) {
            // dL/dbeta_in = lambda_t+1 . d eq_in / d beta_in at each fluid
            // inflow ghost: its 38 terms spread over the warp (lane l takes
            // q = l and l + 32) from the ghost's column of the ring, each lane
            // adding into its own partial sums (summed over the warp at the end)
            unsigned m = __ballot_sync(0xffffffffu, act && x == 0 && !is_solid(own0));
            const int lane = tid & 31;
            while (m) {
                const int col = (tid & ~31) + __ffs(m) - 1;
                m &= m - 1;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int q = lane + 32 * r;
                    if (q < 38) {
                        const float l = q < 19 ? sval_c(sf, 19 + q, col) : sval_c(sg, q, col);
                        ga0 = fmaf(l, inflow_t[3 * q + 0], ga0);
                        ga1 = fmaf(l, inflow_t[3 * q + 1], ga1);
                        ga2 = fmaf(l, inflow_t[3 * q + 2], ga2);
                    }
                }
                has_b = true;
            }
        }
        sg = sn;
        x = xn;
        o = on;
    }
    cp_async_wait<0>();
    bin0 += (double)ga0;
    bin1 += (double)ga1;
    bin2 += (double)ga2;
    warp_partials<float>((double)tau_acc, bin0, bin1, bin2, has_b, red);
}

// d eq_j(n_in, eps_in, beta_in) / d beta_in,a for the 38 populations (one
// thread per population, FP64): the adjoint of the inflow plane.  The table
// is written twice: binary64, then rounded to binary32 after it.
__global__ void k_inflow_derivs(Phys ph, double* out) {
    const int j = threadIdx.x;
    if (j >= 38) return;
    double lf[19], lg[19];
    for (int i = 0; i < 19; ++i) lf[i] = lg[i] = 0.0;
    if (j < 19) lf[j] = 1.0; else lg[j - 19] = 1.0;
    double an, ae, ax, ay, az;
    eq_fields_adjoint(lf, lg, ph.n_in, ph.eps_in, ph.beta_in[0], ph.beta_in[1], ph.beta_in[2], ph, an, ae, ax, ay, az);
    out[3 * j + 0] = ax;
    out[3 * j + 1] = ay;
    out[3 * j + 2] = az;
    float* outf = reinterpret_cast<float*>(out + kInflowTable);
    outf[3 * j + 0] = (float)ax;
    outf[3 * j + 1] = (float)ay;
    outf[3 * j + 2] = (float)az;
}

// The inflow table in the kernels' precision.
template <typename T>
const T* inflow_table(const double* inflow_d) {
    if constexpr (sizeof(T) == 8)
        return inflow_d;
    else
        return reinterpret_cast<const float*>(inflow_d + kInflowTable);
}

cudaError_t launch_inflow_derivs(const Phys& ph, double* out, cudaStream_t st) {
    set_last_launch_count(1);
    k_inflow_derivs<<<1, 64, 0, st>>>(ph, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint of the macroscopic output: n = S sqrt(1 - b2), eps, beta.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_adjoint_macro(const T* __restrict__ A, const double* __restrict__ dn,
                                                       const double* __restrict__ deps, const double* __restrict__ dbeta,
                                                       T* __restrict__ lam, Geom g, Phys ph) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long S = g.S;
    if (is_solid(A[RLB_CHK(idx, 38ll * S)])) {
        for (int q = 0; q < 38; ++q) lam[RLB_CHK(q * S + idx, 38ll * S)] = (T)0;
        return;
    }
    double h[38];
    for (int q = 0; q < 38; ++q) h[q] = (double)A[RLB_CHK(q * S + idx, 38ll * S)];
    double sf = 0, E = 0, Mx = 0, My = 0, Mz = 0;
    for (int i = 0; i < 19; ++i) {
        sf += h[i];
        E += h[19 + i];
        Mx += h[19 + i] * vel_x(i);
        My += h[19 + i] * vel_y(i);
        Mz += h[19 + i] * vel_z(i);
    }
    if (sizeof(T) == 4) {
        sf += ph.n_ref;
        E += ph.eps_ref;
    }
    Mx *= ph.c_l;
    My *= ph.c_l;
    Mz *= ph.c_l;
    const double sq = sqrt(4.0 * E * E - 3.0 * (Mx * Mx + My * My + Mz * Mz));
    const double eps = sq - E;
    const double D = 3.0 * E + eps;
    const double bx = 3.0 * Mx / D, by = 3.0 * My / D, bz = 3.0 * Mz / D;
    const double b2 = bx * bx + by * by + bz * bz;
    const double rt = sqrt(1.0 - b2);
    const double gdn = dn[idx];
    const double aS = gdn * rt;
    const double c = -gdn * sf / rt;
    const double abx = dbeta[idx] + c * bx;
    const double aby = dbeta[g.N + idx] + c * by;
    const double abz = dbeta[2 * (long long)g.N + idx] + c * bz;
    double vE, vx, vy, vz;
    recovery_adjoint<double>(deps[idx], abx, aby, abz, E, sq, D, bx, by, bz, Mx, My, Mz, vE, vx, vy, vz);
    for (int i = 0; i < 19; ++i) {
        lam[RLB_CHK(i * S + idx, 38ll * S)] = (T)aS;
        lam[RLB_CHK((19 + i) * S + idx, 38ll * S)] = (T)(vE + ph.c_l * (vel_x(i) * vx + vel_y(i) * vy + vel_z(i) * vz));
    }
}

// ---------------------------------------------------------------------------
// Adjoint of the initialisation A_0 = eq(n0, eps0, beta0).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_adjoint_fields(const double* __restrict__ n0, const double* __restrict__ e0,
                                                        const double* __restrict__ b0, const T* __restrict__ A0,
                                                        const T* __restrict__ lam, double* __restrict__ dn,
                                                        double* __restrict__ de, double* __restrict__ db, Geom g,
                                                        Phys ph, double* red) {
    const long long S = g.S;
    double bin0 = 0.0, bin1 = 0.0, bin2 = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx = g.N) {
        const int x = idx % g.nx;
        double lf[19], lg[19];
        double an = 0, ae = 0, ax = 0, ay = 0, az = 0;
        const bool solid = is_solid(A0[RLB_CHK(idx, 38ll * S)]);
        if (!solid) {
            for (int i = 0; i < 19; ++i) {
                lf[i] = (double)lam[RLB_CHK(i * S + idx, 38ll * S)];
                lg[i] = (double)lam[RLB_CHK((19 + i) * S + idx, 38ll * S)];
            }
            if (g.xbc == XBC_INFLOW_OUTFLOW && x == 0) {
                eq_fields_adjoint(lf, lg, ph.n_in, ph.eps_in, ph.beta_in[0], ph.beta_in[1], ph.beta_in[2], ph, an,
                                  ae, ax, ay, az);
                bin0 += ax;
                bin1 += ay;
                bin2 += az;
                an = ae = ax = ay = az = 0;
            } else {
                eq_fields_adjoint(lf, lg, n0[idx], e0[idx], b0[idx], b0[g.N + idx], b0[2 * (long long)g.N + idx], ph,
                                  an, ae, ax, ay, az);
            }
        }
        dn[idx] = an;
        de[idx] = ae;
        db[idx] = ax;
        db[g.N + idx] = ay;
        db[2 * (long long)g.N + idx] = az;
    }
    block_reduce4(0.0, bin0, bin1, bin2, red);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline int adj_blocks(int N) { return (N + 127) / 128; }

cudaError_t launch_adjoint_macro(int prec, const Geom& g, const Phys& ph, const void* A, const double* dn,
                                 const double* deps, const double* dbeta, void* lam, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + 127) / 128);
    set_last_launch_count(1);
    if (prec == 0)
        k_adjoint_macro<double><<<nb, 128, 0, st>>>((const double*)A, dn, deps, dbeta, (double*)lam, g, ph);
    else
        k_adjoint_macro<float><<<nb, 128, 0, st>>>((const float*)A, dn, deps, dbeta, (float*)lam, g, ph);
    return cudaGetLastError();
}

namespace {
// The calling thread's current context (the device's primary context under
// the runtime API), through the driver entry point the runtime hands out, so
// that the library needs no link against the driver library.
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(f);
        looked = true;
    }
    CUcontext c = nullptr;
    if (fn) fn(&c);
    return c;
}

// The dynamic shared memory opt-in of a staged kernel, once per context and
// kernel (the attribute belongs to the kernel in a context: a new context
// after a reset needs it again; setting it on every launch costs a host-side
// call that held back the launch queue of short steps).
std::mutex g_optin_mu;
struct OptIn {
    CUcontext ctx;
    const void* kern;
};
OptIn g_optin[64];
int g_optin_n = 0;

cudaError_t smem_opt_in(const void* kern, int bytes) {
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lock(g_optin_mu);
    for (int i = 0; i < g_optin_n; ++i)
        if (g_optin[i].ctx == ctx && g_optin[i].kern == kern) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && g_optin_n < 64) g_optin[g_optin_n++] = {ctx, kern};
    return e;
}
}  // namespace

template <typename T>
static int adjoint_step_t(const Geom& g, const Phys& ph, const T* A, const T* Li, T* Lo, double* red, int nb,
                          const double* inflow_d, cudaStream_t st) {
    const AdjConst<T> c = make_adj_const<T>(ph);
    const T* inflow_t = inflow_table<T>(inflow_d);
    auto persistent_grid = [&](int minb) {
        static int nsm = 0;
        if (nsm == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        }
        const int pg = nsm * minb;
        return pg < nb ? pg : nb;
    };
    // each launcher returns the number of warps whose partial sums it wrote
    auto go = [&](auto kern, bool pipe, int minb) {
        const int grid = pipe ? persistent_grid(minb) : nb;
        kern<<<grid, 128, 0, st>>>(A, Li, Lo, g, ph, c, red, inflow_t);
        return grid * 4;
    };
    int warps = 0;
    if constexpr (sizeof(T) == 4) {
        if (g.adj_pipe == 2) {
            const int coop = g.adj_coop;
            PlaneTab tab;
            for (int q = 0; q < 38; ++q) {
                tab.a[q] = (const float*)A + (long long)q * g.S;
                tab.l[q] = (const float*)Li + (long long)q * g.S;
                tab.o[q] = (float*)Lo + (long long)q * g.S;
            }
            auto staged = [&](auto kern) {
                smem_opt_in((const void*)kern, (int)kStageSmemBytes);  // a failure shows at the launch
                const int grid = persistent_grid(3);
                kern<<<grid, kStageThreads, kStageSmemBytes, st>>>(A, Li, Lo, g, ph, c, red, inflow_t, tab);
                return grid * (kStageThreads / 32);
            };
            // 16-byte copies of lambda_t+1: the buffer must be 16-byte aligned
            if (coop && ((uintptr_t)Li & 15u) == 0) {
                switch (g.xbc) {
                    case XBC_PERIODIC: return staged(k_adjoint_step_coop<XBC_PERIODIC>);
                    case XBC_INFLOW_OUTFLOW: return staged(k_adjoint_step_coop<XBC_INFLOW_OUTFLOW>);
                    default: return staged(k_adjoint_step_coop<XBC_OUTFLOW_BOTH>);
                }
            }
            switch (g.xbc) {
                case XBC_PERIODIC: return staged(k_adjoint_step_staged<XBC_PERIODIC>);
                case XBC_INFLOW_OUTFLOW: return staged(k_adjoint_step_staged<XBC_INFLOW_OUTFLOW>);
                default: return staged(k_adjoint_step_staged<XBC_OUTFLOW_BOTH>);
            }
        }
    }
    if constexpr (sizeof(T) == 8) {
        // persistent (the instantiation the allocation-free step runs too)
        switch (g.xbc) {
            case XBC_PERIODIC: warps = go(k_adjoint_step<T, XBC_PERIODIC, 2, true>, true, 2); break;
            case XBC_INFLOW_OUTFLOW: warps = go(k_adjoint_step<T, XBC_INFLOW_OUTFLOW, 2, true>, true, 2); break;
            default: warps = go(k_adjoint_step<T, XBC_OUTFLOW_BOTH, 2, true>, true, 2); break;
        }
    } else if (g.adj_pipe) {
        switch (g.xbc) {
            case XBC_PERIODIC: warps = go(k_adjoint_step<T, XBC_PERIODIC, 4, true>, true, 4); break;
            case XBC_INFLOW_OUTFLOW: warps = go(k_adjoint_step<T, XBC_INFLOW_OUTFLOW, 4, true>, true, 4); break;
            default: warps = go(k_adjoint_step<T, XBC_OUTFLOW_BOTH, 4, true>, true, 4); break;
        }
    } else {
        switch (g.xbc) {
            case XBC_PERIODIC: warps = go(k_adjoint_step<T, XBC_PERIODIC, 4, false>, false, 4); break;
            case XBC_INFLOW_OUTFLOW: warps = go(k_adjoint_step<T, XBC_INFLOW_OUTFLOW, 4, false>, false, 4); break;
            default: warps = go(k_adjoint_step<T, XBC_OUTFLOW_BOTH, 4, false>, false, 4); break;
        }
    }
    return warps;
}

cudaError_t launch_adjoint_step(int prec, const Geom& g, const Phys& ph, const void* A, const void* lam_in,
                                void* lam_out, double* red, const double* inflow_d, double* dtau, double* dbeta_in,
                                cudaStream_t st) {
    const int nb = adj_blocks(g.N);
    set_last_launch_count(2);
    int warps;
    if (prec == 0)
        warps = adjoint_step_t<double>(g, ph, (const double*)A, (const double*)lam_in, (double*)lam_out, red, nb,
                                       inflow_d, st);
    else
        warps = adjoint_step_t<float>(g, ph, (const float*)A, (const float*)lam_in, (float*)lam_out, red, nb,
                                      inflow_d, st);
    k_finalize<<<1, 1024, 0, st>>>(red, warps, dtau, dbeta_in);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fields(int prec, const Geom& g, const Phys& ph, const double* n0, const double* eps0,
                                  const double* beta0, const void* A0, const void* lam0, double* dn0, double* deps0,
                                  double* dbeta0, double* red, double* dbeta_in, cudaStream_t st) {
    const int nb = adj_blocks(g.N);
    set_last_launch_count(2);
    if (prec == 0)
        k_adjoint_fields<double><<<nb, 128, 0, st>>>(n0, eps0, beta0, (const double*)A0, (const double*)lam0, dn0,
                                                     deps0, dbeta0, g, ph, red);
    else
        k_adjoint_fields<float><<<nb, 128, 0, st>>>(n0, eps0, beta0, (const float*)A0, (const float*)lam0, dn0, deps0,
                                                    dbeta0, g, ph, red);
    k_finalize<<<1, 1024, 0, st>>>(red, nb, nullptr, dbeta_in);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free adjoint step.  Same kernels as launch_adjoint_step, always
// as the persistent grid-stride launch (grid = SMs x resident blocks, capped
// at the block count), with the per-warp partial sums in a fixed static
// device array instead of the context workspace.  Every launch writes all
// grid*16 slots it reads, so the array needs no zeroing; two launches that
// overlap in time on one device (other streams, other contexts) share it and
// race.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_adj_scratch[kAdjScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchSetup {
    double* ptr;    // device address of g_adj_scratch in the context below
    int nsm;        // SM count of the device
    CUcontext ctx;  // the context the set-up was made in
};
ScratchSetup g_scratch[kMaxDevices];

// Set-up, with the device current: the device address of g_adj_scratch, the
// SM count, and every kernel this entry point launches loaded onto the
// device (cudaFuncGetAttributes loads a kernel that lazy module loading has
// not loaded yet), so that no later call loads code, which can allocate.
// Redone when the device's context is not the one it was made in (after
// cudaDeviceReset the old address is stale).
cudaError_t scratch_for_device(int dev, double** ptr, int* nsm) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSetup& s = g_scratch[dev];
    if (!s.ptr || s.ctx != ctx) {
        s.ptr = nullptr;
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_adj_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const void* kernels[] = {
            (const void*)k_adjoint_step<double, XBC_PERIODIC, 2, true>,
            (const void*)k_adjoint_step<double, XBC_INFLOW_OUTFLOW, 2, true>,
            (const void*)k_adjoint_step<double, XBC_OUTFLOW_BOTH, 2, true>,
            (const void*)k_adjoint_step<float, XBC_PERIODIC, 4, true>,
            (const void*)k_adjoint_step<float, XBC_INFLOW_OUTFLOW, 4, true>,
            (const void*)k_adjoint_step<float, XBC_OUTFLOW_BOTH, 4, true>,
            (const void*)k_finalize,
        };
        for (const void* k : kernels) {
            cudaFuncAttributes attr;
            e = cudaFuncGetAttributes(&attr, k);
            if (e != cudaSuccess) return e;
        }
        // the FP32 staged kernels (block-copy and per-thread forms): loaded,
        // and their shared memory opted in
        const void* staged[] = {
            (const void*)k_adjoint_step_coop<XBC_PERIODIC>,   (const void*)k_adjoint_step_coop<XBC_INFLOW_OUTFLOW>,
            (const void*)k_adjoint_step_coop<XBC_OUTFLOW_BOTH>, (const void*)k_adjoint_step_staged<XBC_PERIODIC>,
            (const void*)k_adjoint_step_staged<XBC_INFLOW_OUTFLOW>, (const void*)k_adjoint_step_staged<XBC_OUTFLOW_BOTH>,
        };
        for (const void* k : staged) {
            cudaFuncAttributes attr;
            e = cudaFuncGetAttributes(&attr, k);
            if (e == cudaSuccess) e = smem_opt_in(k, (int)kStageSmemBytes);
            if (e != cudaSuccess) return e;
        }
        s.nsm = n;
        s.ctx = ctx;
        s.ptr = p;
    }
    *ptr = s.ptr;
    *nsm = s.nsm;
    return cudaSuccess;
}

template <typename T, int MINB>
int adjoint_step_noalloc_t(const Geom& g, const Phys& ph, const T* A, const T* Li, T* Lo, double* red, int grid,
                           const double* inflow_d, cudaStream_t st) {
    const AdjConst<T> c = make_adj_const<T>(ph);
    const T* inflow_t = inflow_table<T>(inflow_d);
    switch (g.xbc) {
        case XBC_PERIODIC:
            k_adjoint_step<T, XBC_PERIODIC, MINB, true><<<grid, 128, 0, st>>>(A, Li, Lo, g, ph, c, red, inflow_t);
            break;
        case XBC_INFLOW_OUTFLOW:
            k_adjoint_step<T, XBC_INFLOW_OUTFLOW, MINB, true><<<grid, 128, 0, st>>>(A, Li, Lo, g, ph, c, red,
                                                                                   inflow_t);
            break;
        default:
            k_adjoint_step<T, XBC_OUTFLOW_BOTH, MINB, true><<<grid, 128, 0, st>>>(A, Li, Lo, g, ph, c, red,
                                                                                 inflow_t);
            break;
    }
    return grid;
}
}  // namespace

cudaError_t launch_adjoint_step_noalloc(int prec, const Geom& g, const Phys& ph, const void* A, const void* lam_in,
                                        void* lam_out, const double* inflow_d, double* dtau, double* dbeta_in,
                                        cudaStream_t st, long long* need_doubles) {
    set_last_launch_count(0);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    double* red = nullptr;
    int nsm = 0;
    e = scratch_for_device(dev, &red, &nsm);
    if (e != cudaSuccess) return e;
    const int nb = adj_blocks(g.N);
    if (prec != 0 && g.adj_pipe == 2) {
        // FP32 with the default kernel choice: the staged kernel that
        // rlb_adjoint_step runs (persistent, SMs x 3 blocks of 128)
        const int grid3 = nsm * 3 < nb ? nsm * 3 : nb;
        const long long need = 16ll * grid3;
        if (need_doubles) *need_doubles = need;
        if (need > kAdjScratchDoubles) return cudaErrorInvalidValue;
        set_last_launch_count(2);
        const int warps = adjoint_step_t<float>(g, ph, (const float*)A, (const float*)lam_in, (float*)lam_out, red, nb,
                                                inflow_d, st);
        k_finalize<<<1, 1024, 0, st>>>(red, warps, dtau, dbeta_in);
        return cudaGetLastError();
    }
    const int minb = prec == 0 ? 2 : 4;
    const int grid = nsm * minb < nb ? nsm * minb : nb;
    const long long need = 16ll * grid;  // 4 warps x 4 partial sums per block
    if (need_doubles) *need_doubles = need;
    if (need > kAdjScratchDoubles) return cudaErrorInvalidValue;
    set_last_launch_count(2);
    if (prec == 0)
        adjoint_step_noalloc_t<double, 2>(g, ph, (const double*)A, (const double*)lam_in, (double*)lam_out, red, grid,
                                          inflow_d, st);
    else
        adjoint_step_noalloc_t<float, 4>(g, ph, (const float*)A, (const float*)lam_in, (float*)lam_out, red, grid,
                                         inflow_d, st);
    k_finalize<<<1, 1024, 0, st>>>(red, grid * 4, dtau, dbeta_in);
    return cudaGetLastError();
}

// Bounds-check count of this translation unit (0 in the release build).
RLB_OOB_TAKE_FN(oob_take_adjoint)

}  // namespace rlb

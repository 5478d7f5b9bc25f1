// rlb_f64df.cu -- the FP64 step (binary64 storage) with its arithmetic on the
// FP32 pipe in compensated binary32 pairs (selected with RLB_F64_ARITH=df).
//
// GB300 issues FP64 instructions at about 1/70 of the FP32 rate, and the
// all-FP64 step needs about 210 of them per update (57 for the moment sums
// alone), which caps it near a quarter of its HBM roofline.  This variant
// keeps the binary64 states, the binary64 recovery root and the binary64
// equilibrium coefficients, and moves the rest to pairs of binary32 values
// (rlb_dfloat.cuh: the error-free transformations of Dekker and Knuth):
//   - every loaded population is split into a pair on the integer pipe
//     (df_split: 48 of its 53 significant bits);
//   - the moments are compensated sums of the pairs;
//   - the equilibria are formed as pairs from the binary64 coefficients
//     (Eqs. equil1s, equil2as, equil2bs; the antisymmetric part of g^eq as
//     3 w_p (e_p . M)/c_l from the momentum sums, which equals
//     w_p eps gamma^2 4 q_p/c_l for the recovered fields);
//   - the relaxed value h + omega (eq - h) is a pair, recombined into
//     binary64 with one FP64 addition.
// About 100 FP64 instructions per update remain.  Results agree with the
// all-FP64 step to about 2^-48 per update, not bit for bit; the pairs need
// populations within the binary32 exponent range (|h| from about 2^-74 to
// 2^127; the tests' and benchmarks' workloads lie far inside it).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rlb_collide.cuh"
#include "rlb_device.cuh"
#include "rlb_dfloat.cuh"

namespace rlb {

namespace {

// binary64 constant as a pair (host and device)
struct DfConst {
    float h, l;
};
inline DfConst df_const(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

struct F64dfConst {
    dfl omega;  // 1/tau
};

// one phase: the 19 populations of set 'base' (0: f, 19: g) pulled into
// pairs, with link bounce-back
template <bool SOLID>
__device__ __forceinline__ bool gather_split(const double* __restrict__ A, long long S, int idx, const PullOffsets& o,
                                             int base, dfl* v) {
    double h[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) h[i] = __ldg(RLB_CHK_PTR(A, (base + i) * S + idx + o.src(i), 38ll * S));
    if (SOLID) {
#pragma unroll
        for (int i = 1; i < 19; ++i)
            if (is_solid(h[i])) h[i] = __ldg(RLB_CHK_PTR(A, (base + opp(i)) * S + idx, 38ll * S));
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) v[i] = df_split(h[i]);
    return true;
}

// h + omega (eq - h) as a pair, recombined into binary64
__device__ __forceinline__ double relax(dfl h, dfl eq, dfl om) {
    const dfl neq = df_add(eq, df_neg(h));
    return df_dbl(df_add(h, df_mul(om, neq)));
}

}  // namespace

template <int XBC, bool SOLID>
__global__ void __launch_bounds__(128) k_step_f64_df(const double* __restrict__ A, double* __restrict__ B, Geom g,
                                                     Phys ph, F64dfConst k, Counters cnt, int count,
                                                     long long step_index) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int x, y, z;
    cell_coords(g, idx, x, y, z);
    if (g.zhalo && (z == 0 || z == g.nz - 1)) return;  // z halo planes: filled by the exchange
    const long long S = g.S;
    if (XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1)) {
        if (XBC == XBC_INFLOW_OUTFLOW && x == 0) {
#pragma unroll
            for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = __ldg(RLB_CHK_PTR(A, q * S + idx, 38ll * S));
        }
        return;
    }
    if (SOLID && is_solid(__ldg(RLB_CHK_PTR(A, idx, 38ll * S)))) {  // the cell itself is solid: keep the marker
        const double m = solid_marker_d();
#pragma unroll
        for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = m;
        return;
    }
    const PullOffsets o(g, x, y, z);
    const int dup = (XBC != XBC_PERIODIC && x == g.nx - 2) ? 1 : ((XBC == XBC_OUTFLOW_BOTH && x == 1) ? -1 : 0);
    auto put = [&](int q, double v) {
        B[RLB_CHK(q * S + idx, 38ll * S)] = v;
        if (dup) B[RLB_CHK(q * S + idx + dup, 38ll * S)] = v;
    };
    // ---- g phase: energy-momentum populations (they alone fix eps, beta) ----
    dfl G[19];
    gather_split<SOLID>(A, S, idx, o, 19, G);
    CSum es(G[0].h);
    es.c = G[0].l;
    dfl dg[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        es.add(G[2 * p + 1]);
        es.add(G[2 * p + 2]);
        const dfl t = two_sum(G[2 * p + 1].h, -G[2 * p + 2].h);
        dg[p] = fast_two_sum(t.h, __fadd_rn(t.l, __fsub_rn(G[2 * p + 1].l, G[2 * p + 2].l)));
    }
    CSum sx(dg[0].h), sy(dg[1].h), sz(dg[2].h);
    sx.c = dg[0].l, sy.c = dg[1].l, sz.c = dg[2].l;
    sx.add(dg[3]), sx.add(dg[4]), sx.add(dg[5]), sx.add(dg[6]);
    sy.add(dg[3]), sy.add(df_neg(dg[4])), sy.add(dg[7]), sy.add(dg[8]);
    sz.add(dg[5]), sz.add(df_neg(dg[6])), sz.add(dg[7]), sz.add(df_neg(dg[8]));
    const dfl Dx = sx.result(), Dy = sy.result(), Dz = sz.result();  // M / c_l
    // recovery in binary64: eps = -E + sqrt(4E^2 - 3M^2), beta = 3M/(3E + eps)
    const double E = df_dbl(es.result());
    const double mx = ph.c_l * df_dbl(Dx), my = ph.c_l * df_dbl(Dy), mz = ph.c_l * df_dbl(Dz);
    const double m2 = fma(mx, mx, fma(my, my, mz * mz));
    const double disc = fma(4.0 * E, E, -3.0 * m2);
    double ys, hs;
    rsqrt_seed(disc, ys, hs);
    double sq = disc * ys;
    sq = fma(fma(-sq, sq, disc), hs, sq);
    sq = fma(fma(-sq, sq, disc), hs, sq);
    const double eps = sq - E;
    const double D = fma(3.0, E, eps);
    double rD = rcp_seed(D);
    rD = fma(rD, fma(-D, rD, 1.0), rD);
    rD = fma(rD, fma(-D, rD, 1.0), rD);
    const double r3 = 3.0 * rD;
    const double bx = mx * r3, by = my * r3, bz = mz * r3;
    const double b2 = fma(bx, bx, fma(by, by, bz * bz));
    const double omb2 = 1.0 - b2;
    double gam2 = rcp_seed(omb2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    const double eg = eps * gam2;
    const dfl Bx = df_of(bx), By = df_of(by), Bz = df_of(bz);
    const dfl qv[9] = {Bx, By, Bz, df_add(Bx, By), df_add(Bx, df_neg(By)), df_add(Bx, Bz), df_add(Bx, df_neg(Bz)),
                       df_add(By, Bz), df_add(By, df_neg(Bz))};
    {
        // g^eq_i = w_i [k1 + k2 q_i^2] +- 3 w_i (e_i . M)/c_l,
        //   k1 = (eps - 2 eg b2)/c_l^2, k2 = 6 eg / c_l^2
        const double k1 = (eps - 2.0 * eg * b2) * ph.inv_cl2, k2 = 6.0 * eg * ph.inv_cl2;
        const dfl K1[2] = {df_of(k1 * (1.0 / 18.0)), df_of(k1 * (1.0 / 36.0))};
        const dfl K2[2] = {df_of(k2 * (1.0 / 18.0)), df_of(k2 * (1.0 / 36.0))};
        const dfl A3[2] = {{(float)(1.0 / 6.0), (float)(1.0 / 6.0 - (double)(float)(1.0 / 6.0))},
                           {(float)(1.0 / 12.0), (float)(1.0 / 12.0 - (double)(float)(1.0 / 12.0))}};
        const dfl ev[9] = {Dx, Dy, Dz, df_add(Dx, Dy), df_add(Dx, df_neg(Dy)), df_add(Dx, Dz),
                           df_add(Dx, df_neg(Dz)), df_add(Dy, Dz), df_add(Dy, df_neg(Dz))};
        // g_0^eq = w_0 [4 eps gamma^2 - eps (2 + c_l^2)/c_l^2 - 2 eps gamma^2 b2/c_l^2]   (Eq. equil2bs)
        const double g0 = kW0 * (4.0 * eg - eps * (2.0 * ph.inv_cl2 + 1.0) - 2.0 * eg * b2 * ph.inv_cl2);
        put(19, relax(G[0], df_of(g0), k.omega));
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const int cl = p < 3 ? 0 : 1;
            const dfl gsym = df_add(df_mul(K2[cl], df_mul(qv[p], qv[p])), K1[cl]);
            const dfl gasy = df_mul(A3[cl], ev[p]);
            put(20 + 2 * p, relax(G[2 * p + 1], df_add(gsym, gasy), k.omega));
            put(21 + 2 * p, relax(G[2 * p + 2], df_add(gsym, df_neg(gasy)), k.omega));
        }
    }
    // ---- f phase: number populations ----
    dfl F[19];
    gather_split<SOLID>(A, S, idx, o, 0, F);
    CSum ss(F[0].h);
    ss.c = F[0].l;
#pragma unroll
    for (int i = 1; i < 19; ++i) ss.add(F[i]);
    const double sf = df_dbl(ss.result());
    // f^eq_i = w_i S (1 +- 3 q_i / c_l)   (Eq. equil1s with n gamma = S)
    const dfl FS[2] = {df_of(sf * (1.0 / 18.0)), df_of(sf * (1.0 / 36.0))};
    const double fa = 3.0 * sf * ph.inv_cl;
    const dfl FA[2] = {df_of(fa * (1.0 / 18.0)), df_of(fa * (1.0 / 36.0))};
    put(0, relax(F[0], df_of(kW0 * sf), k.omega));
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int cl = p < 3 ? 0 : 1;
        const dfl fasy = df_mul(FA[cl], qv[p]);
        put(2 * p + 1, relax(F[2 * p + 1], df_add(FS[cl], fasy), k.omega));
        put(2 * p + 2, relax(F[2 * p + 2], df_add(FS[cl], df_neg(fasy)), k.omega));
    }
    const bool unphys = !(pos_finite(sf) && pos_finite(E) && nonneg_finite(disc) && pos_finite(eps) && below_one(b2));
    const bool nonpos = nonpositive_eq(d2f(bx), d2f(by), d2f(bz), (float)ph.c_l);
    if (count) count_flags(cnt, unphys, nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
}

cudaError_t launch_step_f64_df(const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt, bool count,
                               long long step_index, cudaStream_t st, int threads) {
    F64dfConst k;
    const DfConst om = df_const(ph.omega);
    k.omega = {om.h, om.l};
    const unsigned nb = (unsigned)((g.N + threads - 1) / threads);
    const int cs = count ? 1 : 0;
    const double* a = (const double*)A;
    double* b = (double*)B;
    switch (g.xbc) {
        case XBC_PERIODIC:
            k_step_f64_df<XBC_PERIODIC, true><<<nb, threads, 0, st>>>(a, b, g, ph, k, cnt, cs, step_index);
            break;
        case XBC_INFLOW_OUTFLOW:
            k_step_f64_df<XBC_INFLOW_OUTFLOW, true><<<nb, threads, 0, st>>>(a, b, g, ph, k, cnt, cs, step_index);
            break;
        default: k_step_f64_df<XBC_OUTFLOW_BOTH, true><<<nb, threads, 0, st>>>(a, b, g, ph, k, cnt, cs, step_index); break;
    }
    return cudaGetLastError();
}

}  // namespace rlb

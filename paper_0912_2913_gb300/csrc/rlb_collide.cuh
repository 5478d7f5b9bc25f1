// rlb_collide.cuh -- the per-cell FP32 deviation collision shared by the
// plain and the TMA-staged step kernels (same arithmetic, bit for bit).
//
// Populations are stored as d_i = p_i - p_i^ref with p^ref the rest
// equilibrium of (n_ref, eps_ref): f_i^ref = w_i n_ref, g_i^ref = w_i eps_ref
// / c_l^2 (i > 0), g_0^ref = w_0 eps_ref (3 - 2/c_l^2).  Streaming and BGK are
// linear and the reference is uniform and symmetric, so a step maps
// deviations to deviations.  The moments are the reference moments
// (n_ref, eps_ref, 0) plus binary32 sums of the deviations.  Equilibrium
// deviations, formed without cancellation (Eqs. equil1s, equil2as, equil2bs
// minus their rest values):
//   df_i = w_i [dS + 3 S q_i / c_l]
//   dg_i = w_i [d_eps / c_l^2 + eps gamma^2 (6 q_i^2 - 2 b2) / c_l^2] +- w_i eps gamma^2 4 q_i / c_l
//   dg_0 = w_0 [d_eps (3 - 2/c_l^2) + eps gamma^2 b2 (4 - 2/c_l^2)]
// with S = n gamma = n_ref + dS, q_i = e_i . beta, b2 = |beta|^2.
#pragma once

#include "rlb_device.cuh"
#include "rlb_dfloat.cuh"

namespace rlb {

// fetch(q, i): the population of plane q (velocity i = q mod 19) pulled from
// x - e_i, as stored (a solid neighbour yields the solid marker);
// bounce(q, i): the cell's own population of the opposite velocity, the link
// bounce-back value; put(q, v): store the post-collision value.
// A pulled marker is a NaN, so the sum of a phase's 19 values is NaN exactly
// when a marker (or a non-finite population) is among them: the per-value
// marker tests run only then.
template <bool SOLID, class Fetch, class Bounce>
__device__ __forceinline__ void gather_phase(float* v, int base, Fetch fetch, Bounce bounce) {
#pragma unroll
    for (int i = 0; i < 19; ++i) v[i] = fetch(base + i, i);
    if (SOLID) {
        float s = v[0];
#pragma unroll
        for (int i = 1; i < 19; ++i) s += v[i];
        if (isnan(s)) {
#pragma unroll
            for (int i = 1; i < 19; ++i)
                if (is_solid(v[i])) v[i] = bounce(base + i, i);
        }
    }
}

// EARLYF: the f populations are loaded into registers before the g phase's
// arithmetic, so that their loads are in flight during it (the same values,
// the same arithmetic; more registers per thread).
template <bool SOLID, class Fetch, class Bounce, class Put, bool EARLYF = false>
__device__ __forceinline__ void collide_cell_f32(Fetch fetch, Bounce bounce, Put put, const Dev32& c, bool& unphys,
                                                 bool& nonpos) {
    const float om = c.omega;
    // ---- phase 1: energy-momentum populations g_i (they alone fix eps, beta) ----
    float gg[19];
    float f[19];
    if (EARLYF) {
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = fetch(i, i);
    }
    gather_phase<SOLID>(gg, 19, fetch, bounce);
    float dE = gg[0], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        dE += gg[2 * p + 1] + gg[2 * p + 2];
        d[p] = gg[2 * p + 1] - gg[2 * p + 2];
    }
    const float mxf = c.c_l * (d[0] + d[3] + d[4] + d[5] + d[6]);
    const float myf = c.c_l * (d[1] + d[3] - d[4] + d[7] + d[8]);
    const float mzf = c.c_l * (d[2] + d[5] - d[6] + d[7] - d[8]);
    // Recovery, FP64 for the cancellation-prone root: E = eps_ref + sum dg and
    // d4 = E^2 - 3|M|^2/4 in FP64, sqrt(d4) from a binary32 seed and one FP64
    // Newton correction (relative error ~1e-14), eps = 2 sqrt(d4) - E.
    // D = 3E + eps has no cancellation, so beta = 3M/D and 1 - |beta|^2 are
    // formed in binary32 (the quotient is rounded to binary32 either way).
    // The binary32 <-> binary64 conversions run on the integer pipe.
    const double E = c.eps_ref + f2d(dE);
    const double Mx = f2d(mxf), My = f2d(myf), Mz = f2d(mzf);
    const double m2 = fma(Mx, Mx, fma(My, My, Mz * Mz));
    const double d4 = fma(E, E, -0.75 * m2);
    double y0, hy0;
    rsqrt_seed(d4, y0, hy0);
    const double s0 = d4 * y0;
    const double sq = fma(fma(-s0, s0, d4), hy0, s0);
    const double eps = fma(2.0, sq, -E);
    const float Df = d2f(fma(3.0, E, eps));
    const float deps = d2f(eps - c.eps_ref);
    const float epsf = d2f(eps);
    const float r3 = 3.0f / Df;
    const float bx = mxf * r3, by = myf * r3, bz = mzf * r3;
    const float b2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    const float gam2 = 1.0f / (1.0f - b2);
    const float eg = epsf * gam2;
    const float qv[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    {
        const float k1 = (deps - 2.0f * eg * b2) * c.inv_cl2;
        const float k2 = 6.0f * eg * c.inv_cl2;
        const float k3 = 4.0f * eg * c.inv_cl;
        put(19, fmaf(om, (float)kW0 * (deps * c.g0a + eg * b2 * c.g0b) - gg[0], gg[0]));
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const float w = (float)pair_w(p);
            const float gsym = w * fmaf(k2, qv[p] * qv[p], k1);
            const float gasy = w * k3 * qv[p];
            put(20 + 2 * p, fmaf(om, (gsym + gasy) - gg[2 * p + 1], gg[2 * p + 1]));
            put(21 + 2 * p, fmaf(om, (gsym - gasy) - gg[2 * p + 2], gg[2 * p + 2]));
        }
    }
    // ---- phase 2: number populations f_i ----
    if (EARLYF) {
        if (SOLID) {  // the markers test of gather_phase, on the values already loaded
            float s = f[0];
#pragma unroll
            for (int i = 1; i < 19; ++i) s += f[i];
            if (isnan(s)) {
#pragma unroll
                for (int i = 1; i < 19; ++i)
                    if (is_solid(f[i])) f[i] = bounce(i, i);
            }
        }
    } else {
        gather_phase<SOLID>(f, 0, fetch, bounce);
    }
    float dS = f[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) dS += f[i];
    const float sfull = c.n_ref + dS;
    const float fa = 3.0f * sfull * c.inv_cl;
    put(0, fmaf(om, (float)kW0 * dS - f[0], f[0]));
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const float w = (float)pair_w(p);
        const float fsym = w * dS;
        const float fasy = w * fa * qv[p];
        put(2 * p + 1, fmaf(om, (fsym + fasy) - f[2 * p + 1], f[2 * p + 1]));
        put(2 * p + 2, fmaf(om, (fsym - fasy) - f[2 * p + 2], f[2 * p + 2]));
    }
    unphys = !(pos_finite(sfull) && pos_finite(E) && nonneg_finite(d4) && pos_finite(eps) && below_one(b2));
    nonpos = nonpositive_eq(bx, by, bz, c.c_l);
}

// ---------------------------------------------------------------------------
// Compensated FP32 deviation collision, used for lattice speeds c_l > 1.
//
// At c_l > 1 the velocity terms of the g equilibria (w_i eps gamma^2 4 q_i/c_l
// in Eq. equil2as) are c_l times larger than their rest part, while the
// moments that drive the flow -- the energy, the momentum and, multiplied by
// c_l^2, the momentum flux -- are sums in which they cancel.  Storage in
// binary32 keeps each population to a relative 2^-24, which the scheme
// tolerates; binary32 arithmetic in the collision adds rounding errors of the
// same size that are coherent across the 18 moving populations of a cell (one
// rounded beta, one rounded eps gamma^2, weights and 1/c_l rounded to
// binary32), so the collision no longer conserves energy and momentum to that
// accuracy and the error grows over thousands of steps at low viscosity.
// This variant keeps the binary32 storage and removes the arithmetic error:
//   - the moment sums are compensated (error-free pair sums and differences,
//     rounding errors of the running sums collected and added back);
//   - the recovery and the equilibrium coefficients are formed in FP64 and
//     carried as binary32 pairs;
//   - the antisymmetric part of g^eq is formed from the momentum sums
//     themselves, 3 w_p (e_p . M)/c_l, which equals w_p eps gamma^2 4 q_p/c_l
//     for the recovered (eps, beta) (with eps = 3P, (4/3) eps gamma^2 beta =
//     M), so the equilibrium carries exactly the momentum of the gathered
//     populations;
//   - every equilibrium value is a binary32 pair; the non-equilibrium part
//     eq_i - h_i is rounded once to binary32 and the relaxed value
//     h_i + omega (eq_i - h_i) once more, when it is stored.
// ---------------------------------------------------------------------------
template <bool SOLID, class Fetch, class Bounce, class Put>
__device__ __forceinline__ void collide_cell_f32c(Fetch fetch, Bounce bounce, Put put, const Dev32& c, bool& unphys,
                                                  bool& nonpos) {
    const float om = c.omega;
    // ---- phase 1: energy-momentum populations g_i ----
    float gg[19];
    gather_phase<SOLID>(gg, 19, fetch, bounce);
    dfl dg[9];
    CSum esum(gg[0]);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        esum.add(two_sum(gg[2 * p + 1], gg[2 * p + 2]));
        dg[p] = two_sum(gg[2 * p + 1], -gg[2 * p + 2]);
    }
    // M / c_l = sum_p (g_p - g_opp(p)) e_p, per component
    CSum sx(dg[0].h), sy(dg[1].h), sz(dg[2].h);
    sx.c = dg[0].l, sy.c = dg[1].l, sz.c = dg[2].l;
    sx.add(dg[3]), sx.add(dg[4]), sx.add(dg[5]), sx.add(dg[6]);
    sy.add(dg[3]), sy.add(df_neg(dg[4])), sy.add(dg[7]), sy.add(dg[8]);
    sz.add(dg[5]), sz.add(df_neg(dg[6])), sz.add(dg[7]), sz.add(df_neg(dg[8]));
    const dfl Dx = sx.result(), Dy = sy.result(), Dz = sz.result();
    // Recovery in FP64: eps = 2 sqrt(E^2 - 3|M|^2/4) - E, beta = 3M/(3E + eps).
    const double E = c.eps_ref + df_dbl(esum.result());
    const double Mx = c.c_l_d * df_dbl(Dx), My = c.c_l_d * df_dbl(Dy), Mz = c.c_l_d * df_dbl(Dz);
    const double m2 = fma(Mx, Mx, fma(My, My, Mz * Mz));
    const double d4 = fma(E, E, -0.75 * m2);
    double y0, hs;
    rsqrt_seed(d4, y0, hs);
    double sq = d4 * y0;
    sq = fma(fma(-sq, sq, d4), hs, sq);
    sq = fma(fma(-sq, sq, d4), hs, sq);
    const double eps = fma(2.0, sq, -E);
    const double D = fma(3.0, E, eps);
    double rD = rcp_seed(D);
    rD = fma(rD, fma(-D, rD, 1.0), rD);
    rD = fma(rD, fma(-D, rD, 1.0), rD);
    const double r3 = 3.0 * rD;
    const double bx = Mx * r3, by = My * r3, bz = Mz * r3;
    const double b2 = fma(bx, bx, fma(by, by, bz * bz));
    const double omb2 = 1.0 - b2;
    double gam2 = rcp_seed(omb2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    const double eg = eps * gam2;
    const double deps = eps - c.eps_ref;
    // g^eq_i - g^ref_i = w_i [k1 + k2 q_i^2] +- 3 w_i (e_i . M)/c_l,
    //   k1 = (deps - 2 eg b2)/c_l^2, k2 = 6 eg / c_l^2 (per weight class)
    const double k1 = (deps - 2.0 * eg * b2) * c.inv_cl2_d, k2 = 6.0 * eg * c.inv_cl2_d;
    const dfl K1[2] = {df_of(k1 * (1.0 / 18.0)), df_of(k1 * (1.0 / 36.0))};
    const dfl K2[2] = {df_of(k2 * (1.0 / 18.0)), df_of(k2 * (1.0 / 36.0))};
    // 3 w_p as pairs: 1/6 and 1/12
    const dfl A3[2] = {{(float)(1.0 / 6.0), (float)(1.0 / 6.0 - (double)(float)(1.0 / 6.0))},
                       {(float)(1.0 / 12.0), (float)(1.0 / 12.0 - (double)(float)(1.0 / 12.0))}};
    const dfl Bx = df_of(bx), By = df_of(by), Bz = df_of(bz);
    const dfl qv[9] = {Bx, By, Bz, df_add(Bx, By), df_add(Bx, df_neg(By)), df_add(Bx, Bz), df_add(Bx, df_neg(Bz)),
                       df_add(By, Bz), df_add(By, df_neg(Bz))};
    const dfl ev[9] = {Dx, Dy, Dz, df_add(Dx, Dy), df_add(Dx, df_neg(Dy)), df_add(Dx, Dz), df_add(Dx, df_neg(Dz)),
                       df_add(Dy, Dz), df_add(Dy, df_neg(Dz))};
    {
        // g_0^eq - g_0^ref = w_0 [deps (3 - 2/c_l^2) + eg b2 (4 - 2/c_l^2)]   (Eq. equil2bs)
        const double g0 = (1.0 / 3.0) * fma(deps, 3.0 - 2.0 * c.inv_cl2_d, eg * b2 * (4.0 - 2.0 * c.inv_cl2_d));
        put(19, __fmaf_rn(om, df_sub_round(df_of(g0), gg[0]), gg[0]));
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const int cl = p < 3 ? 0 : 1;
            const dfl gsym = df_add(df_mul(K2[cl], df_mul(qv[p], qv[p])), K1[cl]);
            const dfl gasy = df_mul(A3[cl], ev[p]);
            put(20 + 2 * p, __fmaf_rn(om, df_sub_round(df_add(gsym, gasy), gg[2 * p + 1]), gg[2 * p + 1]));
            put(21 + 2 * p, __fmaf_rn(om, df_sub_round(df_add(gsym, df_neg(gasy)), gg[2 * p + 2]), gg[2 * p + 2]));
        }
    }
    // ---- phase 2: number populations f_i ----
    float f[19];
    gather_phase<SOLID>(f, 0, fetch, bounce);
    CSum ssum(f[0]);
#pragma unroll
    for (int i = 1; i < 19; ++i) ssum.add(f[i]);
    const double dS = df_dbl(ssum.result());
    const double S = c.n_ref_d + dS;
    // f^eq_i - f^ref_i = w_i dS +- w_i 3 S q_i / c_l   (Eq. equil1s, n gamma = S)
    const dfl FS[2] = {df_of(dS * (1.0 / 18.0)), df_of(dS * (1.0 / 36.0))};
    const double fa = 3.0 * S * c.inv_cl_d;
    const dfl FA[2] = {df_of(fa * (1.0 / 18.0)), df_of(fa * (1.0 / 36.0))};
    put(0, __fmaf_rn(om, df_sub_round(df_of(dS * (1.0 / 3.0)), f[0]), f[0]));
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int cl = p < 3 ? 0 : 1;
        const dfl fasy = df_mul(FA[cl], qv[p]);
        put(2 * p + 1, __fmaf_rn(om, df_sub_round(df_add(FS[cl], fasy), f[2 * p + 1]), f[2 * p + 1]));
        put(2 * p + 2, __fmaf_rn(om, df_sub_round(df_add(FS[cl], df_neg(fasy)), f[2 * p + 2]), f[2 * p + 2]));
    }
    unphys = !(pos_finite(S) && pos_finite(E) && nonneg_finite(d4) && pos_finite(eps) && below_one(b2));
    nonpos = nonpositive_eq(d2f(bx), d2f(by), d2f(bz), c.c_l);
}

}  // namespace rlb

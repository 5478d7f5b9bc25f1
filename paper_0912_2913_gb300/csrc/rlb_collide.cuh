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

template <bool SOLID, class Fetch, class Bounce, class Put>
__device__ __forceinline__ void collide_cell_f32(Fetch fetch, Bounce bounce, Put put, const Dev32& c, bool& unphys,
                                                 bool& nonpos) {
    const float om = c.omega;
    // ---- phase 1: energy-momentum populations g_i (they alone fix eps, beta) ----
    float gg[19];
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
    const float y0 = rsqrtf(d2f_seed(d4));
    const double s0 = d4 * f2d(y0);
    const double sq = fma(fma(-s0, s0, d4), f2d(0.5f * y0), s0);
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
    float f[19];
    gather_phase<SOLID>(f, 0, fetch, bounce);
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

}  // namespace rlb

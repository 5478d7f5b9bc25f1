// rlb_forward.cu -- forward kernels of librlb: the fused stream-and-collide
// step of the relativistic lattice Boltzmann scheme (Eqs. lbe1, lbe2 with the
// eps = 3P equilibria Eqs. equil1s, equil2as, equil2bs), the equilibrium
// initialisation and the macroscopic output.
//
// One thread owns one cell.  A step pulls the 38 populations that arrive at
// the cell (h_i(x) = A_i(x - e_i), link bounce-back h_i(x) = A_opp(i)(x) when
// x - e_i is solid), forms the five moments, recovers (n gamma, eps, beta) in
// closed form, builds the equilibria pair by pair (velocities i and opp(i)
// share every term but the odd one) and writes the BGK-relaxed populations
// B_i = h_i + (eq_i - h_i)/tau.  State planes are structure-of-arrays, so a
// warp's loads and stores of one plane are 32 consecutive elements (the x
// neighbours are off by one element and share cache sectors).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "rlb_collide.cuh"
#include "rlb_device.cuh"

namespace rlb {

namespace {
int g_last_launches = 0;
}
int last_launch_count() { return g_last_launches; }
void set_last_launch_count(int n) { g_last_launches = n; }


// ---------------------------------------------------------------------------
// FP64 step.
// ---------------------------------------------------------------------------

// Moments S_f, E and d = M / c_l of the FP64 step, summed as a fixed tree
// over eight partials: partial j holds pair j, and for j < 2 also unit
// j + 8 (pair 8 for j = 0, the rest population for j = 1).  They are combined
// as ((P0 + P4) + (P2 + P6)) + ((P1 + P5) + (P3 + P7)), the order in which an
// xor butterfly over eight lanes (offsets 4, 2, 1) adds them on every lane,
// so k_step_f64_split, which spreads the units of a cell over eight lanes,
// forms the same sums; the partials of d that are identically zero are left
// out here (adding an exact zero leaves any value but -0 unchanged).
__device__ __forceinline__ void moments_tree8(const double* f, const double* g, double& sf, double& e, double& dx,
                                              double& dy, double& dz) {
    double sp[9], ep[9], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        sp[p] = f[2 * p + 1] + f[2 * p + 2];
        ep[p] = g[2 * p + 1] + g[2 * p + 2];
        d[p] = g[2 * p + 1] - g[2 * p + 2];
    }
    const double s0 = sp[0] + sp[8], s1 = sp[1] + f[0];
    const double e0 = ep[0] + ep[8], e1 = ep[1] + g[0];
    sf = ((s0 + sp[4]) + (sp[2] + sp[6])) + ((s1 + sp[5]) + (sp[3] + sp[7]));
    e = ((e0 + ep[4]) + (ep[2] + ep[6])) + ((e1 + ep[5]) + (ep[3] + ep[7]));
    // x: pairs 0, 3, 4, 5, 6; y: 1, 3, -4, 7, 8; z: 2, 5, -6, 7, -8
    dx = ((d[0] + d[4]) + d[6]) + (d[5] + d[3]);
    dy = (d[8] - d[4]) + (d[1] + (d[3] + d[7]));
    dz = (-d[8] + (d[2] - d[6])) + (d[5] + d[7]);
}

template <int XBC, bool SOLID>
__global__ void __launch_bounds__(128) k_step_f64(const double* __restrict__ A, double* __restrict__ B, Geom g,
                                                  Phys ph, Counters cnt, int count, long long step_index) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int x, y, z;
    cell_coords(g, idx, x, y, z);
    if (g.zhalo && (z == 0 || z == g.nz - 1)) return;  // z halo planes: filled by the exchange
    const long long S = g.S;
    if (XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1)) {
        // Ghost planes are not collided.  The inflow plane keeps its fixed
        // equilibrium (copied so that every cell of B is written); outflow
        // ghosts are written by the cell they copy.
        if (XBC == XBC_INFLOW_OUTFLOW && x == 0) {
#pragma unroll
            for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = __ldg(RLB_CHK_PTR(A, q * S + idx, 38ll * S));
        }
        return;
    }
    const PullOffsets o(g, x, y, z);
    double f[19], gg[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int s = idx + o.src(i);
        f[i] = __ldg(RLB_CHK_PTR(A, i * S + s, 38ll * S));
        gg[i] = __ldg(RLB_CHK_PTR(A, (19 + i) * S + s, 38ll * S));
    }
    if (SOLID) {
        if (is_solid(f[0])) {  // the cell itself is solid: keep the marker
            const double m = solid_marker_d();
#pragma unroll
            for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = m;
            return;
        }
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (is_solid(f[i])) {  // link bounce-back
                f[i] = __ldg(RLB_CHK_PTR(A, opp(i) * S + idx, 38ll * S));
                gg[i] = __ldg(RLB_CHK_PTR(A, (19 + opp(i)) * S + idx, 38ll * S));
            }
        }
    }
    // d = M / c_l (the pair differences summed along each axis)
    double sf, E, dx, dy, dz;
    moments_tree8(f, gg, sf, E, dx, dy, dz);
    // Recovery with eps = 3P: eps = -E + sqrt(4E^2 - 3M^2), beta = 3M/(3E + eps).
    // Square root and reciprocals from binary32 seeds (converted on the integer
    // pipe, valid for any exponent of the argument) with two FP64 Newton
    // corrections each: full double accuracy at a fraction of the IEEE
    // sequences' cost on this GPU's FP64 pipe.
    const double m2 = fma(dx, dx, fma(dy, dy, dz * dz));  // |M|^2 / c_l^2
    const double disc = fma(4.0 * E, E, ph.m3cl2 * m2);   // 4E^2 - 3|M|^2
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
    const double r3 = ph.three_cl * rD;  // beta = 3 M / D = 3 c_l d / D
    const double bx = dx * r3, by = dy * r3, bz = dz * r3;
    const double b2 = fma(bx, bx, fma(by, by, bz * bz));
    const double omb2 = 1.0 - b2;
    double gam2 = rcp_seed(omb2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    const bool unphys = !(pos_finite(sf) && pos_finite(E) && nonneg_finite(disc) && pos_finite(eps) && below_one(b2));
    // beta rounded to binary32 on the integer pipe (the same rounding as a conversion)
    const bool nonpos = nonpositive_eq(d2f(bx), d2f(by), d2f(bz), (float)ph.c_l);

    // The relaxed values omega eq + (1 - omega) h, with omega and the weights
    // folded into per-run constants (Phys::c_*):
    //   f^eq_i = w_i S_f (1 + 3 q_i / c_l)     (Eq. equil1s with n gamma = S_f)
    //   g^eq_i = w_i [eps/c_l^2 + eps gamma^2 (6 q^2/c_l^2 - 2 b2/c_l^2)] +- w_i eps gamma^2 4 q / c_l
    //   g_0^eq = w_0 [4 eps gamma^2 - eps (2 + c_l^2)/c_l^2 - 2 eps gamma^2 b2/c_l^2]   (Eq. equil2bs)
    const double omw = 1.0 - ph.omega;
    const double q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    const double eg = eps * gam2;
    const double egb2 = eg * b2;
    const double t = fma(-2.0, egb2, eps);  // eps - 2 eg b2
    const double k1w[2] = {t * ph.c_k1[0], t * ph.c_k1[1]};
    const double k2w[2] = {eg * ph.c_k2[0], eg * ph.c_k2[1]};
    const double k3w[2] = {eg * ph.c_k3[0], eg * ph.c_k3[1]};
    const double fsw[2] = {sf * ph.c_fs[0], sf * ph.c_fs[1]};
    const double faw[2] = {sf * ph.c_fa[0], sf * ph.c_fa[1]};
    double outf[19], outg[19];
    outf[0] = fma(omw, f[0], sf * ph.c_f0);
    outg[0] = fma(omw, gg[0], fma(eg, ph.c_g0[0], fma(eps, ph.c_g0[1], egb2 * ph.c_g0[2])));
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int cl = p < 3 ? 0 : 1;
        outf[2 * p + 1] = fma(omw, f[2 * p + 1], fma(faw[cl], q[p], fsw[cl]));
        outf[2 * p + 2] = fma(omw, f[2 * p + 2], fma(-faw[cl], q[p], fsw[cl]));
        const double gsym = fma(k2w[cl], q[p] * q[p], k1w[cl]);
        outg[2 * p + 1] = fma(omw, gg[2 * p + 1], fma(k3w[cl], q[p], gsym));
        outg[2 * p + 2] = fma(omw, gg[2 * p + 2], fma(-k3w[cl], q[p], gsym));
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        B[RLB_CHK(i * S + idx, 38ll * S)] = outf[i];
        B[RLB_CHK((19 + i) * S + idx, 38ll * S)] = outg[i];
    }
    if (XBC != XBC_PERIODIC && x == g.nx - 2) {  // outflow ghost x = nx-1 copies x = nx-2
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            B[RLB_CHK(i * S + idx + 1, 38ll * S)] = outf[i];
            B[RLB_CHK((19 + i) * S + idx + 1, 38ll * S)] = outg[i];
        }
    }
    if (XBC == XBC_OUTFLOW_BOTH && x == 1) {  // outflow ghost x = 0 copies x = 1
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            B[RLB_CHK(i * S + idx - 1, 38ll * S)] = outf[i];
            B[RLB_CHK((19 + i) * S + idx - 1, 38ll * S)] = outg[i];
        }
    }
    if (count) count_flags(cnt, unphys, nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
}

// ---------------------------------------------------------------------------
// FP64 step for small lattices (the 1600-cell shock tube): eight lanes per
// cell.  The FP64 pipe issues one warp instruction about every 76 cycles per
// scheduler on this GPU (1.68 FMA per SM per clock), whatever the number of
// active lanes, so a cell's ~200 FP64 instructions on one thread take some
// 15,000 cycles however few cells share a scheduler.  Here lane j of a cell's
// group pulls and relaxes pair j (and pair 8 for j = 0, the rest population
// for j = 1); the moments are the lanes' partials summed by an xor butterfly
// (the tree of moments_tree8), the recovery is repeated on every lane, and a
// warp issues about half the FP64 instructions.  The arithmetic is that of
// k_step_f64 term for term, so the two give the same values.
// ---------------------------------------------------------------------------
template <int XBC, bool SOLID>
__global__ void __launch_bounds__(128) k_step_f64_split(const double* __restrict__ A, double* __restrict__ B, Geom g,
                                                        Phys ph, Counters cnt, int count, long long step_index) {
    const unsigned full = 0xffffffffu;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = threadIdx.x & 7;  // lane of the cell's group
    const long long cell = t >> 3;
    const bool live = cell < g.N;
    const int idx = live ? (int)cell : 0;
    int x, y, z;
    cell_coords(g, idx, x, y, z);
    const bool halo = g.zhalo && (z == 0 || z == g.nz - 1);  // filled by the exchange
    const bool ghost = XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1);
    const bool work = live && !halo && !ghost;  // a collided cell
    const long long S = g.S;
    const PullOffsets o(g, x, y, z);
    // this lane's populations: pair j (a: +, b: -); lane 0 also pair 8
    // (c: +, d: -), lane 1 the rest population (c)
    const int ia = 2 * j + 1, ib = 2 * j + 2;
    auto pull = [&](int i, double& fv, double& gv) {
        const int src = idx + o.src(i);
        fv = __ldg(RLB_CHK_PTR(A, i * S + src, 38ll * S));
        gv = __ldg(RLB_CHK_PTR(A, (19 + i) * S + src, 38ll * S));
        if (SOLID && is_solid(fv)) {  // link bounce-back
            fv = __ldg(RLB_CHK_PTR(A, opp(i) * S + idx, 38ll * S));
            gv = __ldg(RLB_CHK_PTR(A, (19 + opp(i)) * S + idx, 38ll * S));
        }
    };
    double fa = 0.0, fb = 0.0, ga = 0.0, gb = 0.0, fc = 0.0, fd = 0.0, gc = 0.0, gd = 0.0;
    bool own_solid = false;
    if (work) {
        pull(ia, fa, ga);
        pull(ib, fb, gb);
        if (j == 0) {
            pull(17, fc, gc);
            pull(18, fd, gd);
        } else if (j == 1) {
            fc = __ldg(RLB_CHK_PTR(A, idx, 38ll * S));
            gc = __ldg(RLB_CHK_PTR(A, 19 * S + idx, 38ll * S));
            own_solid = SOLID && is_solid(fc);
        }
    }
    const bool solid = __shfl_sync(full, own_solid, (threadIdx.x & 24) + 1);  // lane 1 holds f_0
    // partials of the moments (the tree of moments_tree8)
    double ps = fa + fb, pe = ga + gb;
    const double dj = ga - gb;
    if (j == 0) {
        ps = ps + (fc + fd);
        pe = pe + (gc + gd);
    } else if (j == 1) {
        ps = ps + fc;
        pe = pe + gc;
    }
    const double d8 = gc - gd;  // pair 8 on lane 0
    const int ex = pair_ex(j), ey = pair_ey(j), ez = pair_ez(j);
    double px = ex ? dj : 0.0;
    double py = j == 0 ? d8 : (ey > 0 ? dj : (ey < 0 ? -dj : 0.0));
    double pz = j == 0 ? -d8 : (ez > 0 ? dj : (ez < 0 ? -dj : 0.0));
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
        ps += __shfl_xor_sync(full, ps, off);
        pe += __shfl_xor_sync(full, pe, off);
        px += __shfl_xor_sync(full, px, off);
        py += __shfl_xor_sync(full, py, off);
        pz += __shfl_xor_sync(full, pz, off);
    }
    const double sf = ps, E = pe, dx = px, dy = py, dz = pz;
    // recovery: as in k_step_f64
    const double m2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double disc = fma(4.0 * E, E, ph.m3cl2 * m2);
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
    const double r3 = ph.three_cl * rD;
    const double bx = dx * r3, by = dy * r3, bz = dz * r3;
    const double b2 = fma(bx, bx, fma(by, by, bz * bz));
    const double omb2 = 1.0 - b2;
    double gam2 = rcp_seed(omb2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    gam2 = fma(gam2, fma(-omb2, gam2, 1.0), gam2);
    const bool unphys = !(pos_finite(sf) && pos_finite(E) && nonneg_finite(disc) && pos_finite(eps) && below_one(b2));
    const bool nonpos = nonpositive_eq(d2f(bx), d2f(by), d2f(bz), (float)ph.c_l);
    // equilibria and relaxation of this lane's populations: as in k_step_f64
    const double omw = 1.0 - ph.omega;
    const double q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    const double eg = eps * gam2;
    const double egb2 = eg * b2;
    const double tt = fma(-2.0, egb2, eps);
    const double k1w[2] = {tt * ph.c_k1[0], tt * ph.c_k1[1]};
    const double k2w[2] = {eg * ph.c_k2[0], eg * ph.c_k2[1]};
    const double k3w[2] = {eg * ph.c_k3[0], eg * ph.c_k3[1]};
    const double fsw[2] = {sf * ph.c_fs[0], sf * ph.c_fs[1]};
    const double faw[2] = {sf * ph.c_fa[0], sf * ph.c_fa[1]};
    double qj = q[0];
#pragma unroll
    for (int p = 1; p < 8; ++p) qj = j == p ? q[p] : qj;
    const int cl = j < 3 ? 0 : 1;
    const double fsc = cl ? fsw[1] : fsw[0], fac = cl ? faw[1] : faw[0];
    const double k1c = cl ? k1w[1] : k1w[0], k2c = cl ? k2w[1] : k2w[0], k3c = cl ? k3w[1] : k3w[0];
    const double ofa = fma(omw, fa, fma(fac, qj, fsc));
    const double ofb = fma(omw, fb, fma(-fac, qj, fsc));
    const double gsym = fma(k2c, qj * qj, k1c);
    const double oga = fma(omw, ga, fma(k3c, qj, gsym));
    const double ogb = fma(omw, gb, fma(-k3c, qj, gsym));
    double ofc, ofd = 0.0, ogc, ogd = 0.0;
    if (j == 0) {  // pair 8 (diagonal weight)
        ofc = fma(omw, fc, fma(faw[1], q[8], fsw[1]));
        ofd = fma(omw, fd, fma(-faw[1], q[8], fsw[1]));
        const double gs8 = fma(k2w[1], q[8] * q[8], k1w[1]);
        ogc = fma(omw, gc, fma(k3w[1], q[8], gs8));
        ogd = fma(omw, gd, fma(-k3w[1], q[8], gs8));
    } else {  // the rest population (lane 1)
        ofc = fma(omw, fc, sf * ph.c_f0);
        ogc = fma(omw, gc, fma(eg, ph.c_g0[0], fma(eps, ph.c_g0[1], egb2 * ph.c_g0[2])));
    }
    auto put = [&](int i, long long at, double fv, double gv) {
        B[RLB_CHK(i * S + at, 38ll * S)] = fv;
        B[RLB_CHK((19 + i) * S + at, 38ll * S)] = gv;
    };
    if (work) {
        if (solid) {  // the cell itself is solid: keep the marker
            const double m = solid_marker_d();
            put(ia, idx, m, m);
            put(ib, idx, m, m);
            if (j == 0) {
                put(17, idx, m, m);
                put(18, idx, m, m);
            } else if (j == 1) {
                put(0, idx, m, m);
            }
        } else {
            auto put_all = [&](long long at) {
                put(ia, at, ofa, oga);
                put(ib, at, ofb, ogb);
                if (j == 0) {
                    put(17, at, ofc, ogc);
                    put(18, at, ofd, ogd);
                } else if (j == 1) {
                    put(0, at, ofc, ogc);
                }
            };
            put_all(idx);
            if (XBC != XBC_PERIODIC && x == g.nx - 2) put_all(idx + 1);  // outflow ghost x = nx-1 copies x = nx-2
            if (XBC == XBC_OUTFLOW_BOTH && x == 1) put_all(idx - 1);      // outflow ghost x = 0 copies x = 1
        }
    } else if (XBC == XBC_INFLOW_OUTFLOW && live && !halo && x == 0) {
        // the inflow plane keeps its fixed equilibrium (copied)
        auto copy = [&](int i) {
            B[RLB_CHK(i * S + idx, 38ll * S)] = __ldg(RLB_CHK_PTR(A, i * S + idx, 38ll * S));
            B[RLB_CHK((19 + i) * S + idx, 38ll * S)] = __ldg(RLB_CHK_PTR(A, (19 + i) * S + idx, 38ll * S));
        };
        copy(ia);
        copy(ib);
        if (j == 0) {
            copy(17);
            copy(18);
        } else if (j == 1) {
            copy(0);
        }
    }
    if (count) {
        const bool mine = j == 0 && work && !solid;
        count_flags(cnt, mine && unphys, mine && nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
    }
}

// ---------------------------------------------------------------------------
// FP32 deviation step.  Populations are stored as d_i = p_i - p_i^ref with
// p^ref the rest equilibrium of (n_ref, eps_ref): f_i^ref = w_i n_ref,
// g_i^ref = w_i eps_ref / c_l^2 (i > 0), g_0^ref = w_0 eps_ref (3 - 2/c_l^2).
// Streaming and BGK are linear and the reference is uniform and symmetric, so
// the step maps deviations to deviations.  The moments are the reference
// moments (n_ref, eps_ref, 0) plus the float sums of the deviations; the
// recovery, where the strong-shock cancellation sits, runs in FP64:
//   E = eps_ref + sum dg,  sqrt(E^2 - 3M^2/4) and 1/(3E + eps) each from a
//   binary32 seed and one FP64 Newton correction (relative error ~1e-14),
//   eps = 2 sqrt(...) - E, beta = 3 M / (3E + eps), 1 - |beta|^2 in FP64.
// The equilibrium deviations are formed without cancellation:
//   df_i = w_i [dS + 3 S q_i / c_l]
//   dg_i = w_i [d_eps / c_l^2 + eps gamma^2 (6 q_i^2 - 2 b2) / c_l^2] +- w_i eps gamma^2 4 q_i / c_l
//   dg_0 = w_0 [d_eps (3 - 2/c_l^2) + eps gamma^2 b2 (4 - 2/c_l^2)]
// with dS = sum df, d_eps = eps - eps_ref (FP64, then rounded).
// ---------------------------------------------------------------------------

// MINB: resident 256-thread blocks per SM the register budget is cut for;
// PREF: prefetch the populations of the f phase into L2 before the g phase
// runs (the default launch: the f loads then hit L2 instead of waiting on
// HBM, measured +16% on the 200x100x100 sphere).
// I: type of the element offsets, int when 38 S < 2^31 (fewer address
// instructions: measured +2 % / +6 % for the two shapes the first step picks
// from on the 200x100x100 sphere), else long long.
// COMP: the compensated collision (collide_cell_f32c), run for c_l > 1.
// EARLY: the f populations are loaded before the g phase's arithmetic.
// TB: threads per block the register budget is cut for.
template <int XBC, bool SOLID, int MINB, bool PREF, typename I = long long, bool COMP = false, bool EARLY = false,
          int TB = 256>
__global__ void __launch_bounds__(TB, MINB) k_step_f32(const float* __restrict__ A, float* __restrict__ B, Geom g,
                                                       Dev32 c, Counters cnt, int count, long long step_index) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int x, y, z;
    cell_coords(g, idx, x, y, z);
    if (g.zhalo && (z == 0 || z == g.nz - 1)) return;  // z halo planes: filled by the exchange
    const I S = (I)g.S;
    // I = unsigned: the f planes (0..18) and the g planes (19..37) are
    // addressed from their own base pointers with unsigned 32-bit element
    // offsets (for lattices with 38 S >= 2^31 and 19 S < 2^32), which costs
    // no more address arithmetic than the int offsets.
    constexpr bool SPLIT = std::is_same<I, unsigned>::value;
    const float* __restrict__ Ag = SPLIT ? A + 19ll * g.S : A;
    float* Bg = SPLIT ? B + 19ll * g.S : B;
    const long long lim = (SPLIT ? 19ll : 38ll) * g.S;  // extent the checked builds test against
    auto pq = [](int q) { return (SPLIT && q >= 19) ? q - 19 : q; };  // plane number within its base
    auto abase = [&](int q) { return (SPLIT && q >= 19) ? Ag : A; };
    if (XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1)) {
        if (XBC == XBC_INFLOW_OUTFLOW && x == 0) {
#pragma unroll
            for (int q = 0; q < 38; ++q)
                ((SPLIT && q >= 19) ? Bg : B)[RLB_CHK(pq(q) * S + idx, lim)] = __ldg(RLB_CHK_PTR(abase(q), pq(q) * S + idx, lim));
        }
        return;
    }
    const PullOffsets o(g, x, y, z);
    const int dup = (XBC != XBC_PERIODIC && x == g.nx - 2) ? 1 : ((XBC == XBC_OUTFLOW_BOTH && x == 1) ? -1 : 0);
    float* Bc = B + idx;
    float* Bgc = Bg + idx;
    auto put = [&](int q, float v) {
        if constexpr (SPLIT) {
            float* b = q >= 19 ? Bgc : Bc;
            b[RLB_CHK_OFF(pq(q) * S, idx, lim)] = v;
            // the outflow copy: dup (+-1) moves the pointer, so that the
            // unsigned offset never has to hold a negative value
            if (dup) (b + dup)[RLB_CHK_OFF(pq(q) * S, idx + dup, lim)] = v;
        } else {
            Bc[RLB_CHK_OFF(q * S, idx, 38ll * S)] = v;
            if (dup) Bc[RLB_CHK_OFF(q * S + dup, idx, 38ll * S)] = v;
        }
    };
    if (SOLID && is_solid(__ldg(RLB_CHK_PTR(abase(19), pq(19) * S + idx, lim)))) {  // the cell itself is solid: keep the marker
        const float m = solid_marker_f();
#pragma unroll
        for (int q = 0; q < 38; ++q) ((SPLIT && q >= 19) ? Bgc : Bc)[RLB_CHK_OFF(pq(q) * S, idx, lim)] = m;
        return;
    }
    if (PREF) {
#pragma unroll
        for (int i = 0; i < 19; ++i) asm volatile("prefetch.global.L2 [%0];" ::"l"(RLB_CHK_PTR(A, i * S + idx + o.src(i), lim)));
    }
    auto fetch = [&](int q, int i) {
        if constexpr (SPLIT)
            return __ldg(RLB_CHK_PTR(abase(q), pq(q) * S + idx + o.src(i), lim));
        else
            return __ldg(RLB_CHK_PTR(A, q * S + idx + o.src(i), 38ll * S));
    };
    auto bounce = [&](int q, int i) {  // link bounce-back
        if constexpr (SPLIT)
            return __ldg(RLB_CHK_PTR(abase(q), (pq(q) - i + opp(i)) * S + idx, lim));
        else
            return __ldg(RLB_CHK_PTR(A, (q - i + opp(i)) * S + idx, 38ll * S));
    };
    bool unphys, nonpos;
    if (COMP)
        collide_cell_f32c<SOLID>(fetch, bounce, put, c, unphys, nonpos);
    else
        collide_cell_f32<SOLID, decltype(fetch), decltype(bounce), decltype(put), EARLY>(fetch, bounce, put, c, unphys,
                                                                                        nonpos);
    if (count) count_flags(cnt, unphys, nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
}

// Persistent variant: a grid of (SMs x resident blocks) threads walks the
// lattice with a grid stride; before colliding its current cell a thread
// issues L2 prefetches for all 38 populations of its next cell, so every
// gather hits L2 while HBM streams the next cells in (software pipelining
// without registers).  Same per-cell arithmetic as k_step_f32.
template <int XBC, bool SOLID, bool CS>
__global__ void __launch_bounds__(256, 3) k_step_f32_pipe(const float* __restrict__ A, float* __restrict__ B, Geom g,
                                                          Dev32 c, Counters cnt, int count, long long step_index) {
    const long long S = g.S;
    const long long stride = (long long)gridDim.x * blockDim.x;
    auto prefetch_cell = [&](int idx) {
        int x, y, z;
        cell_coords(g, idx, x, y, z);
        if (XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1)) return;
        if (g.zhalo && (z == 0 || z == g.nz - 1)) return;
        const PullOffsets o(g, x, y, z);
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(RLB_CHK_PTR(A, (19 + i) * S + idx + o.src(i), 38ll * S)));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(RLB_CHK_PTR(A, i * S + idx + o.src(i), 38ll * S)));
        }
    };
    // 64-bit loop counter: li + stride cannot wrap for any accepted N
    long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (li < g.N) prefetch_cell((int)li);
    for (; li < g.N; li += stride) {
        const int idx = (int)li;
        if (li + stride < g.N) prefetch_cell((int)(li + stride));
        int x, y, z;
        cell_coords(g, idx, x, y, z);
        if (g.zhalo && (z == 0 || z == g.nz - 1)) continue;
        if (XBC != XBC_PERIODIC && (x == 0 || x == g.nx - 1)) {
            if (XBC == XBC_INFLOW_OUTFLOW && x == 0) {
#pragma unroll
                for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = __ldg(RLB_CHK_PTR(A, q * S + idx, 38ll * S));
            }
            continue;
        }
        const PullOffsets o(g, x, y, z);
        const int dup = (XBC != XBC_PERIODIC && x == g.nx - 2) ? 1 : ((XBC == XBC_OUTFLOW_BOTH && x == 1) ? -1 : 0);
        float* Bc = B + idx;
        auto put = [&](int q, float v) {
            if (CS) {
                __stcs(Bc + q * S, v);
                if (dup) __stcs(Bc + q * S + dup, v);
            } else {
                Bc[RLB_CHK_OFF(q * S, idx, 38ll * S)] = v;
                if (dup) Bc[RLB_CHK_OFF(q * S + dup, idx, 38ll * S)] = v;
            }
        };
        if (SOLID && is_solid(__ldg(RLB_CHK_PTR(A, 19 * S + idx, 38ll * S)))) {
            const float m = solid_marker_f();
#pragma unroll
            for (int q = 0; q < 38; ++q) Bc[RLB_CHK_OFF(q * S, idx, 38ll * S)] = m;
            continue;
        }
        auto fetch = [&](int q, int i) { return __ldg(RLB_CHK_PTR(A, q * S + idx + o.src(i), 38ll * S)); };
        auto bounce = [&](int q, int i) { return __ldg(RLB_CHK_PTR(A, (q - i + opp(i)) * S + idx, 38ll * S)); };
        bool unphys, nonpos;
        collide_cell_f32<SOLID>(fetch, bounce, put, c, unphys, nonpos);
        if (count) count_flags(cnt, unphys, nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
    }
}

// ---------------------------------------------------------------------------
// Equilibria of given fields in FP64 (initialisation and inflow plane):
// Eqs. (equil1s), (equil2as), (equil2bs).
// ---------------------------------------------------------------------------
__device__ void equilibrium_f64(double n, double eps, double bx, double by, double bz, const Phys& ph, double* f,
                                double* g) {
    const double b2 = bx * bx + by * by + bz * bz;
    const double gam2 = 1.0 / (1.0 - b2);
    const double ng = n * sqrt(gam2);
    const double eg = eps * gam2;
    const double q[9] = {bx, by, bz, bx + by, bx - by, bx + bz, bx - bz, by + bz, by - bz};
    f[0] = kW0 * ng;
    g[0] = kW0 * (4.0 * eg - eps * (2.0 * ph.inv_cl2 + 1.0) - 2.0 * eg * b2 * ph.inv_cl2);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const double w = pair_w(p);
        const double fa = 3.0 * q[p] * ph.inv_cl;
        f[2 * p + 1] = w * ng * (1.0 + fa);
        f[2 * p + 2] = w * ng * (1.0 - fa);
        const double gs = eps * ph.inv_cl2 + eg * (6.0 * q[p] * q[p] - 2.0 * b2) * ph.inv_cl2;
        const double ga = eg * 4.0 * q[p] * ph.inv_cl;
        g[2 * p + 1] = w * (gs + ga);
        g[2 * p + 2] = w * (gs - ga);
    }
}

// Rest equilibrium of the FP32 deviation reference.
__device__ __forceinline__ void reference_eq(const Phys& ph, double* fr, double* gr) {
    fr[0] = kW0 * ph.n_ref;
    gr[0] = kW0 * ph.eps_ref * (3.0 - 2.0 * ph.inv_cl2);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const double w = pair_w(p);
        fr[2 * p + 1] = fr[2 * p + 2] = w * ph.n_ref;
        gr[2 * p + 1] = gr[2 * p + 2] = w * ph.eps_ref * ph.inv_cl2;
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_init(const double* __restrict__ n, const double* __restrict__ eps,
                                              const double* __restrict__ beta, const uint8_t* __restrict__ solid,
                                              T* __restrict__ A, T* __restrict__ B, Geom g, Phys ph) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long S = g.S;
    if (solid && solid[idx]) {
        T m;
        if constexpr (sizeof(T) == 8) m = solid_marker_d(); else m = solid_marker_f();
        for (int q = 0; q < 38; ++q) A[RLB_CHK(q * S + idx, 38ll * S)] = B[RLB_CHK(q * S + idx, 38ll * S)] = m;
        return;
    }
    const int x = idx % g.nx;
    double f[19], gg[19];
    if (g.xbc == XBC_INFLOW_OUTFLOW && x == 0)
        equilibrium_f64(ph.n_in, ph.eps_in, ph.beta_in[0], ph.beta_in[1], ph.beta_in[2], ph, f, gg);
    else
        equilibrium_f64(n[idx], eps[idx], beta[idx], beta[g.N + idx], beta[2 * (long long)g.N + idx], ph, f, gg);
    if constexpr (sizeof(T) == 4) {
        double fr[19], gr[19];
        reference_eq(ph, fr, gr);
        for (int i = 0; i < 19; ++i) {
            f[i] -= fr[i];
            gg[i] -= gr[i];
        }
    }
    for (int i = 0; i < 19; ++i) {
        A[RLB_CHK(i * S + idx, 38ll * S)] = B[RLB_CHK(i * S + idx, 38ll * S)] = (T)f[i];
        A[RLB_CHK((19 + i) * S + idx, 38ll * S)] = B[RLB_CHK((19 + i) * S + idx, 38ll * S)] = (T)gg[i];
    }
}

// ---------------------------------------------------------------------------
// Macroscopic output of a stored state (no gather: the moments of the
// post-collision populations equal those of the gathered ones, the
// collision conserves them).  IEEE sqrt and division.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_macro(const T* __restrict__ A, double* __restrict__ n,
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
        f[i] = (double)A[RLB_CHK(i * S + idx, 38ll * S)];
        gg[i] = (double)A[RLB_CHK((19 + i) * S + idx, 38ll * S)];
    }
    double sf, E, mx, my, mz;
    moments_pairs(f, gg, sf, E, mx, my, mz);
    if constexpr (sizeof(T) == 4) {
        sf += ph.n_ref;
        E += ph.eps_ref;
    }
    mx *= ph.c_l;
    my *= ph.c_l;
    mz *= ph.c_l;
    const double m2 = mx * mx + my * my + mz * mz;
    const double disc = 4.0 * E * E - 3.0 * m2;
    const double e = sqrt(disc) - E;
    const double D = 3.0 * E + e;
    const double bx = 3.0 * mx / D, by = 3.0 * my / D, bz = 3.0 * mz / D;
    const double b2 = bx * bx + by * by + bz * bz;
    const double nn = sf * sqrt(1.0 - b2);
    n[idx] = nn;
    eps[idx] = e;
    beta[idx] = bx;
    beta[g.N + idx] = by;
    beta[2 * (long long)g.N + idx] = bz;
    const bool bad = !(pos_finite(sf) && pos_finite(E) && nonneg_finite(disc) && pos_finite(e) && below_one(b2) &&
                       pos_finite(nn));
    if (bad) atomicAdd(bad_count, 1ull);
}

__global__ void k_conversions(const float* __restrict__ fi, const double* __restrict__ di, long long n,
                              double* __restrict__ fo, float* __restrict__ dout) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        fo[k] = f2d(fi[k]);
        dout[k] = d2f(di[k]);
    }
}

cudaError_t launch_conversions(const float* fi, const double* di, long long n, double* fo, float* dout) {
    if (n > 0) k_conversions<<<1024, 256>>>(fi, di, n, fo, dout);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

__global__ void k_check_solid_planes(Geom g, const uint8_t* __restrict__ solid, unsigned long long* flag) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int plane = g.ny * g.nz;
    if (t >= 4 * plane) return;
    const int which = t / plane, yz = t - which * plane;
    const int xs[4] = {0, 1, g.nx - 2, g.nx - 1};
    if (solid[(long long)yz * g.nx + xs[which]]) atomicAdd(flag, 1ull);
}

// ---------------------------------------------------------------------------
// Halo exchange of a z decomposition.  Plane q of a state is [z][y][x], so
// the values of one population on one z plane are nxy consecutive elements.
// blockIdx.y = 0..19: segments 0..9 carry the ten populations with e_z = +1
// (f then g) from lower's plane nz_l - 2 to upper's plane 0; segments 10..19
// the ten with e_z = -1 from upper's plane 1 to lower's plane nz_l - 1.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int zface_velocity(int j, int sign) {  // j-th velocity (0..4) with e_z = sign
    int k = 0;
    for (int i = 1; i < 19; ++i)
        if (vel_z(i) == sign) {
            if (k == j) return i;
            ++k;
        }
    return -1;
}

template <typename T>
__global__ void k_halo_exchange(long long nxy, T* __restrict__ lower, long long S_l, int nz_l, T* __restrict__ upper,
                                long long S_u) {
    const int seg = blockIdx.y;
    const bool up = seg < 10;
    const int j = up ? seg : seg - 10;
    const int i = zface_velocity(j % 5, up ? 1 : -1);
    const int q = (j < 5 ? 0 : 19) + i;
    const T* src = up ? lower + q * S_l + (long long)(nz_l - 2) * nxy : upper + q * S_u + nxy;
    T* dst = up ? upper + q * S_u : lower + q * S_l + (long long)(nz_l - 1) * nxy;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nxy; k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

cudaError_t launch_halo_exchange(int elem, long long nxy, void* lower, long long S_lower, int nz_lower, void* upper,
                                 long long S_upper, cudaStream_t st) {
    g_last_launches = 1;
    long long nb = (nxy + 255) / 256;
    if (nb > 4096) nb = 4096;
    const dim3 grid((unsigned)nb, 20);
    if (elem == 8)
        k_halo_exchange<double><<<grid, 256, 0, st>>>(nxy, (double*)lower, S_lower, nz_lower, (double*)upper, S_upper);
    else
        k_halo_exchange<float><<<grid, 256, 0, st>>>(nxy, (float*)lower, S_lower, nz_lower, (float*)upper, S_upper);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

Dev32 make_dev32(const Phys& ph) {
    Dev32 c;
    c.omega = (float)ph.omega;
    c.omw = (float)(1.0 - ph.omega);
    c.c_l = (float)ph.c_l;
    c.inv_cl = (float)ph.inv_cl;
    c.inv_cl2 = (float)ph.inv_cl2;
    c.n_ref = (float)ph.n_ref;
    c.g0a = (float)(3.0 - 2.0 * ph.inv_cl2);
    c.g0b = (float)(4.0 - 2.0 * ph.inv_cl2);
    c.eps_ref = ph.eps_ref;
    c.n_ref_d = ph.n_ref;
    c.c_l_d = ph.c_l;
    c.inv_cl_d = ph.inv_cl;
    c.inv_cl2_d = ph.inv_cl2;
    return c;
}

cudaError_t launch_init(int prec, const Geom& g, const Phys& ph, const double* n, const double* eps,
                        const double* beta, const uint8_t* solid, void* A, void* B, cudaStream_t st) {
    g_last_launches = 1;
    if (prec == 0)
        k_init<double><<<blocks_for(g.N, 128), 128, 0, st>>>(n, eps, beta, solid, (double*)A, (double*)B, g, ph);
    else
        k_init<float><<<blocks_for(g.N, 128), 128, 0, st>>>(n, eps, beta, solid, (float*)A, (float*)B, g, ph);
    return cudaGetLastError();
}

static int sm_count() {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    return nsm;
}

// Threads per block of the one-cell-per-thread step kernels: a lattice with
// fewer blocks than SMs (the 1600-cell shock tube) runs 32-thread blocks, so
// that its cells spread over up to 32x more SMs (the per-cell arithmetic,
// FP64 above all, is then the step's latency).  Results do not depend on it.
static int step_block(long long N, int full) { return blocks_for(N, full) < (unsigned)sm_count() ? 32 : full; }

template <int XBC, bool SOLID>
static void launch_step_t(int prec, const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt, bool count,
                          long long step_index, cudaStream_t st) {
    if (prec == 0) {
        const int tb = step_block(g.N, 128);
        if (g.f64df) {
            launch_step_f64_df(g, ph, A, B, cnt, count, step_index, st, tb);
            return;
        }
        // eight lanes per cell while the lanes fit one warp per scheduler
        // (N <= 16 x SMs), unless RLB_F64_SPLIT says otherwise; same values
        if (g.f64split == 1 || (g.f64split < 0 && g.N <= 16ll * sm_count())) {
            k_step_f64_split<XBC, SOLID><<<blocks_for(8 * g.N, 128), 128, 0, st>>>(
                (const double*)A, (double*)B, g, ph, cnt, count ? 1 : 0, step_index);
            return;
        }
        k_step_f64<XBC, SOLID><<<blocks_for(g.N, tb), tb, 0, st>>>((const double*)A, (double*)B, g, ph, cnt,
                                                                    count ? 1 : 0, step_index);
    } else {
        const Dev32 c = make_dev32(ph);
        const int tb = step_block(g.N, 256);
        const unsigned nb = blocks_for(g.N, tb);
        const int cs = count ? 1 : 0;
        const bool idx32 = 38 * g.S < (1ll << 31);
        const bool split32 = !idx32 && 19 * g.S < (1ll << 32);  // unsigned offsets per population set
        if (ph.c_l > 1.0) {
            // lattice speeds above 1: the compensated collision (one launch
            // shape; the TMA-staged and tuning variants use the binary32 one)
            if (idx32)
                k_step_f32<XBC, SOLID, 2, false, int, true><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs,
                                                                                 step_index);
            else if (split32)
                k_step_f32<XBC, SOLID, 2, false, unsigned, true><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt,
                                                                                      cs, step_index);
            else
                k_step_f32<XBC, SOLID, 2, false, long long, true><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c,
                                                                                       cnt, cs, step_index);
            return;
        }
        if (g.tma && launch_step_f32_tma(g, c, (const float*)A, (float*)B, cnt, count, step_index, st) == cudaSuccess)
            return;
        cudaGetLastError();
        switch (g.variant) {
            case 0: k_step_f32<XBC, SOLID, 3, false><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index); break;
            case 1:
                if (idx32)
                    k_step_f32<XBC, SOLID, 3, true, int><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index);
                else if (split32)
                    k_step_f32<XBC, SOLID, 3, true, unsigned><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs,
                                                                               step_index);
                else
                    k_step_f32<XBC, SOLID, 3, true><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index);
                break;
            case 2:
                if (idx32)
                    k_step_f32<XBC, SOLID, 4, false, int><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index);
                else if (split32)
                    k_step_f32<XBC, SOLID, 4, false, unsigned><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs,
                                                                                step_index);
                else
                    k_step_f32<XBC, SOLID, 4, false><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index);
                break;
            case 3: k_step_f32<XBC, SOLID, 4, true><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index); break;
            case 6:
            case 7:
            case 8: {
                // the f populations loaded before the g arithmetic (EARLY), in
                // blocks of 128 threads x 6 or 7 per SM or 64 x 12 (80, 72 and
                // 80 registers)
                const float* a = (const float*)A;
                float* b = (float*)B;
                const int v = g.variant;
                const int t = v == 8 ? (tb < 64 ? tb : 64) : (tb < 128 ? tb : 128);
                const unsigned n = blocks_for(g.N, t);
#define RLB_EARLY_LAUNCH(MB, TBK)                                                                                        \
    do {                                                                                                                 \
        if (idx32) k_step_f32<XBC, SOLID, MB, false, int, false, true, TBK><<<n, t, 0, st>>>(a, b, g, c, cnt, cs, step_index); \
        else if (split32) k_step_f32<XBC, SOLID, MB, false, unsigned, false, true, TBK><<<n, t, 0, st>>>(a, b, g, c, cnt, cs, step_index); \
        else k_step_f32<XBC, SOLID, MB, false, long long, false, true, TBK><<<n, t, 0, st>>>(a, b, g, c, cnt, cs, step_index); \
    } while (0)
                if (v == 6) RLB_EARLY_LAUNCH(6, 128);
                else if (v == 7) RLB_EARLY_LAUNCH(7, 128);
                else RLB_EARLY_LAUNCH(12, 64);
#undef RLB_EARLY_LAUNCH
                break;
            }
            case 4:
            case 5: {
                unsigned grid = (unsigned)sm_count() * (unsigned)(g.pipe_blocks > 0 ? g.pipe_blocks : 3);
                if (grid > nb) grid = nb;
                if (g.variant == 4)
                    k_step_f32_pipe<XBC, SOLID, false><<<grid, 256, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index);
                else
                    k_step_f32_pipe<XBC, SOLID, true><<<grid, 256, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index);
                break;
            }
            default: k_step_f32<XBC, SOLID, 3, true><<<nb, tb, 0, st>>>((const float*)A, (float*)B, g, c, cnt, cs, step_index); break;
        }
    }
}

cudaError_t launch_step(int prec, const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt, bool count,
                        long long step_index, cudaStream_t st) {
    // The solid-marker checks are always compiled in: a lattice without
    // solid cells never matches the marker, and the check costs no memory
    // traffic.
    g_last_launches = 1;
    switch (g.xbc) {
        case XBC_PERIODIC: launch_step_t<XBC_PERIODIC, true>(prec, g, ph, A, B, cnt, count, step_index, st); break;
        case XBC_INFLOW_OUTFLOW:
            launch_step_t<XBC_INFLOW_OUTFLOW, true>(prec, g, ph, A, B, cnt, count, step_index, st);
            break;
        default: launch_step_t<XBC_OUTFLOW_BOTH, true>(prec, g, ph, A, B, cnt, count, step_index, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_macro(int prec, const Geom& g, const Phys& ph, const void* A, double* n, double* eps,
                         double* beta, Counters cnt, cudaStream_t st) {
    g_last_launches = 1;
    if (prec == 0)
        k_macro<double><<<blocks_for(g.N, 128), 128, 0, st>>>((const double*)A, n, eps, beta, g, ph, cnt.macro_bad);
    else
        k_macro<float><<<blocks_for(g.N, 128), 128, 0, st>>>((const float*)A, n, eps, beta, g, ph, cnt.macro_bad);
    return cudaGetLastError();
}

cudaError_t launch_check_solid_planes(const Geom& g, const uint8_t* solid, unsigned long long* flag,
                                      cudaStream_t st) {
    g_last_launches = 1;
    const long long n = 4ll * g.ny * g.nz;
    k_check_solid_planes<<<blocks_for(n, 256), 256, 0, st>>>(g, solid, flag);
    return cudaGetLastError();
}

// Bounds-check count of this translation unit (0 in the release build).
RLB_OOB_TAKE_FN(oob_take_forward)

#ifdef RLB_CHECK_BOUNDS
// The checker itself on one index (no memory is accessed with it): counts a
// violation and returns 0 when the index lies outside [0, n).
static __device__ long long g_rlb_chk_result;
__global__ void k_bounds_selftest(long long i, long long n) { g_rlb_chk_result = RLB_CHK(i, n); }

long long bounds_selftest(long long i, long long n, cudaStream_t s) {
    k_bounds_selftest<<<1, 1, 0, s>>>(i, n);
    long long r = -1;
    if (cudaMemcpyFromSymbolAsync(&r, g_rlb_chk_result, sizeof r, 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    return r;
}
#endif

}  // namespace rlb

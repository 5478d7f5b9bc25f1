// rlb_device.cuh -- device-side building blocks of librlb's kernels.
//
// D3Q19 velocity set of the paper (Fig. 2: one rest velocity, six of speed
// c_l, twelve of speed sqrt(2) c_l; weights 1/3, 1/18, 1/36), written for the
// kernels in opposite pairs: velocity 2p+1 is e_p below and velocity 2p+2 is
// -e_p (p = 0..8), velocity 0 is at rest.  The population planes of a state
// follow this order (documented in include/rlb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rlb_internal.h"

namespace rlb {

// e_p of the nine pairs: +x, +y, +z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1).
__host__ __device__ constexpr int pair_ex(int p) { return (p == 0 || (p >= 3 && p <= 6)) ? 1 : 0; }
__host__ __device__ constexpr int pair_ey(int p) {
    return (p == 1 || p == 3 || p == 7 || p == 8) ? 1 : (p == 4 ? -1 : 0);
}
__host__ __device__ constexpr int pair_ez(int p) {
    return (p == 2 || p == 5 || p == 7) ? 1 : ((p == 6 || p == 8) ? -1 : 0);
}
// Velocity i (0..18) as integers.
__host__ __device__ constexpr int vel_x(int i) { return i == 0 ? 0 : ((i & 1) ? pair_ex((i - 1) >> 1) : -pair_ex((i - 1) >> 1)); }
__host__ __device__ constexpr int vel_y(int i) { return i == 0 ? 0 : ((i & 1) ? pair_ey((i - 1) >> 1) : -pair_ey((i - 1) >> 1)); }
__host__ __device__ constexpr int vel_z(int i) { return i == 0 ? 0 : ((i & 1) ? pair_ez((i - 1) >> 1) : -pair_ez((i - 1) >> 1)); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// Pair weight: 1/18 for the axis pairs (speed c_l), 1/36 for the diagonal pairs.
__host__ __device__ constexpr double pair_w(int p) { return p < 3 ? 1.0 / 18.0 : 1.0 / 36.0; }
constexpr double kW0 = 1.0 / 3.0;

// Solid cells carry a quiet-NaN marker with a payload in every plane; the
// arithmetic of a step never produces these payloads.  A pulled value equal
// to the marker means "the neighbour is solid" (link bounce-back).
constexpr unsigned long long kSolidBits64 = 0x7FF8D0D05011D000ull;
constexpr unsigned int kSolidBits32 = 0x7FC5011Du;

__device__ __forceinline__ bool is_solid(double v) {
    return (unsigned long long)__double_as_longlong(v) == kSolidBits64;
}
__device__ __forceinline__ bool is_solid(float v) { return __float_as_uint(v) == kSolidBits32; }
__device__ __forceinline__ double solid_marker_d() { return __longlong_as_double((long long)kSolidBits64); }
__device__ __forceinline__ float solid_marker_f() { return __uint_as_float(kSolidBits32); }

// Finite and > 0 / finite and >= 0, on the bit pattern (no FP64 pipe work).
__device__ __forceinline__ bool pos_finite(double v) {
    long long b = __double_as_longlong(v);
    return b > 0 && b < 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool nonneg_finite(double v) {
    long long b = __double_as_longlong(v);
    return (b >= 0 && b < 0x7FF0000000000000ll) || b == (long long)0x8000000000000000ull;
}
// 0 <= v < 1 (v is a sum of squares).
__device__ __forceinline__ bool below_one(double v) {
    long long b = __double_as_longlong(v);
    return b >= 0 && b < 0x3FF0000000000000ll;
}
__device__ __forceinline__ bool pos_finite(float v) {
    int b = __float_as_int(v);
    return b > 0 && b < 0x7F800000;
}
__device__ __forceinline__ bool below_one(float v) {
    int b = __float_as_int(v);
    return b >= 0 && b < 0x3F800000;
}

// binary32 <-> binary64 conversions on the integer pipe.  On GB300 the
// hardware conversions issue at the FP64 rate (1/64 of FP32), so the FP32
// deviation kernels move them to the ALU:
//  - f2d: exact for normal numbers, zero, inf and NaN; binary32 subnormals
//    (below 1.2e-38) become zero;
//  - d2f: round to nearest even, exact as the hardware conversion for
//    results in the normal binary32 range; results below it flush to zero,
//    above it become inf;
//  - d2f_seed: truncation, for seeds of Newton iterations only.
__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned sign = u & 0x80000000u;
    const unsigned mhi = (u >> 3) & 0xFFFFFu;
    unsigned hi = sign | ((e + 896u) << 20) | mhi;
    unsigned lo = u << 29;
    if (e == 0u) hi = sign, lo = 0u;
    if (e == 255u) hi = sign | 0x7FF00000u | mhi;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned r = lo & 0x1FFFFFFFu;
    const unsigned up = (r > 0x10000000u) || (r == 0x10000000u && (m & 1u));
    unsigned bits = sign | ((((unsigned)e << 23) + m) + up);
    if (e <= 0) bits = sign;
    if (e >= 255) bits = sign | 0x7F800000u;
    if (((hi >> 20) & 0x7FFu) == 0x7FFu) bits = sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
    return __uint_as_float(bits);
}
__device__ __forceinline__ float d2f_seed(double d) {
    const unsigned hi = (unsigned)__double2hiint(d);
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;
    unsigned bits = (hi & 0x80000000u) | (((unsigned)e << 23) + ((hi & 0xFFFFFu) << 3));
    if (e <= 0) bits = hi & 0x80000000u;
    if (e >= 255) bits = (hi & 0x80000000u) | 0x7F800000u;
    return __uint_as_float(bits);
}

// Binary64 seeds of 1/sqrt(x) and 1/x for Newton iterations, taken from the
// binary32 instructions for a positive normal binary64 x of any exponent:
// x = m 2^k with m in [1, 4) (k even; for 1/sqrt) or in [1, 2) (for 1/x), the
// binary32 seed is formed for m, and the result is multiplied by 2^(-k/2) or
// 2^-k.  Both scalings are exact and are integer operations on the exponent
// field, so no FP64 instruction is added.  Zero, subnormal, negative,
// infinite and NaN arguments (states the callers flag as unphysical) take the
// unscaled binary32 seed.
__device__ __forceinline__ double scale_pow2(double x, int k) {  // x 2^k, x and the result normal
    return __hiloint2double(__double2hiint(x) + k * (1 << 20), __double2loint(x));
}
__device__ __forceinline__ int seed_shift(double x, int emax) {
    const int hi = __double2hiint(x);
    const int e = (hi >> 20) & 0x7FF;
    return (hi >= 0 && e >= 1 && e <= emax) ? e - 1023 : 0;
}
// y ~ 1/sqrt(x), and y/2
__device__ __forceinline__ void rsqrt_seed(double x, double& y, double& half_y) {
    const int k = seed_shift(x, 0x7FE) & ~1;
    const float sf = rsqrtf(d2f_seed(scale_pow2(x, -k)));
    const double s = f2d(sf), hs = f2d(0.5f * sf);
    // k = 0 also for the special arguments, whose seed must not be rescaled
    y = k == 0 ? s : scale_pow2(s, -(k / 2));
    half_y = k == 0 ? hs : scale_pow2(s, -(k / 2) - 1);
}
__device__ __forceinline__ double rcp_seed(double x) {
    const int k = seed_shift(x, 0x7FC);
    return scale_pow2(f2d(__frcp_rn(d2f_seed(scale_pow2(x, -k)))), -k);
}

// Offsets (in cells) from cell (x, y, z) to the source x - e of a pull, for
// the components -1 / 0 / +1 of e, with periodic wrap.  For a non-periodic x
// the interior cells never wrap, so the same formula serves every case.
struct PullOffsets {
    int xm, xp, ym, yp, zm, zp;  // source at x-1 / x+1, y-1 / y+1, z-1 / z+1

    PullOffsets() = default;
    __device__ __forceinline__ PullOffsets(const Geom& g, int x, int y, int z) {
        xm = (x == 0) ? g.nx - 1 : -1;
        xp = (x == g.nx - 1) ? -(g.nx - 1) : 1;
        ym = (y == 0) ? (g.ny - 1) * g.nx : -g.nx;
        yp = (y == g.ny - 1) ? -(g.ny - 1) * g.nx : g.nx;
        zm = (z == 0) ? (g.nz - 1) * g.nxy : -g.nxy;
        zp = (z == g.nz - 1) ? -(g.nz - 1) * g.nxy : g.nxy;
    }
    // Offset of the source cell x - e_i of velocity i.
    __device__ __forceinline__ int src(int i) const {
        const int ex = vel_x(i), ey = vel_y(i), ez = vel_z(i);
        return (ex > 0 ? xm : (ex < 0 ? xp : 0)) + (ey > 0 ? ym : (ey < 0 ? yp : 0)) +
               (ez > 0 ? zm : (ez < 0 ? zp : 0));
    }
    // Offset of the destination x + e_i (the cell that pulls velocity i from x).
    __device__ __forceinline__ int dst(int i) const {
        const int ex = vel_x(i), ey = vel_y(i), ez = vel_z(i);
        return (ex > 0 ? xp : (ex < 0 ? xm : 0)) + (ey > 0 ? yp : (ey < 0 ? ym : 0)) +
               (ez > 0 ? zp : (ez < 0 ? zm : 0));
    }
};

// ---------------------------------------------------------------------------
// Moments in pair form: S = sum f, E = sum g, M = c_l sum g e.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void moments_pairs(const T* f, const T* g, T& sf, T& e, T& mx, T& my, T& mz) {
    T s = f[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) s += f[i];
    T d[9];
    T es = g[0];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        es += g[2 * p + 1] + g[2 * p + 2];
        d[p] = g[2 * p + 1] - g[2 * p + 2];
    }
    sf = s;
    e = es;
    mx = d[0] + d[3] + d[4] + d[5] + d[6];
    my = d[1] + d[3] - d[4] + d[7] + d[8];
    mz = d[2] + d[5] - d[6] + d[7] - d[8];
}

// Optional bounds checking (a debug build, -DRLB_CHECK_BOUNDS): every
// element index into a state buffer (38 S elements) in the step, adjoint and
// equation-of-state kernels goes through RLB_CHK; an index outside the buffer
// is counted (per translation unit) and replaced by an in-range one, so the
// access itself stays inside the buffer.  The release build compiles the
// indices unchanged.  RLB_CHK_OFF checks base + off and returns off;
// RLB_CHK_PTR(p, e, n) is the pointer p + e with e checked.
#ifdef RLB_CHECK_BOUNDS
static __device__ unsigned long long g_rlb_oob_count;
template <typename I>
__device__ __forceinline__ I rlb_chk(I i, long long n) {
    if (i < 0 || (long long)i >= n) {
        atomicAdd(&g_rlb_oob_count, 1ull);
        return (I)0;
    }
    return i;
}
template <typename I>
__device__ __forceinline__ I rlb_chk_off(I off, long long base, long long n) {
    if (base + (long long)off < 0 || base + (long long)off >= n) {
        atomicAdd(&g_rlb_oob_count, 1ull);
        return (I)(-base);
    }
    return off;
}
#define RLB_CHK(i, n) rlb_chk((i), (long long)(n))
#define RLB_CHK_OFF(off, base, n) rlb_chk_off((off), (long long)(base), (long long)(n))
#define RLB_CHK_PTR(p, e, n) ((p) + rlb_chk((e), (long long)(n)))
// Host side, per translation unit: read and clear the count.
#define RLB_OOB_TAKE_FN(name)                                                              \
    unsigned long long name() {                                                            \
        unsigned long long v = 0, z = 0;                                                   \
        if (cudaMemcpyFromSymbol(&v, g_rlb_oob_count, sizeof v) != cudaSuccess) return ~0ull; \
        cudaMemcpyToSymbol(g_rlb_oob_count, &z, sizeof z);                                 \
        return v;                                                                          \
    }
#else
#define RLB_CHK(i, n) (i)
#define RLB_CHK_OFF(off, base, n) (off)
// Expands to the unbracketed tokens p + e, so pointer arithmetic groups as written.
#define RLB_CHK_PTR(p, e, n) p + e
#define RLB_OOB_TAKE_FN(name) \
    unsigned long long name() { return 0; }
#endif

// Cell coordinates by multiply-high division with host-computed magic
// numbers (division by an invariant integer, Granlund and Montgomery 1994).
__device__ __forceinline__ unsigned fast_div(unsigned n, const FastDiv& d) {
    return (__umulhi(n, d.mul) + n) >> d.shift;
}
__device__ __forceinline__ void cell_coords(const Geom& g, int idx, int& x, int& y, int& z) {
    const int yz = (int)fast_div((unsigned)idx, g.div_nx);
    x = idx - yz * g.nx;
    z = (int)fast_div((unsigned)yz, g.div_ny);
    y = yz - z * g.ny;
}

// Warp-aggregated statistics: each warp adds its counts to one of
// kCounterSlots slots, so no address sees much contention; the smallest
// flagged update id of the warp goes to first_bad with one atomicMin, and
// only when it beats the value already there.
__device__ __forceinline__ void count_flags(const Counters& c, bool unphys, bool nonpos, unsigned long long bad_id) {
    const unsigned act = __activemask();
    const unsigned mu = __ballot_sync(act, unphys);
    const unsigned mp = __ballot_sync(act, nonpos);
    if ((mu | mp) == 0u) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    if (mu) {
        unsigned long long id = unphys ? bad_id : ~0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(act, id, off);
            // lanes outside 'act' return undefined values to shuffles; only
            // take values from active lanes
            const int src = lane ^ off;
            if (((act >> src) & 1u) && o < id) id = o;
        }
        if (lane == leader && id < *(volatile unsigned long long*)c.first_bad) atomicMin(c.first_bad, id);
    }
    if (lane == leader) {
        const unsigned slot = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (kCounterSlots - 1);
        if (mu) atomicAdd(c.slots + slot, (unsigned long long)__popc(mu));
        if (mp) atomicAdd(c.slots + kCounterSlots + slot, (unsigned long long)__popc(mp));
    }
}

// Positivity of the equilibria (the condition c_i . u < c_l^2/3 stated for the
// tachyon runs, with the matching g-bracket of Eq. equil2as), decided in
// binary32 on beta rounded to binary32, every operation rounded on its own
// (no contraction):  flag when, for some direction pair with q = e_p.beta,
//   c_l - 3|q| <= 0   or   (1 - 3 b2) + |q| (6|q| - 4 c_l) <= 0,
// with b2 = (bx*bx + by*by) + bz*bz.
__device__ __forceinline__ bool nonpositive_eq(float bx, float by, float bz, float cl) {
    const float q[9] = {bx, by, bz, __fadd_rn(bx, by), __fsub_rn(bx, by), __fadd_rn(bx, bz),
                        __fsub_rn(bx, bz), __fadd_rn(by, bz), __fsub_rn(by, bz)};
    const float b2 = __fadd_rn(__fadd_rn(__fmul_rn(bx, bx), __fmul_rn(by, by)), __fmul_rn(bz, bz));
    const float c0 = __fsub_rn(1.0f, __fmul_rn(3.0f, b2));
    const float four_cl = __fmul_rn(4.0f, cl);
    bool flag = false;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const float aq = fabsf(q[p]);
        const float fb = __fsub_rn(cl, __fmul_rn(3.0f, aq));
        const float gb = __fadd_rn(c0, __fmul_rn(aq, __fsub_rn(__fmul_rn(6.0f, aq), four_cl)));
        flag |= (fb <= 0.0f) | (gb <= 0.0f);
    }
    return flag;
}

}  // namespace rlb

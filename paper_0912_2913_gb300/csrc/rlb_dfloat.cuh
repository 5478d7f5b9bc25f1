// rlb_dfloat.cuh -- compensated arithmetic on pairs of binary32 values.
//
// A value is carried as x = h + l, two binary32 numbers with |l| no larger
// than half an ulp of h (a "double-float", about 48 significant bits).  The
// operations are built from the error-free transformations of Dekker (1971,
// "A floating-point technique for extending the available precision") and
// Knuth (TAOCP vol. 2, section 4.2.2):
//   two_sum(a, b):      s + e = a + b exactly, s = fl(a + b)   (6 operations)
//   fast_two_sum(a, b): the same when |a| >= |b| or a = 0     (3 operations)
//   two_prod(a, b):     p + e = a * b exactly, p = fl(a * b), e by one fused
//                       multiply-add                           (2 operations)
// Every operation below is an explicitly rounded intrinsic, so the compiler
// can neither contract nor reorder them.  These run on the FP32 pipe, which
// on GB300 issues about 70x more operations per clock than the FP64 pipe.
#pragma once

#include <cuda_runtime.h>

#include "rlb_device.cuh"

namespace rlb {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.h, -x.l}; }

// x + y with both parts carried (the "accurate" double-float sum).
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    dfl s = two_sum(x.h, y.h);
    const dfl t = two_sum(x.l, y.l);
    s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    dfl p = two_prod(x.h, y.h);
    const float e = __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.l, p.l));
    return fast_two_sum(p.h, e);
}

// Split of a binary64 value: h = x rounded to binary32, l = (x - h) rounded
// (the conversions on the integer pipe, one FP64 subtraction).
__device__ __forceinline__ dfl df_of(double x) {
    const float h = d2f(x);
    return {h, d2f(x - f2d(h))};
}

// Split of a binary64 value into a pair on the integer pipe (no FP64
// instruction): h = x rounded to binary32 (d2f), and the remainder x - h,
// exact in binary64 as the signed integer R of the 29 mantissa bits below
// h's precision (minus 2^29 when h was rounded up) times 2^(E - 52), rounded
// once more to binary32 (I2F), so h + l carries 48 of x's 53 significant
// bits.  Valid while both parts are binary32 normals: |x| between about
// 2^-100 and 2^127; zero stays zero.
__device__ __forceinline__ dfl df_split(double x) {
    const float h = d2f(x);
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FFu);  // biased exponent of x
    const int r29 = (int)(lo & 0x1FFFFFFFu);
    const int up = (r29 > 0x10000000) || (r29 == 0x10000000 && ((lo >> 29) & 1u));
    const int R = r29 - (up << 29);           // x - h = +-R 2^(e - 1075)
    const float fr = __int2float_rn(R);
    // scale by 2^(e - 1075) on the exponent field; the sign of x
    const unsigned b = __float_as_uint(fr);
    const unsigned scaled = (b + (unsigned)((e - 1075) * (1 << 23))) ^ (hi & 0x80000000u);
    const int eb = (int)((b >> 23) & 0xFFu) + (e - 1075);  // biased exponent of l
    const float l = (R == 0 || eb <= 0) ? 0.0f : __uint_as_float(scaled);
    return {h, l};
}

// h + l in binary64 (exact for a normalised pair).
__device__ __forceinline__ double df_dbl(dfl x) { return f2d(x.h) + f2d(x.l); }

// The binary32 value nearest to x - b for a pair x and a binary32 b: the
// difference of the leading parts is formed without error, then the small
// parts are added and the result rounded once.
__device__ __forceinline__ float df_sub_round(dfl x, float b) {
    const dfl t = two_sum(x.h, -b);
    return __fadd_rn(t.h, __fadd_rn(t.l, x.l));
}

// Compensated running sum (the rounding error of every addition is collected
// in a second binary32 and added back at the end).
struct CSum {
    float s, c;
    __device__ __forceinline__ explicit CSum(float first) : s(first), c(0.0f) {}
    __device__ __forceinline__ void add(float v) {
        const dfl t = two_sum(s, v);
        s = t.h;
        c = __fadd_rn(c, t.l);
    }
    // adds a pair h + l (its small part goes straight to the compensation)
    __device__ __forceinline__ void add(dfl v) {
        add(v.h);
        c = __fadd_rn(c, v.l);
    }
    __device__ __forceinline__ dfl result() const { return fast_two_sum(s, c); }
};

}  // namespace rlb

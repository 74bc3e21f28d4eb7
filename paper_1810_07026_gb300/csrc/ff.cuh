// Double-float ("ff") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, which carries about 48 significant
// bits.  On GB300 the FP32 pipe issues 64 times the FP64 pipe's operations per
// clock, so a handful of FP32 operations per FP64-class operation still comes
// out far ahead.  The building blocks are the classical error-free
// transformations -- Knuth's TwoSum, Dekker's FastTwoSum (|a| >= |b|) and the
// FMA form of TwoProduct -- and the short double-word addition and
// multiplication made from them (as in the double-double literature, e.g.
// Hida, Li and Bailey's QD library and Joldes, Muller and Popescu, ACM TOMS
// 2017), written here from those definitions.  Addition is accurate to a few
// units of 2^-48 of the larger operand, multiplication to a few units of 2^-48
// relative; the LJ kernel's parity against the FP64 oracle is the test.
#pragma once

#include <cuda_runtime.h>

namespace airebo {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }

// exact a + b = s + e
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
// exact a + b = s + e when |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}
// exact a * b = p + e
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    float e = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ ff ff_sqr(ff a) {
    ff p = two_prod(a.hi, a.hi);
    float e = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, e);
}
// 1/a for a > 0: the FP32 reciprocal y, then one Newton step on the residual
// 1 - a y formed in double-float (the error squares: about 2^-46)
__device__ __forceinline__ ff ff_rcp(ff a) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    ff p = ff_mul_f(a, y);
    ff r = ff_add_f(ff_neg(p), 1.0f);          // 1 - a y, small
    return fast_two_sum(y, __fmul_rn(y, r.hi));
}
// 1/sqrt(a) for a > 0: the FP32 estimate y, then one Newton step
// y + y (1 - a y^2) / 2 with the residual in double-float
__device__ __forceinline__ ff ff_rsqrt(ff a) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    ff p = ff_mul_f(ff_mul_f(a, y), y);
    ff r = ff_add_f(ff_neg(p), 1.0f);          // 1 - a y^2, small
    return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), r.hi));
}

__device__ __forceinline__ ff ff_from_double(double x) {
    float h = __double2float_rn(x);
    return ff{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Fixed-point force accumulation: v * 2^FIX_BITS as a signed 64-bit integer.
// hi and lo are each scaled by 2^40 and rounded to an integer, so each added
// value carries an error of at most 2^-40 (about 1e-12 eV/A); integer sums are
// exact and independent of the order of the atomic additions.
constexpr int FIX_BITS = 40;
constexpr float FIX_SCALE = 1099511627776.0f;         // 2^40
constexpr double FIX_INV = 1.0 / 1099511627776.0;      // 2^-40
constexpr float FIX_LIMIT = 1.0e6f;                    // |v| below 2^20: eight such terms stay below 2^63

// v * 2^FIX_BITS rounded to an integer (half away from zero), from the bits
// of v with integer operations only: the float-to-64-bit-integer conversion
// instruction shares the narrow FP64 pipe on this GPU.  For |v| < 2^22.
__device__ __forceinline__ long long f2fix(float v) {
    unsigned b = __float_as_uint(v);
    int e = (int)((b >> 23) & 0xffu);
    long long m = (long long)((b & 0x7fffffu) | 0x800000u);        // zero: m * 2^-110 rounds to 0
    int sh = e - (127 + 23 - FIX_BITS);                              // v * 2^40 = m * 2^sh
    long long up = m << (sh > 0 ? sh : 0);
    int k = -sh;
    k = k < 1 ? 1 : (k > 63 ? 63 : k);
    long long dn = (m + (1ll << (k - 1))) >> k;
    long long r = sh >= 0 ? up : dn;
    return (b >> 31) ? -r : r;
}

// hi + lo in fixed point.  lo * 2^40 is below 2^22 in magnitude unless the
// value is beyond ~64 eV/A; then adding 1.5 * 2^23 rounds it to an integer in
// the float's significand (the usual shift trick), two operations.
__device__ __forceinline__ long long ff_to_fixed(ff a) {
    float t = __fmul_rn(a.lo, FIX_SCALE);
    long long lo;
    if (fabsf(t) < 4194304.0f) lo = (long long)(__float_as_int(__fadd_rn(t, 12582912.0f)) - 0x4B400000);
    else lo = f2fix(a.lo);
    return f2fix(a.hi) + lo;
}

}  // namespace airebo

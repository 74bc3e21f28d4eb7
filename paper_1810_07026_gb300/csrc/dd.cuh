// Double-float value type for the torsion term of AIREBO_DF64.
//
// A dd is the unevaluated sum hi + lo of two FP32 numbers (about 48
// significant bits), with the double-float operations of ff.cuh behind the
// usual operators, so that the generic term code (terms.cuh) runs on the FP32
// pipe at FP64-class accuracy.  GB300 issues 64 FP32 operations per FP64
// operation; a double-float operation takes 2 to 20 of them.
//
// Accuracy per operation, measured on the device by airebo_dd_check over 4M
// operands (largest errors):
// * addition: 8.7e-15 of |a| + |b| (the short double-word sum, with no
//   cancellation-free guarantee);
// * relative: multiplication 1.3e-14, division 3.7e-14, reciprocal 2.5e-14,
//   reciprocal square root 3.9e-14;
// * absolute: sin and cos of pi t 8e-15.  They are written here from their
//   Taylor series after reduction to a quadrant.
// The parity tests hold the DF64 path to the FP64 tolerances.
//
// On the host the same operations run through double (parameter set-up only).
#pragma once

#include "ff.cuh"

namespace airebo {

#ifdef __CUDACC__
#define DDH __host__ __device__ __forceinline__
#define DDH_CALL static __host__ __device__ __noinline__     // a long function: called, not inlined
#else
#define DDH inline
#define DDH_CALL static inline
#endif

struct dd {
    float hi, lo;
    dd() = default;
    constexpr DDH dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    constexpr DDH dd(float x) : hi(x), lo(0.0f) {}
    constexpr DDH dd(int x) : dd((double)x) {}
    static constexpr DDH dd raw(float h, float l) { return dd(h, l, 0); }
    constexpr DDH explicit operator double() const { return (double)hi + (double)lo; }
    constexpr DDH explicit operator float() const { return hi + lo; }
    constexpr DDH explicit operator int() const { return (int)hi; }     // after floor (lo = 0)

private:
    constexpr DDH dd(float h, float l, int) : hi(h), lo(l) {}
};

#ifdef __CUDA_ARCH__
__device__ __forceinline__ ff to_ff(dd a) { return ff{a.hi, a.lo}; }
__device__ __forceinline__ dd of_ff(ff a) { return dd::raw(a.hi, a.lo); }
#endif

// ------------------------------------------------------------------ arithmetic
DDH dd operator-(dd a) { return dd::raw(-a.hi, -a.lo); }
DDH dd operator+(dd a, dd b) {
#ifdef __CUDA_ARCH__
    return of_ff(ff_add(to_ff(a), to_ff(b)));
#else
    return dd((double)a + (double)b);
#endif
}
DDH dd operator-(dd a, dd b) { return a + (-b); }
DDH dd operator*(dd a, dd b) {
#ifdef __CUDA_ARCH__
    return of_ff(ff_mul(to_ff(a), to_ff(b)));
#else
    return dd((double)a * (double)b);
#endif
}
// a / b: the FP32 quotient q1, then q2 from the double-float remainder a - b q1
DDH dd operator/(dd a, dd b) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b.hi));
    float q1 = __fmul_rn(a.hi, r);
    ff rem = ff_sub(to_ff(a), ff_mul_f(to_ff(b), q1));
    float q2 = __fmul_rn(rem.hi, r);
    return of_ff(fast_two_sum(q1, q2));
#else
    return dd((double)a / (double)b);
#endif
}
DDH dd& operator+=(dd& a, dd b) { a = a + b; return a; }
DDH dd& operator-=(dd& a, dd b) { a = a - b; return a; }
DDH dd& operator*=(dd& a, dd b) { a = a * b; return a; }
DDH dd& operator/=(dd& a, dd b) { a = a / b; return a; }

// comparisons (hi first; NaN compares false)
DDH bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
DDH bool operator>(dd a, dd b) { return b < a; }
DDH bool operator<=(dd a, dd b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
DDH bool operator>=(dd a, dd b) { return b <= a; }
DDH bool operator==(dd a, dd b) { return a.hi == b.hi && a.lo == b.lo; }
DDH bool operator!=(dd a, dd b) { return !(a == b); }

// ------------------------------------------------------------------ the term code's helpers
// order-preserving integer key of an FP32 value (NaN beyond the infinities)
DDH int okey32(float x) {
#ifdef __CUDA_ARCH__
    int b = __float_as_int(x);
#else
    int b;
    memcpy(&b, &x, sizeof(b));
#endif
    return b < 0 ? -(b & 0x7fffffff) : b;
}
DDH bool lt_(dd a, dd b) {
    int ka = okey32(a.hi), kb = okey32(b.hi);
    return ka < kb || (ka == kb && a.lo < b.lo);
}
DDH bool lt_nonneg(dd a, dd b) { return lt_(a, b); }
DDH bool is_zero(dd t) { return t.hi == 0.0f; }

DDH dd rsqrt_(dd a) {
#ifdef __CUDA_ARCH__
    return of_ff(ff_rsqrt(to_ff(a)));
#else
    return dd(1.0 / std::sqrt((double)a));
#endif
}
DDH dd rcp_(dd a) {
#ifdef __CUDA_ARCH__
    return of_ff(ff_rcp(to_ff(a)));
#else
    return dd(1.0 / (double)a);
#endif
}


// sin(pi t) and cos(pi t): t = n/2 + u with |u| <= 1/4 (exact), then the
// Taylor series of sin and cos of pi u to the 17th and 16th power, and the
// quadrant n.
DDH_CALL void sincospi_(dd t, dd* s, dd* c) {
#ifdef __CUDA_ARCH__
    float nf = rintf(__fmul_rn(t.hi, 2.0f));
    dd u = t - dd(__fmul_rn(nf, 0.5f));
    constexpr double PI = 3.14159265358979323846264;
    dd x = u * dd(PI);
    dd x2 = x * x;
    // sin x = x (1 - x^2/(2 3) (1 - x^2/(4 5) (1 - ...))), cos x = 1 - x^2/(1 2) (1 - x^2/(3 4) (...))
    dd ps = dd(1.0f), pc = dd(1.0f);
#pragma unroll
    for (int m = 8; m >= 1; m--) {
        ps = dd(1.0f) - x2 * ps * dd(1.0 / ((2 * m) * (2 * m + 1)));
        pc = dd(1.0f) - x2 * pc * dd(1.0 / ((2 * m - 1) * (2 * m)));
    }
    dd sn = x * ps, cn = pc;
    int q = ((int)nf) & 3;
    if (q == 0) { *s = sn; *c = cn; }
    else if (q == 1) { *s = cn; *c = -sn; }
    else if (q == 2) { *s = -sn; *c = -cn; }
    else { *s = -cn; *c = sn; }
#else
    double v = (double)t;
    *s = dd(std::sin(M_PI * v)); *c = dd(std::cos(M_PI * v));
#endif
}

}  // namespace airebo

// An FP32 value with a rigorous bound on its error, for the b* screen of the
// FP64 path.
//
// An ef holds a value v and a bound e >= 0 on |v - x|, where x is the result
// of the same formula in exact arithmetic on the FP64 inputs and the FP64
// parameter set.  Inputs enter with their FP64-to-FP32 rounding error,
// parameters and spline coefficients with theirs (computed exactly on the
// host), and every operation adds its own rounding error, with the bound
// itself computed in round-toward-+infinity:
//   a + b : e_a + e_b + |r|, r the exact rounding error of the sum (TwoSum)
//   a * b : |a| e_b + |b| e_a + e_a e_b + |r|, r = fma(a, b, -ab) exactly
//           (plus 2^-126 for a product below 2^-100, where r may underflow)
//   f(a)  : sup |f'| over [a - e_a, a + e_a] times e_a, plus the function's
//           own error (4 ulp for rsqrtf, expf, cospif and the approximate
//           reciprocal, twice their documented maxima)
// so exact operations on exact values keep a zero bound (sums of bond
// weights that are exactly 1 give an exact coordination, which then sits on
// a spline knot exactly).  The values use the round-to-nearest intrinsics,
// which the compiler does not contract into fused multiply-adds behind the
// error terms' back.
//
// Branches: the switch S(t) is Lipschitz with constant pi/2 across its
// branch points, the clamps with 1, |x| with 1, so their bounds need no
// care.  A spline whose argument interval [v - e, v + e] reaches across an
// interior knot (where the FP64 evaluation may take the other piece) returns
// an infinite bound; so does a reciprocal or square root whose argument
// interval reaches zero.  An infinite bound sends the pair to the FP64 pass.
#pragma once

#include <cfloat>

namespace airebo {

struct ef {
    float v, e;
    ef() = default;
    constexpr HD ef(float x) : v(x), e(0.0f) {}
    constexpr HD ef(int x) : v((float)x), e(0.0f) {}
    // a double rounded to FP32, with its rounding error (rounded up)
    constexpr HD ef(double x) : v((float)x), e(err_of(x)) {}
    static constexpr HD ef raw(float v, float e) { return ef(v, e, 0); }
    static constexpr HD float err_of(double x) {
        double d = x - (double)(float)x;
        return (float)((d < 0 ? -d : d) * (1.0 + 2.384185791015625e-07));   // (1 + 2^-22) covers the cast
    }

private:
    constexpr HD ef(float v_, float e_, int) : v(v_), e(e_) {}
};

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float ru_add(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float ru_mul(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float ru_fma(float a, float b, float c) { return __fmaf_ru(a, b, c); }
__device__ __forceinline__ float rd_sub(float a, float b) { return __fsub_rd(a, b); }
#else
inline float ru_add(float a, float b) { return (a + b) * 1.0000002f; }
inline float ru_mul(float a, float b) { return (a * b) * 1.0000002f; }
inline float ru_fma(float a, float b, float c) { return (a * b + c) * 1.0000002f; }
inline float rd_sub(float a, float b) { return (a - b) - 1.2e-7f * (a > b ? a - b : b - a); }
#endif

constexpr float EF_U = 5.9604645e-08f;        // 2^-24
constexpr float EF_TINY = 1.4e-45f;           // the smallest subnormal
constexpr float EF_FN = 4.76837158e-07f;      // 2^-21: four ulp, the bound used for the FP32 functions
constexpr float EF_INF = __builtin_huge_valf();

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float rn_add(float a, float b) { return a + b; }
inline float rn_sub(float a, float b) { return a - b; }
inline float rn_mul(float a, float b) { return a * b; }
inline float rn_fma(float a, float b, float c) { return std::fma(a, b, c); }
#endif

// |v| u + 2^-149: a bound on the rounding error of a result v
HD float ef_round(float v) { return ru_fma(fabsf(v), EF_U, EF_TINY); }

HD ef operator-(ef a) { return ef::raw(-a.v, a.e); }
HD ef operator+(ef a, ef b) {
    float v = rn_add(a.v, b.v);
    float bb = rn_sub(v, a.v);                                       // TwoSum (Knuth)
    float r = rn_add(rn_sub(a.v, rn_sub(v, bb)), rn_sub(b.v, bb));
    return ef::raw(v, ru_add(ru_add(a.e, b.e), fabsf(r)));
}
HD ef operator-(ef a, ef b) { return a + (-b); }
HD ef operator*(ef a, ef b) {
    float v = rn_mul(a.v, b.v);
    float r = rn_fma(a.v, b.v, -v);                                  // exact unless the product underflows
    float e = ru_mul(fabsf(a.v), b.e);
    e = ru_fma(fabsf(b.v), a.e, e);
    e = ru_fma(a.e, b.e, e);
    e = ru_add(e, fabsf(r));
    if (fabsf(v) < 1e-30f) e = ru_add(e, 1.2e-38f);
    return ef::raw(v, e);
}
HD ef& operator+=(ef& a, ef b) { a = a + b; return a; }
HD ef& operator-=(ef& a, ef b) { a = a - b; return a; }
HD ef& operator*=(ef& a, ef b) { a = a * b; return a; }

// branch decisions of the generic code compare the values
HD bool lt_(ef a, ef b) { return a.v < b.v; }
// an exact zero only (the knot shortcuts of the splines then see exact knots)
HD bool is_zero(ef t) { return t.v == 0.0f && t.e == 0.0f; }

// 1/sqrt(a) for a > 0: sup |f'| on [lo, hi] is (1/2) lo^-3/2
HD ef rsqrt_(ef a) {
    float lo = rd_sub(a.v, a.e);
    float v = rsqrt_(a.v);
    if (!(lo > 0.0f)) return ef::raw(v, EF_INF);
    float rl = ru_mul(rsqrt_(lo), 1.0000005f);              // an upper bound of lo^-1/2
    float d = ru_mul(ru_mul(ru_mul(rl, rl), rl), 0.5f);
    return ef::raw(v, ru_fma(d, a.e, ru_mul(fabsf(v), EF_FN)));
}
// 1/a for a > 0: sup |f'| = lo^-2
HD ef rcp_(ef a) {
    float lo = rd_sub(a.v, a.e);
    float v = rcp_(a.v);
    if (!(lo > 0.0f)) return ef::raw(v, EF_INF);
    float rl = ru_mul(rcp_(lo), 1.0000005f);
    return ef::raw(v, ru_fma(ru_mul(rl, rl), a.e, ru_mul(fabsf(v), EF_FN)));
}
// e^a: |e^X - e^v| <= e^v (e^|X - v| - 1) <= e^v e_a (1 + e_a) for e_a <= 1/2
HD ef exp_(ef a) {
    float v = exp_(a.v);
    if (!(a.e <= 0.5f)) return ef::raw(v, EF_INF);
    float vu = ru_mul(v, 1.0000005f);
    float e = ru_mul(ru_mul(vu, a.e), ru_add(1.0f, a.e));
    return ef::raw(v, ru_fma(fabsf(v), EF_FN, e));
}

// ------------------------------------------------------------------ specialisations of the term code
// S(t): exact where the whole interval lies in a flat part, else Lipschitz pi/2
template <> HD ef Sw<ef>(ef t, ef& dS) {
    dS = ef(0.0f);
    if (ru_add(t.v, t.e) <= 0.0f) return ef(1.0f);
    if (rd_sub(t.v, t.e) >= 1.0f) return ef(0.0f);
    float tc = fminf(fmaxf(t.v, 0.0f), 1.0f);
    float s, c;
    sincospi_(tc, &s, &c);
    float v = 0.5f * (1.0f + c);
    // cospif (4 ulp, at most 2^-21 absolute), the addition (2^-23) and the
    // halving (exact): below 4e-7 absolute
    return ef::raw(v, ru_fma(1.5707964f, t.e, 4.0e-07f));
}

// clamp: Lipschitz 1 (the bound carries over, plus the end's own error)
template <> HD ef clamp_<ef>(ef x, ef lo, ef hi, bool& cl) {
    cl = false;
    if (x.v < lo.v) { cl = true; return ef::raw(lo.v, ru_add(x.e, lo.e)); }
    if (x.v > hi.v) { cl = true; return ef::raw(hi.v, ru_add(x.e, hi.e)); }
    if (!(x.v == x.v)) { cl = true; return ef::raw(lo.v, EF_INF); }
    return ef::raw(x.v, ru_add(x.e, ru_add(lo.e, hi.e)));    // the true clamp may still bite within the ends' errors
}

// does [x - e, x + e] reach the knot k (with its own error)?  Exact values
// never do: the FP64 evaluation then compares the very same numbers.
HD bool ef_reaches(ef x, ef k) {
    if (x.e == 0.0f && k.e == 0.0f) return false;
    return fabsf(x.v - k.v) <= ru_add(ru_add(x.e, k.e), ef_round(x.v - k.v));
}

template <> HD ef quintic<ef, false>(const Quintic<ef>& q, ef x, ef& dfdx) {
    bool cl;
    dfdx = ef(0.0f);
    x = clamp_<ef>(x, q.k[0], q.k[q.n], cl);
    int m = 0;
    while (m + 1 < q.n && x.v > q.k[m + 1].v) m++;
    bool straddle = (m > 0 && ef_reaches(x, q.k[m])) || (m + 1 < q.n && ef_reaches(x, q.k[m + 1]));
    ef t = (x - q.k[m]) * q.invh[m];
    const ef* a = q.a[m];
    ef f = a[5];
    f = f * t + a[4];
    f = f * t + a[3];
    f = f * t + a[2];
    f = f * t + a[1];
    f = f * t + a[0];
    if (straddle) f.e = EF_INF;
    return f;
}

// an interior integer knot k (lo < k < hi) within reach of x
HD bool ef_reaches_int(ef x, int lo, int hi) {
    float k = rintf(x.v);
    return k > (float)lo && k < (float)hi && ef_reaches(x, ef(k));
}

template <> HD ef bicubic<ef, false>(const ef* tab, ef x, ef y, ef& fx, ef& fy) {
    bool cx, cy;
    fx = ef(0.0f);
    fy = ef(0.0f);
    x = clamp_<ef>(x, ef(0.0f), ef(4.0f), cx);
    y = clamp_<ef>(y, ef(0.0f), ef(4.0f), cy);
    bool straddle = ef_reaches_int(x, 0, 4) || ef_reaches_int(y, 0, 4);
    int ix = clamp_cell((int)floorf(x.v), 3);
    int iy = clamp_cell((int)floorf(y.v), 3);
    ef tx = x - ef(ix), ty = y - ef(iy);
    const ef* a = tab + (ix * 4 + iy) * 16;
    ef f(0.0f);
    if (is_zero(tx) && is_zero(ty)) {
        f = a[0];
    } else {
        for (int p = 3; p >= 0; p--) {
            const ef* c = a + p * 4;
            ef cp = ((c[3] * ty + c[2]) * ty + c[1]) * ty + c[0];
            f = f * tx + cp;
        }
    }
    if (straddle) f.e = EF_INF;
    return f;
}

// the cell of a tricubic; an argument within reach of an interior knot
// poisons tx (the value then carries an infinite bound)
template <> HD int tri_cell_index<ef>(ef& x, ef& y, ef& z, bool& clx, bool& cly, bool& clz, ef& tx, ef& ty, ef& tz) {
    x = clamp_<ef>(x, ef(0.0f), ef(4.0f), clx);
    y = clamp_<ef>(y, ef(0.0f), ef(4.0f), cly);
    z = clamp_<ef>(z, ef(1.0f), ef(9.0f), clz);
    bool straddle = ef_reaches_int(x, 0, 4) || ef_reaches_int(y, 0, 4) || ef_reaches_int(z, 1, 9);
    int ix = clamp_cell((int)floorf(x.v), 3);
    int iy = clamp_cell((int)floorf(y.v), 3);
    int iz = clamp_cell((int)floorf(z.v - 1.0f), 7);
    tx = x - ef(ix); ty = y - ef(iy); tz = z - ef(1) - ef(iz);
    if (straddle) tx.e = EF_INF;
    return (ix * 4 + iy) * 8 + iz;
}

template <>
HD ef tricubic_cell<ef, false>(const ef* a, ef tx, ef ty, ef tz, bool, bool, bool, ef& fx, ef& fy, ef& fz) {
    fx = fy = fz = ef(0.0f);
    if (is_zero(tx) && is_zero(ty) && is_zero(tz)) return a[0];
    ef f(0.0f);
    for (int p = 3; p >= 0; p--) {
        ef cp(0.0f);
        for (int q = 3; q >= 0; q--) {
            const ef* c = a + (p * 4 + q) * 4;
            ef cq = ((c[3] * tz + c[2]) * tz + c[1]) * tz + c[0];
            cp = cp * ty + cq;
        }
        f = f * tx + cp;
    }
    if (!(tx.e < EF_INF)) f.e = EF_INF;       // a poisoned cell
    return f;
}

// g_C with its N-blend: the single-function branches only where the blend
// weight is exact
template <> HD ef gfun<ef, false>(const DevParams<ef>& P, int tc, ef cs, ef N, ef& dg_dcos, ef& dg_dN) {
    dg_dcos = ef(0.0f);
    dg_dN = ef(0.0f);
    if (tc == 0) {
        ef dQ;
        ef Qn = Sw<ef>((N - P.gN0) * P.gNinv, dQ);
        ef d;
        if (Qn.e == 0.0f && Qn.v >= 1.0f) return quintic<ef, false>(P.gC2, cs, d);
        if (Qn.e == 0.0f && Qn.v <= 0.0f) return quintic<ef, false>(P.gC1, cs, d);
        ef G = quintic<ef, false>(P.gC1, cs, d);
        ef gam = quintic<ef, false>(P.gC2, cs, d);
        return G + Qn * (gam - G);
    }
    ef d;
    return quintic<ef, false>(P.gH, cs, d);
}

// ------------------------------------------------------------------ the FP32 short list as ef
// Each FP32 copy of an FP64 list value enters with its rounding error.
struct EfIn {
    const float* p;
    HD ef operator[](size_t i) const {
        float v = p[i];
        return ef::raw(v, ru_fma(fabsf(v), 5.9604652e-08f, EF_TINY));    // 2^-24 (1 + 2^-22)
    }
};
// The bond weights and coordinations are exact (1, 2, 3, ...) for most
// atoms.  Their FP32 copies carry that fact in the last mantissa bit: an
// inexact copy has it set (the short-list kernel sets it, within 2 ulp of
// the FP64 value), an exact one has it clear, or set if the value itself
// ends in a 1 (then it is counted as inexact).
HD float ef_mark_inexact(double x) {
    float v = (float)x;
    if ((double)v == x) return v;
#ifdef __CUDA_ARCH__
    return __int_as_float(__float_as_int(v) | 1);
#else
    unsigned b; memcpy(&b, &v, 4); b |= 1u; memcpy(&v, &b, 4); return v;
#endif
}
struct EfInMarked {
    const float* p;
    HD ef operator[](size_t i) const {
        float v = p[i];
#ifdef __CUDA_ARCH__
        bool inexact = __float_as_int(v) & 1;
#else
        unsigned b; memcpy(&b, &v, 4); bool inexact = b & 1u;
#endif
        return ef::raw(v, inexact ? ru_fma(fabsf(v), 2.3841860e-07f, EF_TINY) : 0.0f);   // 2 ulp (2^-22 |v|)
    }
};
struct GraphEf {
    int n, stride;
    const int8_t* type;
    const int* cnt; const int* nj; const int* nimg;
    EfIn dx, dy, dz, r, ir;
    EfInMarked w, nC, nH;
    HD explicit GraphEf(const Graph<float>& g)
        : n(g.n), stride(g.stride), type(g.type), cnt(g.cnt), nj(g.nj), nimg(g.nimg), dx{g.dx}, dy{g.dy}, dz{g.dz},
          r{g.r}, ir{g.ir}, w{g.w}, nC{g.nC}, nH{g.nH} {}
};

// A displacement component rounded to FP32, with a bound on the rounding
// from the rounded value alone: |x - RN(x)| <= 2^-24 |RN(x)| for a normal
// result, plus the smallest subnormal for one below the normal range.  One
// conversion and FP32 work (the exact error, x - (double)RN(x), would take
// three more FP64-pipe instructions); the bound is the worst case of the
// rounding at this magnitude, at most twice the largest error it can make.
HD ef ef_round(double x) {
    float v = (float)x;
    return ef::raw(v, ru_add(ru_mul(fabsf(v), 5.9604645e-8f), 1.4e-45f));
}

// b* of the pair i -> (j, image) (the bond order at the fixed length r* along
// the FP64 displacement d), with its bound
template <class GT>
HD ef bstar_value_ef(const DevParams<ef>& P, const GT& G, int i, int j, double dx, double dy, double dz) {
    int p = pidx(G.type[i], G.type[j]);
    ef x = ef_round(dx), y = ef_round(dy), z = ef_round(dz);
    ef r2 = x * x + y * y + z * z;
    ef inv_r = rsqrt_(r2);
    ef rs = P.rstar[p];
    ef ux = x * inv_r * rs, uy = y * inv_r * rs, uz = z * inv_r * rs;
    ef gux(0.0f), guy(0.0f), guz(0.0f), gumag(0.0f);
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    Sink none{nullptr, 0, false, {0, 0, 0, 0, 0, 0}, false, {0, 0, 0, 0, 0, 0}};
    return bond_order_c<ef, false, Sink, GT>(P, G, i, j, ux, uy, uz, rs, rcp_(rs), ef(0.0f), none, gux, guy, guz, gumag,
                                           fix, fiy, fiz, fjx, fjy, fjz);
}

}  // namespace airebo

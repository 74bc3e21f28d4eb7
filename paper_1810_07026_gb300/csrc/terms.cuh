// AIREBO term arithmetic for the CUDA path: switches, splines, bond order
// (forward and reverse), REBO bond, torsion, LJ pair with C_ij, b* pair.
//
// Every function here works on one interaction (one bond, one pair) and is
// written for one GPU thread; the kernels in kernels.cuh map threads and warps
// onto interactions.  Energies follow Sec. 2.1 of Hoehnerbach & Bientinesi:
//   E^REBO_ij = f_R(r_ij) + b_ij f_A(r_ij)                             (Alg. 1)
//   b_ij = 1/2 (p_ij + p_ji) + pi^rc_ij + pi^dh_ij                      (Sec. 2.1.3)
//   p_ij = [1 + sum_k w_ik g_i(cos theta_jik) e^lambda_jik + P_ij]^-1/2  (Sec. 2.1.3)
//   E^tors = sum w_ki w_ij w_jl V^tors(omega_kijl)                      (Alg. 2)
//   E^LJ_ij = (S_r S_b(b*_ij) + 1 - S_r) C_ij V^LJ(r_ij)                (Alg. 3, Sec. 2.1.2)
// Forces use the forward/reverse pattern of Sec. 2: a forward pass forms the
// sums, the reverse pass pushes dE/d(sum) back onto every bond vector.
// Each gradient with respect to a bond vector v = x_b - x_a is applied as
// F_b -= g, F_a += g and adds -v (x) g to the virial.
//
// R is the arithmetic type of the geometry, splines and bond order (double
// for the FP64 path, float for the mixed path, and the double-float dd of
// dd.cuh for the torsion term of the DF64 path); forces, energies and virial
// are always accumulated in double.
#pragma once

#include <cstdint>
#include <cmath>
#include <cstring>
#include <type_traits>

#ifdef __CUDACC__
#define HD __host__ __device__ __forceinline__
#else
#define HD inline
#endif

namespace airebo {

constexpr int MAXN = 16;           // largest number of REBO neighbours per atom (slots fit 4 bits);
                                   // the slot stride starts at 8, the bound assumed in Sec. 4.3, and grows
constexpr int NTRI_CELLS = 4 * 4 * 8;

// ------------------------------------------------------------------ images
HD int pack_img(int sx, int sy, int sz) { return (sx & 0xff) | ((sy & 0xff) << 8) | ((sz & 0xff) << 16); }
HD int img_x(int p) { return (int)(int8_t)(p & 0xff); }
HD int img_y(int p) { return (int)(int8_t)((p >> 8) & 0xff); }
HD int img_z(int p) { return (int)(int8_t)((p >> 16) & 0xff); }
HD int img_add(int a, int b) { return pack_img(img_x(a) + img_x(b), img_y(a) + img_y(b), img_z(a) + img_z(b)); }

// ------------------------------------------------------------------ atomics
HD void atomic_add(double* p, double v) {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
}

// ------------------------------------------------------------------ math wrappers
// -x by flipping the sign bit: an integer op, not an FP64 instruction
HD double neg_(double x) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
#else
    return -x;
#endif
}
// 1/sqrt(x) and 1/x in FP64 for positive, finite, normal x (every use here:
// squared lengths and 1 + sum + P >= 0.95).  The hardware's approximate FP64
// reciprocal (square root) is refined by one third-order Newton-Raphson step
// (Householder's method): with y0 = (1 + d)/sqrt(x), e = 1 - x y0^2 and
// y1 = y0 (1 + e/2 + 3e^2/8), the relative error becomes O(d^3); for 1/x,
// e = 1 - x y0 and y1 = y0 (1 + e + e^2).  Checked against correctly rounded
// results on the device (tests/test_gpu_math.py).
HD double rsqrt_(double x) {
#ifdef __CUDA_ARCH__
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-(x * y), y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
#else
    return 1.0 / std::sqrt(x);
#endif
}
HD float rsqrt_(float x) {
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / std::sqrt(x);
#endif
}
HD double rcp_(double x) {
#ifdef __CUDA_ARCH__
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
#else
    return 1.0 / x;
#endif
}
HD float rcp_(float x) {
#ifdef __CUDA_ARCH__
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else
    return 1.0f / x;
#endif
}
HD double floor_(double x) { return floor(x); }
HD float floor_(float x) { return floorf(x); }
HD double sqrt_(double x) { return sqrt(x); }
HD float sqrt_(float x) { return sqrtf(x); }
HD double exp_(double x) { return exp(x); }
HD float exp_(float x) { return expf(x); }
// t == 0 (either sign) by the bit pattern: an integer test, no FP64 compare
HD bool is_zero(double t) {
#ifdef __CUDA_ARCH__
    return (__double_as_longlong(t) << 1) == 0;
#else
    return t == 0.0;
#endif
}
HD bool is_zero(float t) {
#ifdef __CUDA_ARCH__
    return (__float_as_int(t) << 1) == 0;
#else
    return t == 0.0f;
#endif
}
HD void sincospi_(double t, double* s, double* c) {
#ifdef __CUDA_ARCH__
    sincospi(t, s, c);
#else
    *s = std::sin(M_PI * t); *c = std::cos(M_PI * t);
#endif
}
HD void sincospi_(float t, float* s, float* c) {
#ifdef __CUDA_ARCH__
    sincospif(t, s, c);
#else
    *s = (float)std::sin(M_PI * (double)t); *c = (float)std::cos(M_PI * (double)t);
#endif
}

}  // namespace airebo

#ifdef __CUDACC__
#include "dd.cuh"          // the double-float value type (R = dd: the DF64 torsion term)
#endif

namespace airebo {

// ------------------------------------------------------------------ parameters
template <class R> struct Quintic {
    int n;             // number of intervals
    R k[6];            // knots
    R invh[5];         // 1 / interval width
    R a[5][6];         // power-basis coefficients in t = (x - k_m) / h_m
    R da[5][5];        // those of the derivative in x: (p + 1) a[p + 1] / h_m
};

// Device copy of the parameter set; pair-indexed arrays use 0 = CC, 1 = CH, 2 = HH.
template <class R> struct DevParams {
    R Dmin[3], Dmax[3], Dinv[3];
    R Q[3], alpha[3], A[3], B[3][3], beta[3][3];
    int nB[3];
    R rhoH[2];                      // rho between an H centre and a neighbour of type t
    R lam;
    R gN0, gNinv, Fx0, Fxinv;
    Quintic<R> gC1, gC2, gH;
    R guard0, guardinv;
    R sigma[3], sig2[3], eps4[3], rc2[3], swlo[3], swlo2[3], swinv[3], Srlo[3], Srhi[3], Srhi2[3], Srinv[3];
    R bmin[3], bmax[3], binv[3], rstar[3];
    R teps[3];
    int kind;                        // inter-molecular term: 0 Lennard-Jones (AIREBO), 1 Morse (AIREBO-M)
    R meps[3], malpha[3], mre[3];    // Morse well depth, stiffness, minimum
    R rpath2;                        // no C_ij path reaches beyond sqrt(rpath2)
    const R* Ptab;                   // 3 tables (CC, CH, HC) x 16 cells x 16 coefficients
    const R* Ftab;                   // 3 tables (CC, CH, HH) x 128 cells x 64 coefficients
    const R* Ttab;                   // T_CC: 128 cells x 64 coefficients
    const unsigned char* Tnz;        // 1 where a T_CC cell has a nonzero coefficient
    // the knot data (value and first derivatives) of the same splines, for
    // arguments that lie on knots: P 3 x 25 x (f, fx, fy); pi^rc 3 x 225 x
    // (f, fx, fy, fz); T_CC 225 x (f, fx, fy, fz)
    const R* Pknot;
    const R* Fknot;
    const R* Tknot;
    double* kg;                      // dE/d(power-basis coefficient) of every spline, or null (layout KG_*)
};

// Layout of the spline-coefficient gradient: the three angular splines
// (5 intervals x 6 coefficients each), then the P, pi^rc and T tables in
// their device layout.
constexpr int KG_GC1 = 0, KG_GC2 = 30, KG_GH = 60, KG_P = 90, KG_F = KG_P + 3 * 256;
constexpr int KG_T = KG_F + 3 * NTRI_CELLS * 64, KG_N = KG_T + NTRI_CELLS * 64;

HD int pidx(int ti, int tj) { return ti + tj; }

// a < b for non-negative, non-NaN a and b, by their IEEE bit patterns: an
// integer compare, which keeps squared-distance tests off the FP64 pipe
HD bool lt_nonneg(double a, double b) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(a) < __double_as_longlong(b);
#else
    return a < b;
#endif
}
HD bool lt_nonneg(float a, float b) { return a < b; }

// Ordered comparisons of FP64 values as 64-bit integers: the sign-magnitude
// bit pattern turned into two's complement orders like the values (-0 maps
// to 0; a NaN sorts beyond the infinity of its sign).  Comparisons are
// frequent in the splines, switches and clamps of the bond order, and an FP64
// compare takes an FP64-pipe issue; these take integer operations.  FP32
// values compare natively.
HD long long okey(double x) {
#ifdef __CUDA_ARCH__
    long long b = __double_as_longlong(x);
#else
    long long b;
    memcpy(&b, &x, sizeof(b));
#endif
    return b < 0 ? -(b & 0x7fffffffffffffffLL) : b;
}
HD bool lt_(double a, double b) {
#ifdef __CUDA_ARCH__
    return okey(a) < okey(b);
#else
    return a < b;
#endif
}
HD bool lt_(float a, float b) { return a < b; }
template <class R> HD bool gt_(R a, R b) { return lt_(b, a); }
template <class R> HD bool le_(R a, R b) { return !lt_(b, a); }
template <class R> HD bool ge_(R a, R b) { return !lt_(a, b); }
// clamp to [lo, hi]; for FP64 a NaN ends at one of the ends (its key lies
// beyond the infinities), for FP32 at lo
template <class R> HD R clamp_(R x, R lo, R hi, bool& cl) {
    cl = false;
    if (lt_(x, lo)) { x = lo; cl = true; }
    if (gt_(x, hi)) { x = hi; cl = true; }
    if (sizeof(R) == 4 && !(x == x)) { x = lo; cl = true; }
    return x;
}

// ------------------------------------------------------------------ switches
// S(t) = 1 for t <= 0, 0 for t >= 1, (1 + cos pi t)/2 between; dS = dS/dt
template <class R> HD R Sw(R t, R& dS) {
    if (le_(t, R(0))) { dS = R(0); return R(1); }
    if (ge_(t, R(1))) { dS = R(0); return R(0); }
    R s, c;
    sincospi_(t, &s, &c);
    dS = R(-0.5 * M_PI) * s;
    return R(0.5) * (R(1) + c);
}
// bond weight w(r) and dw/dr
template <class R> HD R wfun(const DevParams<R>& P, int p, R r, R& dw) {
    R dS;
    R w = Sw<R>((r - P.Dmin[p]) * P.Dinv[p], dS);
    dw = dS * P.Dinv[p];
    return w;
}
// the same with 1 - w formed without cancellation (1 - cos = sin^2 / (1 + cos)),
// so that C_ij = 1 - w keeps its relative precision when w is close to 1
template <class R> HD R wfun_c(const DevParams<R>& P, int p, R r, R& dw, R& omw) {
    R t = (r - P.Dmin[p]) * P.Dinv[p];
    if (le_(t, R(0))) { dw = R(0); omw = R(0); return R(1); }
    if (ge_(t, R(1))) { dw = R(0); omw = R(1); return R(0); }
    R s, c;
    sincospi_(t, &s, &c);
    dw = R(-0.5 * M_PI) * s * P.Dinv[p];
    omw = gt_(c, R(0)) ? R(0.5) * s * s * rcp_(R(1) + c) : R(0.5) * (R(1) - c);
    return R(0.5) * (R(1) + c);
}

// ------------------------------------------------------------------ splines
// D = true: value and derivative(s); D = false: value only
template <class R, bool D = true> HD R quintic(const Quintic<R>& q, R x, R& dfdx) {
    bool cl;
    x = clamp_<R>(x, q.k[0], q.k[q.n], cl);
    int m = 0;
    while (m + 1 < q.n && gt_(x, q.k[m + 1])) m++;
    R t = (x - q.k[m]) * q.invh[m];
    const R* a = q.a[m];
    R f = a[5];
    f = f * t + a[4];
    f = f * t + a[3];
    f = f * t + a[2];
    f = f * t + a[1];
    f = f * t + a[0];
    if (D) {
        const R* b = q.da[m];
        R d = b[4];
        d = d * t + b[3];
        d = d * t + b[2];
        d = d * t + b[1];
        d = d * t + b[0];
        dfdx = cl ? R(0) : d;
    } else {
        dfdx = R(0);
    }
    return f;
}

// The knot, an integer in [lo, hi] (0 <= lo < hi <= 15), that a spline
// argument x lies on after the clamp to [lo, hi], or -1 when it lies between
// two knots; cl: x was clamped.  For FP64 by integer operations on the bit
// pattern (no FP64-pipe issue): x in (lo, hi) is an integer when the
// mantissa bits below its binary point are zero.
HD int knot_of(double x, int lo, int hi, bool& cl) {
    long long k = okey(x), klo = okey((double)lo), khi = okey((double)hi);
    cl = false;
    if (k <= klo) { cl = k < klo; return lo; }
    if (k >= khi) { cl = k > khi; return hi; }
    long long b = k;                             // x > lo >= 0: the key is the bit pattern
    int e = (int)(b >> 52) - 1023;               // 0 <= e <= 3 for 1 <= x < 16
    if (e < 0) return -1;
    long long m = b & 0xFFFFFFFFFFFFFLL;
    if (m & ((1LL << (52 - e)) - 1)) return -1;
    return (int)((1LL << e) | (m >> (52 - e)));
}
HD int knot_of(float x, int lo, int hi, bool& cl) {
    cl = false;
    if (!(x > (float)lo)) { cl = x < (float)lo || !(x == x); return lo; }
    if (x >= (float)hi) { cl = x > (float)hi; return hi; }
    int k = (int)x;
    return (float)k == x ? k : -1;
}
// value and first derivatives of a knot all zero
template <class R> HD bool knot_zero(const R* t) {
    if constexpr (std::is_floating_point<R>::value) return is_zero(t[0]) && is_zero(t[1]) && is_zero(t[2]) && is_zero(t[3]);
    else return false;
}
// the knot of the tricubic grid (N_ij, N_ji in [0, 4], N^conj in [1, 9]) that
// (x, y, z) lies on, as (x * 5 + y) * 9 + z - 1, or -1
template <class R> HD int tri_knot(R x, R y, R z, bool& clx, bool& cly, bool& clz) {
    int kx = knot_of(x, 0, 4, clx), ky = knot_of(y, 0, 4, cly), kz = knot_of(z, 1, 9, clz);
    return (kx < 0 || ky < 0 || kz < 0) ? -1 : (kx * 5 + ky) * 9 + (kz - 1);
}

// clamp a spline argument (a NaN too: every table index stays in range)
template <class R> HD void clamp_arg(R& x, R lo, R hi, bool& cl) { x = clamp_<R>(x, lo, hi, cl); }
HD int clamp_cell(int c, int hi) { return c < 0 ? 0 : (c > hi ? hi : c); }

// bicubic on the integer grid [0,4]^2, 16 power-basis coefficients per cell
template <class R, bool D = true> HD R bicubic(const R* tab, R x, R y, R& fx, R& fy) {
    bool cx, cy;
    clamp_arg<R>(x, R(0), R(4), cx);
    clamp_arg<R>(y, R(0), R(4), cy);
    int ix = clamp_cell((int)floor_(x), 3);
    int iy = clamp_cell((int)floor_(y), 3);
    R tx = x - R(ix), ty = y - R(iy);
    const R* a = tab + (ix * 4 + iy) * 16;
    if (is_zero(tx) && is_zero(ty)) {        // at a knot (integer N^C, N^H): the corner coefficients
        fx = (D && !cx) ? a[4] : R(0);
        fy = (D && !cy) ? a[1] : R(0);
        return a[0];
    }
    // at t = 0 in a dimension only its powers 0 and 1 (0 without derivatives)
    // contribute: the loops stop there, with the same sums as the full ones
    int pt = is_zero(tx) ? (D ? 1 : 0) : 3;
    bool ty0 = is_zero(ty);
    R f = 0, dx = 0, dy = 0;
#pragma unroll
    for (int p = 3; p >= 0; p--) {
        if (p > pt) continue;
        const R* c = a + p * 4;
        R cp = ty0 ? c[0] : ((c[3] * ty + c[2]) * ty + c[1]) * ty + c[0];
        if (D) {
            R dcp = ty0 ? c[1] : (R(3) * c[3] * ty + R(2) * c[2]) * ty + c[1];
            dx = dx * tx + f;
            dy = dy * tx + dcp;
        }
        f = f * tx + cp;
    }
    fx = (D && !cx) ? dx : R(0);
    fy = (D && !cy) ? dy : R(0);
    return f;
}

// tricubic on [0,4]x[0,4]x[1,9], 64 power-basis coefficients per cell
template <class R> HD int tri_cell_index(R& x, R& y, R& z, bool& clx, bool& cly, bool& clz, R& tx, R& ty, R& tz) {
    clamp_arg<R>(x, R(0), R(4), clx);
    clamp_arg<R>(y, R(0), R(4), cly);
    clamp_arg<R>(z, R(1), R(9), clz);
    int ix = clamp_cell((int)floor_(x), 3);
    int iy = clamp_cell((int)floor_(y), 3);
    int iz = clamp_cell((int)floor_(z - R(1)), 7);
    tx = x - R(ix); ty = y - R(iy); tz = z - R(1) - R(iz);
    return (ix * 4 + iy) * 8 + iz;
}
template <class R, bool D = true>
HD R tricubic_cell(const R* a, R tx, R ty, R tz, bool clx, bool cly, bool clz, R& fx, R& fy, R& fz) {
    if (is_zero(tx) && is_zero(ty) && is_zero(tz)) {   // at a knot: the corner coefficients
        fx = (D && !clx) ? a[16] : R(0);
        fy = (D && !cly) ? a[4] : R(0);
        fz = (D && !clz) ? a[1] : R(0);
        return a[0];
    }
    // at t = 0 in a dimension only its powers 0 and 1 (0 without derivatives)
    // contribute: the loops stop there, with the same sums as the full ones
    int pt = is_zero(tx) ? (D ? 1 : 0) : 3, qt = is_zero(ty) ? (D ? 1 : 0) : 3;
    bool tz0 = is_zero(tz);
    R f = 0, dx = 0, dy = 0, dz = 0;
#pragma unroll
    for (int p = 3; p >= 0; p--) {
        if (p > pt) continue;
        R cp = 0, cpy = 0, cpz = 0;
#pragma unroll
        for (int q = 3; q >= 0; q--) {
            if (q > qt) continue;
            const R* c = a + (p * 4 + q) * 4;
            R cq = tz0 ? c[0] : ((c[3] * tz + c[2]) * tz + c[1]) * tz + c[0];
            if (D) {
                R dcq = tz0 ? c[1] : (R(3) * c[3] * tz + R(2) * c[2]) * tz + c[1];
                cpy = cpy * ty + cp;
                cpz = cpz * ty + dcq;
            }
            cp = cp * ty + cq;
        }
        if (D) {
            dx = dx * tx + f;
            dy = dy * tx + cpy;
            dz = dz * tx + cpz;
        }
        f = f * tx + cp;
    }
    fx = (D && !clx) ? dx : R(0);
    fy = (D && !cly) ? dy : R(0);
    fz = (D && !clz) ? dz : R(0);
    return f;
}

// Gradient of a spline value with respect to its coefficients.  Every
// spline here is linear in its power-basis coefficients, so d value / d a_m
// is the monomial m at the (clamped) local coordinates; adj = dE/d value.
template <class R> HD void kg_quintic(double* g, const Quintic<R>& q, R x, double adj) {
    bool cl;
    x = clamp_<R>(x, q.k[0], q.k[q.n], cl);
    int m = 0;
    while (m + 1 < q.n && gt_(x, q.k[m + 1])) m++;
    double t = (double)((x - q.k[m]) * q.invh[m]), tp = 1.0;
    for (int p = 0; p < 6; p++, tp *= t) atomic_add(g + m * 6 + p, adj * tp);
}
template <class R> HD void kg_bicubic(double* g, R x, R y, double adj) {
    bool cx, cy;
    clamp_arg<R>(x, R(0), R(4), cx);
    clamp_arg<R>(y, R(0), R(4), cy);
    int ix = clamp_cell((int)floor_(x), 3);
    int iy = clamp_cell((int)floor_(y), 3);
    double tx = (double)(x - R(ix)), ty = (double)(y - R(iy));
    g += (ix * 4 + iy) * 16;
    double xp = adj;
    for (int p = 0; p < 4; p++, xp *= tx) {
        double v = xp;
        for (int q = 0; q < 4; q++, v *= ty) atomic_add(g + p * 4 + q, v);
    }
}
template <class R> HD void kg_tricubic(double* g, R tx, R ty, R tz, double adj) {
    double xp = adj;
    for (int p = 0; p < 4; p++, xp *= (double)tx) {
        double yp = xp;
        for (int q = 0; q < 4; q++, yp *= (double)ty) {
            double v = yp;
            for (int r = 0; r < 4; r++, v *= (double)tz) atomic_add(g + (p * 4 + q) * 4 + r, v);
        }
    }
}

// ------------------------------------------------------------------ neighbour data
// Short REBO list of one step: slot s of atom i at index i * G.stride + s.
template <class R> struct Graph {
    int n;
    int stride;              // slots per atom (<= MAXN)
    const int8_t* type;
    const int* cnt;          // neighbours per atom
    const int* nj;           // neighbour atom
    const int* nimg;         // packed image of the neighbour relative to i
    const R* dx; const R* dy; const R* dz;   // x_j + S L - x_i
    const R* r; const R* ir; const R* w; const R* dw;   // |d|, 1/|d|, w, dw/dr
    const R* omw;                            // 1 - w
    const R* nC; const R* nH;                // sum of w over C / H neighbours
};

// The short REBO list of one precision read in another arithmetic type: the
// torsion term of the DF64 path runs in double-float on the FP64 list.
template <class R, class S> struct ConvArray {
    const S* p;
    HD R operator[](size_t i) const { return R(p[i]); }
};
template <class R, class S> struct GraphAs {
    int n, stride;
    const int8_t* type;
    const int* cnt; const int* nj; const int* nimg;
    ConvArray<R, S> dx, dy, dz, r, ir, w, dw, omw, nC, nH;
    HD explicit GraphAs(const Graph<S>& g)
        : n(g.n), stride(g.stride), type(g.type), cnt(g.cnt), nj(g.nj), nimg(g.nimg), dx{g.dx}, dy{g.dy}, dz{g.dz},
          r{g.r}, ir{g.ir}, w{g.w}, dw{g.dw}, omw{g.omw}, nC{g.nC}, nH{g.nH} {}
};

// Slot of atom o among the REBO neighbours of c (MAXN when absent).  The
// loops over N(c) \ {o} below run over the other slots by index, so that
// threads whose atoms have equal neighbour counts run equal trip counts
// instead of each skipping o at a different iteration.
template <class GT> HD int slot_of(const GT& G, int c, int o) {
    int nc = G.cnt[c];
    for (int a = 0; a < nc; a++)
        if (G.nj[c * G.stride + a] == o) return a;
    return MAXN;
}

// accumulation of forces (atomics) and the virial of one thread
struct Sink {
    double* f;          // 3 x n, SoA
    int n;
    bool virial;
    double W[6];
    bool pgrad;         // accumulate dE/d(epsilon) and dE/d(sigma) of the inter-molecular term
    double G[6];        // dE/d eps[CC, CH, HH], dE/d sigma[CC, CH, HH]
    HD void pair(int a, int b, double vx, double vy, double vz, double gx, double gy, double gz) {
        atomic_add(f + b, neg_(gx)); atomic_add(f + n + b, neg_(gy)); atomic_add(f + 2 * n + b, neg_(gz));
        atomic_add(f + a, gx); atomic_add(f + n + a, gy); atomic_add(f + 2 * n + a, gz);
        if (virial) {
            W[0] -= vx * gx; W[1] -= vy * gy; W[2] -= vz * gz;
            W[3] -= vx * gy; W[4] -= vx * gz; W[5] -= vy * gz;
        }
    }
#ifdef __CUDACC__
    // the same from double-float vectors
    HD void pair(int a, int b, dd vx, dd vy, dd vz, dd gx, dd gy, dd gz) {
        pair(a, b, (double)vx, (double)vy, (double)vz, (double)gx, (double)gy, (double)gz);
    }
    HD void half(int b, dd vx, dd vy, dd vz, dd gx, dd gy, dd gz, double& fax, double& fay, double& faz) {
        half(b, (double)vx, (double)vy, (double)vz, (double)gx, (double)gy, (double)gz, fax, fay, faz);
    }
#endif
    // gradient on the vector from a to b, where the force on a is kept by the caller
    HD void half(int b, double vx, double vy, double vz, double gx, double gy, double gz,
                 double& fax, double& fay, double& faz) {
        atomic_add(f + b, neg_(gx)); atomic_add(f + n + b, neg_(gy)); atomic_add(f + 2 * n + b, neg_(gz));
        fax += gx; fay += gy; faz += gz;
        if (virial) {
            W[0] -= vx * gx; W[1] -= vy * gy; W[2] -= vz * gz;
            W[3] -= vx * gy; W[4] -= vx * gz; W[5] -= vy * gz;
        }
    }
};

// The dot product of a direction v (3 x n, SoA) with the forces a term would
// apply, in place of applying them: with the same calls as Sink, the forward
// and reverse passes of a term give v . F of that term (a Jacobian-vector
// product of the forces, used for parameter derivatives of the forces).
struct JSink {
    const double* v;
    int n;
    double jdot;
    bool virial;        // never: the interface of Sink
    double W[6];
    HD double vdot(int a, double gx, double gy, double gz) const {
        return v[a] * gx + v[n + a] * gy + v[2 * n + a] * gz;
    }
    // force +g on a, -g on b
    HD void pair(int a, int b, double, double, double, double gx, double gy, double gz) {
        jdot += vdot(a, gx, gy, gz) - vdot(b, gx, gy, gz);
    }
    // force -g on b; +g on a, kept by the caller (applied with add)
    HD void half(int b, double, double, double, double gx, double gy, double gz,
                 double& fax, double& fay, double& faz) {
        jdot -= vdot(b, gx, gy, gz);
        fax += gx; fay += gy; faz += gz;
    }
    HD void add(int a, double fx, double fy, double fz) { jdot += vdot(a, fx, fy, fz); }
};

// ------------------------------------------------------------------ bond order
// One side of b_ij: centre c, partner o.  The forward pass fills it.
template <class R> struct Side {
    R NC, NH, N;        // coordination of c without o, by neighbour species
    R conj;             // sum over C neighbours k != o of w_ck F(x_ck)
    R sum;              // sum_k w g e^lambda
    R dsum_dN;          // d sum / d N (through the g_C mixing)
    R P, dPdNC, dPdNH;
    R p;                // p^{sigma pi}
};

// angular function g_c(cos) (with the g_C mixing in N for a carbon centre);
// only the branch the mixing weight needs is evaluated
template <class R, bool D = true>
HD R gfun(const DevParams<R>& P, int tc, R cs, R N, R& dg_dcos, R& dg_dN) {
    dg_dN = R(0);
    if (tc == 0) {
        R dQ;
        R Qn = Sw<R>((N - P.gN0) * P.gNinv, dQ);
        if (ge_(Qn, R(1))) return quintic<R, D>(P.gC2, cs, dg_dcos);
        if (le_(Qn, R(0))) return quintic<R, D>(P.gC1, cs, dg_dcos);
        R d1, d2;
        R G = quintic<R, D>(P.gC1, cs, d1);
        R gam = quintic<R, D>(P.gC2, cs, d2);
        if (D) {
            dg_dcos = d1 + Qn * (d2 - d1);
            dg_dN = dQ * P.gNinv * (gam - G);
        }
        return G + Qn * (gam - G);
    }
    return quintic<R, D>(P.gH, cs, dg_dcos);
}

// the coefficient gradient of gfun with dE/dg = adj
template <class R> HD void kg_gfun(const DevParams<R>& P, int tc, R cs, R N, double adj) {
    if (tc == 0) {
        R dQ;
        R Qn = Sw<R>((N - P.gN0) * P.gNinv, dQ);
        if (!is_zero(Qn)) kg_quintic<R>(P.kg + KG_GC2, P.gC2, cs, adj * (double)Qn);
        if (lt_(Qn, R(1))) kg_quintic<R>(P.kg + KG_GC1, P.gC1, cs, adj * (1.0 - (double)Qn));
        return;
    }
    kg_quintic<R>(P.kg + KG_GH, P.gH, cs, adj);
}

// e^lambda_jik, lambda = lam [(rho_kH - r_ik) - (rho_jH - r_ij)] for an H centre, else 1
template <class R> HD R exp_lambda(const DevParams<R>& P, int tc, int tk, int to, R rck, R umag) {
    if (tc == 0) return R(1);
    return exp_(P.lam * ((P.rhoH[tk] - rck) - (P.rhoH[to] - umag)));
}

// Per-thread store of the angular terms of a side's first SC_K neighbours
// (the clamped cos, g, dg/dcos -- zero where cos was clamped -- and
// e^lambda), written by the forward pass of a bond order and read back by its
// reverse pass, which then skips their evaluation.  It lives in shared memory
// as [value][slot][thread], so that a warp's accesses are consecutive;
// p == nullptr: no store.
constexpr int SC_K = 4;
template <class R> struct SideCache {
    R* p;
    int stride;          // threads per block
    HD R& at(int t, int v) const { return p[(t * 4 + v) * stride]; }
    HD SideCache side(int s) const { return SideCache{p ? p + s * SC_K * 4 * stride : nullptr, stride}; }
};
// the store of both sides of one thread: 2 SC_K 4 values
template <class R> constexpr int side_cache_len() { return 2 * SC_K * 4; }

template <class R, bool D, class GT = Graph<R>>
HD void side_forward(const DevParams<R>& P, const GT& G, int c, int o, R ux, R uy, R uz, R inv_u, R umag,
                     Side<R>& s, SideCache<R> sc = SideCache<R>{nullptr, 0}) {
    int tc = G.type[c], to = G.type[o];
    int nc = G.cnt[c];
    int so = slot_of(G, c, o);
    int m = nc - (so < MAXN);
    s.NC = 0; s.NH = 0; s.conj = 0;
    for (int t = 0; t < m; t++) {
        int a = t + (t >= so);
        int q = c * G.stride + a;
        int k = G.nj[q];
        R w = G.w[q];
        if (G.type[k] == 0) {
            s.NC += w;
            R x = G.nC[k] + G.nH[k] - w;
            R dF;
            s.conj += w * Sw<R>((x - P.Fx0) * P.Fxinv, dF);
        } else {
            s.NH += w;
        }
    }
    s.N = s.NC + s.NH;
    s.sum = 0; s.dsum_dN = 0;
    for (int t = 0; t < m; t++) {
        int a = t + (t >= so);
        int q = c * G.stride + a;
        int k = G.nj[q];
        R cs = (ux * G.dx[q] + uy * G.dy[q] + uz * G.dz[q]) * inv_u * G.ir[q];
        bool clc;
        cs = clamp_<R>(cs, R(-1), R(1), clc);
        R dgc, dgN;
        R g = gfun<R, D>(P, tc, cs, s.N, dgc, dgN);
        R e = exp_lambda<R>(P, tc, G.type[k], to, G.r[q], umag);
        s.sum += G.w[q] * g * e;
        if constexpr (D) {
            s.dsum_dN += G.w[q] * dgN * e;
            if (sc.p && t < SC_K) {
                sc.at(t, 0) = cs; sc.at(t, 1) = g; sc.at(t, 2) = clc ? R(0) : dgc; sc.at(t, 3) = e;
            }
        }
    }
    s.P = 0; s.dPdNC = 0; s.dPdNH = 0;
    if (!(tc == 1 && to == 1)) {
        int tab = (tc == 0 && to == 0) ? 0 : (tc == 0 ? 1 : 2);
        bool knot = false;
        if constexpr (std::is_floating_point<R>::value) {
            // integer N^C and N^H (every bond fully on): the knot data, which
            // the bicubic interpolates exactly, instead of its polynomial
            bool cx, cy;
            int kx = knot_of(s.NC, 0, 4, cx), ky = knot_of(s.NH, 0, 4, cy);
            if (kx >= 0 && ky >= 0) {
                const R* k = P.Pknot + (tab * 25 + kx * 5 + ky) * 3;
                s.P = k[0];
                if (D) { s.dPdNC = cx ? R(0) : k[1]; s.dPdNH = cy ? R(0) : k[2]; }
                knot = true;
            }
        }
        if (!knot) s.P = bicubic<R, D>(P.Ptab + tab * 256, s.NC, s.NH, s.dPdNC, s.dPdNH);
    }
    s.p = rsqrt_(R(1) + s.sum + s.P);
}

// Reverse of one side.  dEdp: adjoint of p; dEdN_direct: adjoint of N_co
// from pi^rc / pi^dh; dEdconj: adjoint of the conjugation sum.  Accumulates
// the gradient with respect to the partner vector u (sign as given) and to
// its length; applies the forces on the neighbours of c.
template <class R, class SinkT>
HD void side_reverse(const DevParams<R>& P, const Graph<R>& G, int c, int o, R ux, R uy, R uz, R inv_u, R umag,
                     const Side<R>& s, R dEdp, R dEdN_direct, R dEdconj, SinkT& sink,
                     R& gux, R& guy, R& guz, R& gumag, double& fcx, double& fcy, double& fcz,
                     SideCache<R> sc = SideCache<R>{nullptr, 0}) {
    int tc = G.type[c], to = G.type[o];
    int nc = G.cnt[c];
    R ac = R(-0.5) * s.p * s.p * s.p * dEdp;       // dE/dsum = dE/dP
    R dEdN = dEdN_direct + ac * s.dsum_dN;
    R dEdNC = dEdN + ac * s.dPdNC;
    R dEdNH = dEdN + ac * s.dPdNH;
    if (P.kg && !(tc == 1 && to == 1)) {
        int tab = (tc == 0 && to == 0) ? 0 : (tc == 0 ? 1 : 2);
        kg_bicubic<R>(P.kg + KG_P + tab * 256, s.NC, s.NH, (double)ac);
    }
    int so = slot_of(G, c, o);
    int m = nc - (so < MAXN);
    for (int t = 0; t < m; t++) {
        int a = t + (t >= so);
        int q = c * G.stride + a;
        int k = G.nj[q];
        int tk = G.type[k];
        R dxk = G.dx[q], dyk = G.dy[q], dzk = G.dz[q];
        R rck = G.r[q], inv_r = G.ir[q], w = G.w[q], dw = G.dw[q];
        R cs, g, dgc, e;          // dgc: zero where cos was clamped
        if (sc.p && t < SC_K) {   // from the forward pass
            cs = sc.at(t, 0); g = sc.at(t, 1); dgc = sc.at(t, 2); e = sc.at(t, 3);
        } else {
            R cs_raw = (ux * dxk + uy * dyk + uz * dzk) * inv_u * inv_r;
            bool cl;
            cs = clamp_<R>(cs_raw, R(-1), R(1), cl);
            R dgN;
            g = gfun<R, true>(P, tc, cs, s.N, dgc, dgN);
            if (cl) dgc = R(0);
            e = exp_lambda<R>(P, tc, tk, to, rck, umag);
        }
        if (P.kg) kg_gfun<R>(P, tc, cs, s.N, (double)(ac * w * e));
        // d E / d w_ck
        R dEdw = (tk == 0 ? dEdNC : dEdNH) + ac * g * e;
        R Fx = R(0), dFx = R(0);
        if (tk == 0) {
            R x = G.nC[k] + G.nH[k] - w;
            Fx = Sw<R>((x - P.Fx0) * P.Fxinv, dFx);
            dFx *= P.Fxinv;
            dEdw += dEdconj * Fx;
        }
        R dEdr = dEdw * dw;
        if (tc == 1) {           // lambda depends on r_ck (-lam) and on |u| (+lam)
            R t = ac * w * g * e * P.lam;
            dEdr -= t;
            gumag += t;
        }
        R dEdcs = ac * w * e * dgc;
        // cos = u.d / (|u| |d|)
        R a1 = dEdcs * inv_u * inv_r, a2 = dEdcs * cs * inv_r * inv_r, a3 = dEdcs * cs * inv_u * inv_u;
        R er = dEdr * inv_r;
        R gxk = er * dxk + a1 * ux - a2 * dxk;
        R gyk = er * dyk + a1 * uy - a2 * dyk;
        R gzk = er * dzk + a1 * uz - a2 * dzk;
        gux += a1 * dxk - a3 * ux;
        guy += a1 * dyk - a3 * uy;
        guz += a1 * dzk - a3 * uz;
        sink.half(k, dxk, dyk, dzk, gxk, gyk, gzk, fcx, fcy, fcz);
        // conjugation: x_ck = sum_{m in N(k), m != c} w_km
        if (tk == 0 && !is_zero(dFx) && !is_zero(dEdconj)) {
            R coef = dEdconj * w * dFx;
            int nk = G.cnt[k];
            for (int b = 0; b < nk; b++) {
                int qq = k * G.stride + b;
                int m = G.nj[qq];
                if (m == c) continue;
                R dwm = G.dw[qq];
                if (is_zero(dwm)) continue;
                R t = coef * dwm * G.ir[qq];
                sink.pair(k, m, G.dx[qq], G.dy[qq], G.dz[qq], t * G.dx[qq], t * G.dy[qq], t * G.dz[qq]);
            }
        }
    }
}

// angle guard of the dihedral sums: 1 unless |cos| is within the guard band of 1
template <class R> HD R guardf(const DevParams<R>& P, R cs, R& dgd) {
    bool neg = lt_(cs, R(0));
    R a = neg ? -cs : cs;
    R dS;
    R g = Sw<R>((a - P.guard0) * P.guardinv, dS);
    dgd = dS * P.guardinv * (neg ? R(-1) : R(1));
    return g;
}

// sum over k in N(i)\j, l in N(j)\{i,k} of (1 - cos^2 w) w_ik w_jl s_i s_j, and
// (reverse) its gradient times dEdD.  u = vector standing for r_ij.
template <class R, bool REVD, class SinkT, class GT = Graph<R>>
HD R dihedral_sum(const DevParams<R>& P, const GT& G, int i, int j, R ux, R uy, R uz, R inv_u,
                  R dEdD, SinkT& sink, R& gux, R& guy, R& guz,
                  double& fix, double& fiy, double& fiz, double& fjx, double& fjy, double& fjz) {
    R D = 0;
    int ni = G.cnt[i], nj = G.cnt[j];
    int sj = slot_of(G, i, j), si_ = slot_of(G, j, i);
    int mi = ni - (sj < MAXN), mj = nj - (si_ < MAXN);
    for (int ta = 0; ta < mi; ta++) {
        int a = ta + (ta >= sj);
        int qa = i * G.stride + a;
        int k = G.nj[qa];
        R ax = G.dx[qa], ay = G.dy[qa], az = G.dz[qa];
        R inv_ra = G.ir[qa], wik = G.w[qa];
        R csi = (ux * ax + uy * ay + uz * az) * inv_u * inv_ra;
        R dsi;
        R si = guardf<R>(P, csi, dsi);
        if (is_zero(si)) continue;
        // n1 = u x a
        R n1x = uy * az - uz * ay, n1y = uz * ax - ux * az, n1z = ux * ay - uy * ax;
        R n1s = n1x * n1x + n1y * n1y + n1z * n1z;
        R in1s = rcp_(n1s);
        for (int tb = 0; tb < mj; tb++) {
            int b = tb + (tb >= si_);
            int qb = j * G.stride + b;
            int l = G.nj[qb];
            if (l == k) continue;              // a three-ring
            R bx = G.dx[qb], by = G.dy[qb], bz = G.dz[qb];
            R inv_rb = G.ir[qb], wjl = G.w[qb];
            R csj = -(ux * bx + uy * by + uz * bz) * inv_u * inv_rb;
            R dsj;
            R sj = guardf<R>(P, csj, dsj);
            if (is_zero(sj)) continue;
            R n2x = uy * bz - uz * by, n2y = uz * bx - ux * bz, n2z = ux * by - uy * bx;
            R n2s = n2x * n2x + n2y * n2y + n2z * n2z;
            R inv12 = rsqrt_(n1s * n2s);
            R cw = (n1x * n2x + n1y * n2y + n1z * n2z) * inv12;
            R one_m = R(1) - cw * cw;
            D += one_m * wik * wjl * si * sj;
            if constexpr (REVD) {
            R dwik = G.dw[qa], dwjl = G.dw[qb];     // the forward pass reads no dw/dr
            R in2s = rcp_(n2s);
            R dcw = dEdD * R(-2) * cw * wik * wjl * si * sj;
            R dwi = dEdD * one_m * wjl * si * sj;
            R dwj = dEdD * one_m * wik * si * sj;
            R dci = dEdD * one_m * wik * wjl * sj * dsi;   // dE/dcos theta_jik
            R dcj = dEdD * one_m * wik * wjl * si * dsj;   // dE/dcos theta_ijl
            // gradient of cw with respect to n1, n2
            R c1 = dcw * cw * in1s, c2 = dcw * cw * in2s, c12 = dcw * inv12;
            R g1x = c12 * n2x - c1 * n1x, g1y = c12 * n2y - c1 * n1y, g1z = c12 * n2z - c1 * n1z;
            R g2x = c12 * n1x - c2 * n2x, g2y = c12 * n1y - c2 * n2y, g2z = c12 * n1z - c2 * n2z;
            // n1 = u x a: d/du = a x g1, d/da = g1 x u ; n2 = u x b likewise
            gux += ay * g1z - az * g1y + by * g2z - bz * g2y;
            guy += az * g1x - ax * g1z + bz * g2x - bx * g2z;
            guz += ax * g1y - ay * g1x + bx * g2y - by * g2x;
            R gax = g1y * uz - g1z * uy, gay = g1z * ux - g1x * uz, gaz = g1x * uy - g1y * ux;
            R gbx = g2y * uz - g2z * uy, gby = g2z * ux - g2x * uz, gbz = g2x * uy - g2y * ux;
            // weights
            R ea = dwi * dwik * inv_ra, eb = dwj * dwjl * inv_rb;
            gax += ea * ax; gay += ea * ay; gaz += ea * az;
            gbx += eb * bx; gby += eb * by; gbz += eb * bz;
            // guards: csi = u.a/(|u||a|), csj = -u.b/(|u||b|)
            R i1 = dci * inv_u * inv_ra, i2 = dci * csi * inv_ra * inv_ra, i3 = dci * csi * inv_u * inv_u;
            gax += i1 * ux - i2 * ax; gay += i1 * uy - i2 * ay; gaz += i1 * uz - i2 * az;
            gux += i1 * ax - i3 * ux; guy += i1 * ay - i3 * uy; guz += i1 * az - i3 * uz;
            R j1 = dcj * inv_u * inv_rb, j2 = dcj * csj * inv_rb * inv_rb, j3 = dcj * csj * inv_u * inv_u;
            gbx += -j1 * ux - j2 * bx; gby += -j1 * uy - j2 * by; gbz += -j1 * uz - j2 * bz;
            gux += -j1 * bx - j3 * ux; guy += -j1 * by - j3 * uy; guz += -j1 * bz - j3 * uz;
            sink.half(k, ax, ay, az, gax, gay, gaz, fix, fiy, fiz);
            sink.half(l, bx, by, bz, gbx, gby, gbz, fjx, fjy, fjz);
            }
        }
    }
    return D;
}

// The S_b switch of the LJ term evaluated inside a reverse bond order: the
// forward pass gives b*, and the reverse pass then runs with
// dE/db* = scale * dS_b/db* (zero outside the transition, which skips it).
template <class R> struct BstarSwitch {
    R bmin, binv, scale;     // in
    R Sb, dSb;               // out: S_b(b*) and dS_b/db*
};

// b_ij with u standing for r_ij (inv_u = 1/|u|).  REV = false: the value only,
// without any derivative work.  REV = true: also the reverse pass with
// eps = dE/db, which applies the forces on all neighbours and returns the
// gradient with respect to u and its length in gu*, gumag, and the forces on
// i and j themselves in fi*, fj* (excluding the u gradient, which the caller
// applies).
template <class R, bool REV, class SinkT = Sink, class GT = Graph<R>>
HD R bond_order(const DevParams<R>& P, const GT& G, int i, int j, R ux, R uy, R uz, R umag, R inv_u,
                R eps, SinkT& sink, R& gux, R& guy, R& guz, R& gumag,
                double& fix, double& fiy, double& fiz, double& fjx, double& fjy, double& fjz,
                BstarSwitch<R>* bsw = nullptr, SideCache<R> sc = SideCache<R>{nullptr, 0}) {
    Side<R> si, sj;
    side_forward<R, REV, GT>(P, G, i, j, ux, uy, uz, inv_u, umag, si, sc.side(0));
    side_forward<R, REV, GT>(P, G, j, i, -ux, -uy, -uz, inv_u, umag, sj, sc.side(1));
    int ti = G.type[i], tj = G.type[j];
    R Nconj = R(1) + si.conj * si.conj + sj.conj * sj.conj;
    // pi^rc: the carbon side's coordination first for a C-H bond
    int tab = (ti == tj) ? (ti == 0 ? 0 : 2) : 1;
    bool swap = (ti == 1 && tj == 0);
    R xa = swap ? sj.N : si.N, xb = swap ? si.N : sj.N, xc = Nconj;
    bool clx = false, cly = false, clz = false;
    R tx = 0, ty = 0, tz = 0;
    R Fa, Fb, Fc, pirc;
    R pidh = 0, D = 0, Tv = 0, Ta = 0, Tb = 0, Tc = 0;
    int cell = 0;
    bool dih;
    // all three arguments on knots (integer coordinations, the common case of
    // saturated bonds): the knot data of pi^rc and T, which the tricubics
    // interpolate exactly; not with the coefficient gradient, which wants the cell
    int kn = -1;
    if constexpr (std::is_floating_point<R>::value) {
        if (!(REV && P.kg)) kn = tri_knot<R>(xa, xb, xc, clx, cly, clz);
    }
    if (kn >= 0) {
        const R* k = P.Fknot + (tab * 225 + kn) * 4;
        pirc = k[0];
        Fa = (REV && !clx) ? k[1] : R(0); Fb = (REV && !cly) ? k[2] : R(0); Fc = (REV && !clz) ? k[3] : R(0);
        const R* t = P.Tknot + kn * 4;
        dih = (ti == 0 && tj == 0) && !knot_zero<R>(t);
        if (dih) {
            Tv = t[0];
            Ta = (REV && !clx) ? t[1] : R(0); Tb = (REV && !cly) ? t[2] : R(0); Tc = (REV && !clz) ? t[3] : R(0);
        }
    } else {
        cell = tri_cell_index<R>(xa, xb, xc, clx, cly, clz, tx, ty, tz);
        pirc = tricubic_cell<R, REV>(P.Ftab + (tab * NTRI_CELLS + cell) * 64, tx, ty, tz, clx, cly, clz, Fa, Fb, Fc);
        // pi^dh (C-C only), skipped where the T_CC cell is identically zero
        // (unless its coefficients' gradient is wanted)
        dih = (ti == 0 && tj == 0) && (P.Tnz[cell] || (REV && P.kg));
        if (dih) Tv = tricubic_cell<R, REV>(P.Ttab + cell * 64, tx, ty, tz, clx, cly, clz, Ta, Tb, Tc);
    }
    R dFdNi = swap ? Fb : Fa, dFdNj = swap ? Fa : Fb;
    if (dih) {
        R dummy = 0;
        D = dihedral_sum<R, false, SinkT, GT>(P, G, i, j, ux, uy, uz, inv_u, R(0), sink, dummy, dummy, dummy,
                                              fix, fiy, fiz, fjx, fjy, fjz);
        pidh = Tv * D;
    }
    R b = R(0.5) * (si.p + sj.p) + pirc + pidh;
    if constexpr (!REV) {
        return b;
    } else {
    if (bsw) {
        R dS;
        bsw->Sb = Sw<R>((b - bsw->bmin) * bsw->binv, dS);
        bsw->dSb = dS * bsw->binv;
        eps = bsw->scale * bsw->dSb;
        if (is_zero(eps)) return b;     // no gradient flows through b* (nor to the spline knots)
    }
    if (P.kg) {
        kg_tricubic<R>(P.kg + KG_F + (tab * NTRI_CELLS + cell) * 64, tx, ty, tz, (double)eps);
        if (dih) kg_tricubic<R>(P.kg + KG_T + cell * 64, tx, ty, tz, (double)(eps * D));
    }
    R dEdNi = eps * (dFdNi + D * Ta);
    R dEdNj = eps * (dFdNj + D * Tb);
    R dEdNconj = eps * (Fc + D * Tc);
    R half = R(0.5) * eps;
    R gvx = 0, gvy = 0, gvz = 0;     // side j works on -u
    side_reverse<R>(P, G, i, j, ux, uy, uz, inv_u, umag, si, half, dEdNi, dEdNconj * R(2) * si.conj, sink,
                    gux, guy, guz, gumag, fix, fiy, fiz, sc.side(0));
    side_reverse<R>(P, G, j, i, -ux, -uy, -uz, inv_u, umag, sj, half, dEdNj, dEdNconj * R(2) * sj.conj, sink,
                    gvx, gvy, gvz, gumag, fjx, fjy, fjz, sc.side(1));
    gux -= gvx; guy -= gvy; guz -= gvz;
    if (dih) {
        dihedral_sum<R, true, SinkT, GT>(P, G, i, j, ux, uy, uz, inv_u, eps * Tv, sink, gux, guy, guz,
                                         fix, fiy, fiz, fjx, fjy, fjz);
    }
    return b;
    }
}

// bond_order of an unbonded pair in a canonical orientation: the carbon
// first for a C-H pair, the lower index first for a like pair.  b_ij = b_ji
// with u -> -u for the symmetric tables of the potential, but not for a
// perturbed (asymmetric) pi^rc or T table, so the orientation must not depend
// on which atom's list row holds the pair; and the lanes of a warp of C-H
// pairs then walk the carbon's neighbours in the same side pass.  The swap is
// made on the arguments and undone on the results.
template <class R, bool REV, class SinkT = Sink, class GT = Graph<R>>
HD R bond_order_c(const DevParams<R>& P, const GT& G, int i, int j, R ux, R uy, R uz, R umag, R inv_u,
                  R eps, SinkT& sink, R& gux, R& guy, R& guz, R& gumag,
                  double& fix, double& fiy, double& fiz, double& fjx, double& fjy, double& fjz,
                  BstarSwitch<R>* bsw = nullptr, SideCache<R> sc = SideCache<R>{nullptr, 0}) {
    int ti = G.type[i], tj = G.type[j];
    bool sw = (ti == 1 && tj == 0) || (ti == tj && j < i);
    int a = sw ? j : i, b = sw ? i : j;
    R vx = sw ? -ux : ux, vy = sw ? -uy : uy, vz = sw ? -uz : uz;
    R gvx = R(0), gvy = R(0), gvz = R(0);
    double fax = 0, fay = 0, faz = 0, fbx = 0, fby = 0, fbz = 0;
    R bo = bond_order<R, REV, SinkT, GT>(P, G, a, b, vx, vy, vz, umag, inv_u, eps, sink, gvx, gvy, gvz, gumag,
                                         fax, fay, faz, fbx, fby, fbz, bsw, sc);
    if constexpr (REV) {
        gux += sw ? -gvx : gvx; guy += sw ? -gvy : gvy; guz += sw ? -gvz : gvz;
        fix += sw ? fbx : fax; fiy += sw ? fby : fay; fiz += sw ? fbz : faz;
        fjx += sw ? fax : fbx; fjy += sw ? fay : fby; fjz += sw ? faz : fbz;
    }
    return bo;
}

// ------------------------------------------------------------------ REBO bond (Alg. 1)
template <class R>
HD double rebo_bond(const DevParams<R>& P, const Graph<R>& G, int i, int slot, Sink& sink,
                    SideCache<R> sc = SideCache<R>{nullptr, 0}) {
    int q = i * G.stride + slot;
    int j = G.nj[q];
    int p = pidx(G.type[i], G.type[j]);
    R ux = G.dx[q], uy = G.dy[q], uz = G.dz[q], r = G.r[q], ir = G.ir[q];
    R w = G.w[q], dw = G.dw[q];
    R eR = exp_(-P.alpha[p] * r);
    R qr = R(1) + P.Q[p] * ir;
    R AeR = P.A[p] * eR;
    R fR = w * qr * AeR;
    R dfR = dw * qr * AeR - w * P.Q[p] * ir * ir * AeR - P.alpha[p] * fR;
    R sB = 0, dsB = 0;
    for (int m = 0; m < P.nB[p]; m++) {
        R e = P.B[p][m] * exp_(-P.beta[p][m] * r);
        sB += e;
        dsB -= P.beta[p][m] * e;
    }
    R fA = -w * sB;
    R dfA = -dw * sB - w * dsB;
    R gux = 0, guy = 0, guz = 0, gumag = 0;
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    R b = bond_order<R, true>(P, G, i, j, ux, uy, uz, r, ir, fA, sink, gux, guy, guz, gumag,
                              fix, fiy, fiz, fjx, fjy, fjz, nullptr, sc);
    R dEdr = dfR + b * dfA + gumag;
    R e = dEdr * ir;
    gux += e * ux; guy += e * uy; guz += e * uz;
    // vector u runs from i to j
    double gx = (double)gux, gy = (double)guy, gz = (double)guz;
    atomic_add(sink.f + i, fix + gx); atomic_add(sink.f + sink.n + i, fiy + gy); atomic_add(sink.f + 2 * sink.n + i, fiz + gz);
    atomic_add(sink.f + j, fjx - gx); atomic_add(sink.f + sink.n + j, fjy - gy); atomic_add(sink.f + 2 * sink.n + j, fjz - gz);
    if (sink.virial) {
        sink.W[0] -= (double)ux * gx; sink.W[1] -= (double)uy * gy; sink.W[2] -= (double)uz * gz;
        sink.W[3] -= (double)ux * gy; sink.W[4] -= (double)ux * gz; sink.W[5] -= (double)uy * gz;
    }
    return (double)(fR + b * fA);
}

// ------------------------------------------------------------------ torsion (Alg. 2)
// omega is the dihedral angle with trans = pi; cos^2(omega/2) = (1 + cos omega)/2
template <class R, class GT>
HD double torsion_bond(const DevParams<R>& P, const GT& G, int i, int slot, Sink& sink) {
    int q = i * G.stride + slot;
    int j = G.nj[q];
    R ux = G.dx[q], uy = G.dy[q], uz = G.dz[q];
    R wij = G.w[q], dwij = G.dw[q];
    R inv_u = G.ir[q];
    double E = 0;
    bool any = false;
    R gux = 0, guy = 0, guz = 0;
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    int ni = G.cnt[i], nj = G.cnt[j];
    int sj = slot_of(G, i, j), si_ = slot_of(G, j, i);
    int mi = ni - (sj < MAXN), mj = nj - (si_ < MAXN);
    for (int ta = 0; ta < mi; ta++) {
        int a = ta + (ta >= sj);
        int qa = i * G.stride + a;
        int k = G.nj[qa];
        R ax = G.dx[qa], ay = G.dy[qa], az = G.dz[qa];
        R wik = G.w[qa], dwik = G.dw[qa];
        R inv_ra = G.ir[qa];
        R csi = (ux * ax + uy * ay + uz * az) * inv_u * inv_ra;
        R dsi;
        R si = guardf<R>(P, csi, dsi);
        if (is_zero(si)) continue;
        R n1x = uy * az - uz * ay, n1y = uz * ax - ux * az, n1z = ux * ay - uy * ax;
        R n1s = n1x * n1x + n1y * n1y + n1z * n1z;
        R in1s = rcp_(n1s);
        for (int tb = 0; tb < mj; tb++) {
            int b = tb + (tb >= si_);
            int qb = j * G.stride + b;
            int l = G.nj[qb];
            if (l == k) continue;              // a three-ring
            R bx = G.dx[qb], by = G.dy[qb], bz = G.dz[qb];
            R wjl = G.w[qb], dwjl = G.dw[qb];
            R inv_rb = G.ir[qb];
            R csj = -(ux * bx + uy * by + uz * bz) * inv_u * inv_rb;
            R dsj;
            R sj = guardf<R>(P, csj, dsj);
            if (is_zero(sj)) continue;
            R n2x = uy * bz - uz * by, n2y = uz * bx - ux * bz, n2z = ux * by - uy * bx;
            R n2s = n2x * n2x + n2y * n2y + n2z * n2z;
            R inv12 = rsqrt_(n1s * n2s);
            R in2s = inv12 * inv12 * n1s;
            R cw = (n1x * n2x + n1y * n2y + n1z * n2z) * inv12;
            R h = R(0.5) * (R(1) + cw);
            R h2 = h * h, h4 = h2 * h2;
            R eps = P.teps[(G.type[k] == 1) + (G.type[l] == 1)];
            R Vt = eps * (R(256.0 / 405.0) * h4 * h - R(0.1));
            R dVdcw = eps * R(256.0 / 405.0) * R(2.5) * h4;
            R wprod = wik * wij * wjl;
            R ss = si * sj;
            E += (double)(wprod * ss * Vt);
            any = true;
            R dcw = wprod * ss * dVdcw;
            R sV = ss * Vt;
            R dwi = dwik * wij * wjl * sV;
            R dwj = wik * wij * dwjl * sV;
            R dwm = wik * dwij * wjl * sV;
            R dci = wprod * sj * dsi * Vt;
            R dcj = wprod * si * dsj * Vt;
            R c1 = dcw * cw * in1s, c2 = dcw * cw * in2s, c12 = dcw * inv12;
            R g1x = c12 * n2x - c1 * n1x, g1y = c12 * n2y - c1 * n1y, g1z = c12 * n2z - c1 * n1z;
            R g2x = c12 * n1x - c2 * n2x, g2y = c12 * n1y - c2 * n2y, g2z = c12 * n1z - c2 * n2z;
            gux += ay * g1z - az * g1y + by * g2z - bz * g2y;
            guy += az * g1x - ax * g1z + bz * g2x - bx * g2z;
            guz += ax * g1y - ay * g1x + bx * g2y - by * g2x;
            R gax = g1y * uz - g1z * uy, gay = g1z * ux - g1x * uz, gaz = g1x * uy - g1y * ux;
            R gbx = g2y * uz - g2z * uy, gby = g2z * ux - g2x * uz, gbz = g2x * uy - g2y * ux;
            R ea = dwi * inv_ra, eb = dwj * inv_rb, em = dwm * inv_u;
            gax += ea * ax; gay += ea * ay; gaz += ea * az;
            gbx += eb * bx; gby += eb * by; gbz += eb * bz;
            gux += em * ux; guy += em * uy; guz += em * uz;
            R i1 = dci * inv_u * inv_ra, i2 = dci * csi * inv_ra * inv_ra, i3 = dci * csi * inv_u * inv_u;
            gax += i1 * ux - i2 * ax; gay += i1 * uy - i2 * ay; gaz += i1 * uz - i2 * az;
            gux += i1 * ax - i3 * ux; guy += i1 * ay - i3 * uy; guz += i1 * az - i3 * uz;
            R j1 = dcj * inv_u * inv_rb, j2 = dcj * csj * inv_rb * inv_rb, j3 = dcj * csj * inv_u * inv_u;
            gbx += -j1 * ux - j2 * bx; gby += -j1 * uy - j2 * by; gbz += -j1 * uz - j2 * bz;
            gux += -j1 * bx - j3 * ux; guy += -j1 * by - j3 * uy; guz += -j1 * bz - j3 * uz;
            sink.half(k, ax, ay, az, gax, gay, gaz, fix, fiy, fiz);
            sink.half(l, bx, by, bz, gbx, gby, gbz, fjx, fjy, fjz);
        }
    }
    if (!any) return 0.0;
    double gx = (double)gux, gy = (double)guy, gz = (double)guz;
    atomic_add(sink.f + i, fix + gx); atomic_add(sink.f + sink.n + i, fiy + gy); atomic_add(sink.f + 2 * sink.n + i, fiz + gz);
    atomic_add(sink.f + j, fjx - gx); atomic_add(sink.f + sink.n + j, fjy - gy); atomic_add(sink.f + 2 * sink.n + j, fjz - gz);
    if (sink.virial) {
        sink.W[0] -= (double)ux * gx; sink.W[1] -= (double)uy * gy; sink.W[2] -= (double)uz * gz;
        sink.W[3] -= (double)ux * gy; sink.W[4] -= (double)ux * gz; sink.W[5] -= (double)uy * gz;
    }
    return E;
}

// The same torsion of one bond with its double sum factored.  Every term of
// the gradient is linear in its (k, l) pieces: the gradient with respect to
// n1 = u x a_k, summed over l, is wij [sum_l q n2_l - |n1|^-2 (sum_l dcw cos w) n1]
// (q = dcw / (|n1| |n2|)), and likewise for n2 summed over k; the guard and
// weight derivatives collect sum_l w_jl s_j V and sum_k w_ik s_i V.  So each
// (k, l) pair forms only cos w, V, dV/dcos w and those sums; the cross
// products with u and the forces on k (on l) are applied once per
// neighbour.  The l-side values and sums of up to TORS_L neighbours of j sit
// in a per-thread store in shared memory ([value][slot][thread]); a j with
// more neighbours takes torsion_bond.  GT: the graph view (the FP64 short
// list read as double-float in the DF64 kernel).
constexpr int TORS_L = 3, TORS_V = 12;      // slots, values per slot
template <class R> struct TorsStore {
    R* p;
    int stride;
    HD R& at(int t, int v) const { return p[(t * TORS_V + v) * stride]; }
};
template <class R, class GT = Graph<R>>
HD double torsion_bond_f(const DevParams<R>& P, const GT& G, int i, int slot, Sink& sink, TorsStore<R> S) {
    int q = i * G.stride + slot;
    int j = G.nj[q];
    int ni = G.cnt[i], nj = G.cnt[j];
    int sj_ = slot_of(G, i, j), si_ = slot_of(G, j, i);
    int mi = ni - (sj_ < MAXN), mj = nj - (si_ < MAXN);
    if (mj > TORS_L) return torsion_bond<R>(P, G, i, slot, sink);
    R ux = G.dx[q], uy = G.dy[q], uz = G.dz[q];
    R wij = G.w[q], dwij = G.dw[q];
    R inv_u = G.ir[q];
    // the l side: n2 = u x b_l (0-2) and 1/|n2| (3), w_jl s_j (4), s_j (5) and
    // ds_j (6); then the sums over k: q n1_k (7-9), dcw cos w (10), w_ik s_i V (11)
    for (int tb = 0; tb < mj; tb++) {
        int qb = j * G.stride + tb + (tb >= si_);
        R bx = G.dx[qb], by = G.dy[qb], bz = G.dz[qb];
        R csj = -(ux * bx + uy * by + uz * bz) * inv_u * G.ir[qb];
        R dsj;
        R sj = guardf<R>(P, csj, dsj);
        R n2x = uy * bz - uz * by, n2y = uz * bx - ux * bz, n2z = ux * by - uy * bx;
        S.at(tb, 0) = n2x; S.at(tb, 1) = n2y; S.at(tb, 2) = n2z;
        S.at(tb, 3) = is_zero(sj) ? R(0) : rsqrt_(n2x * n2x + n2y * n2y + n2z * n2z);
        S.at(tb, 4) = G.w[qb] * sj; S.at(tb, 5) = sj; S.at(tb, 6) = dsj;
        for (int v = 7; v < TORS_V; v++) S.at(tb, v) = R(0);
    }
    bool any = false;
    double Ssum = 0;                 // sum over (k, l) of w_ik s_i w_jl s_j V
    R gux = 0, guy = 0, guz = 0;
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    for (int ta = 0; ta < mi; ta++) {
        int qa = i * G.stride + ta + (ta >= sj_);
        int k = G.nj[qa];
        R ax = G.dx[qa], ay = G.dy[qa], az = G.dz[qa];
        R wik = G.w[qa], inv_ra = G.ir[qa];
        R csi = (ux * ax + uy * ay + uz * az) * inv_u * inv_ra;
        R dsi;
        R si = guardf<R>(P, csi, dsi);
        if (is_zero(si)) continue;
        R n1x = uy * az - uz * ay, n1y = uz * ax - ux * az, n1z = ux * ay - uy * ax;
        R rn1 = rsqrt_(n1x * n1x + n1y * n1y + n1z * n1z);
        R wsi = wik * si;
        int tk = G.type[k] == 1;
        R Ax = 0, Ay = 0, Az = 0, Bk = 0, Ik = 0;     // sum_l q n2_l, sum_l dcw cos w, sum_l w_jl s_j V
        bool kany = false;
        for (int tb = 0; tb < mj; tb++) {
            int l = G.nj[j * G.stride + tb + (tb >= si_)];
            if (l == k) continue;              // a three-ring
            if (is_zero(S.at(tb, 5))) continue;
            R n2x = S.at(tb, 0), n2y = S.at(tb, 1), n2z = S.at(tb, 2);
            R inv12 = rn1 * S.at(tb, 3);
            R cw = (n1x * n2x + n1y * n2y + n1z * n2z) * inv12;
            R h = R(0.5) * (R(1) + cw);
            R h2 = h * h, h4 = h2 * h2;
            R eps = P.teps[tk + (G.type[l] == 1)];
            R Vt = eps * (R(256.0 / 405.0) * h4 * h - R(0.1));
            R dVdcw = eps * R(256.0 / 405.0) * R(2.5) * h4;
            R wsj = S.at(tb, 4);
            R wkl = wsi * wsj;
            Ssum += (double)(wkl * Vt);
            Ik += wsj * Vt;
            S.at(tb, 11) += wsi * Vt;
            R dcw = wkl * dVdcw;             // times w_ij below
            R qq = dcw * inv12, dd = dcw * cw;
            Ax += qq * n2x; Ay += qq * n2y; Az += qq * n2z; Bk += dd;
            S.at(tb, 7) += qq * n1x; S.at(tb, 8) += qq * n1y; S.at(tb, 9) += qq * n1z; S.at(tb, 10) += dd;
            kany = true;
        }
        if (!kany) continue;
        any = true;
        // the gradient with respect to n1, then to a_k and u through n1 = u x a_k
        R c1 = rn1 * rn1 * Bk;
        R g1x = wij * (Ax - c1 * n1x), g1y = wij * (Ay - c1 * n1y), g1z = wij * (Az - c1 * n1z);
        R gax = g1y * uz - g1z * uy, gay = g1z * ux - g1x * uz, gaz = g1x * uy - g1y * ux;
        gux += ay * g1z - az * g1y; guy += az * g1x - ax * g1z; guz += ax * g1y - ay * g1x;
        // the weight w_ik and the guard s_i
        R ea = G.dw[qa] * wij * si * Ik * inv_ra;
        gax += ea * ax; gay += ea * ay; gaz += ea * az;
        R dci = wik * wij * dsi * Ik;
        R i1 = dci * inv_u * inv_ra, i2 = dci * csi * inv_ra * inv_ra, i3 = dci * csi * inv_u * inv_u;
        gax += i1 * ux - i2 * ax; gay += i1 * uy - i2 * ay; gaz += i1 * uz - i2 * az;
        gux += i1 * ax - i3 * ux; guy += i1 * ay - i3 * uy; guz += i1 * az - i3 * uz;
        sink.half(k, ax, ay, az, gax, gay, gaz, fix, fiy, fiz);
    }
    if (!any) return 0.0;
    for (int tb = 0; tb < mj; tb++) {
        R sj = S.at(tb, 5);
        if (is_zero(sj)) continue;
        int qb = j * G.stride + tb + (tb >= si_);
        R bx = G.dx[qb], by = G.dy[qb], bz = G.dz[qb];
        R inv_rb = G.ir[qb];
        R n2x = S.at(tb, 0), n2y = S.at(tb, 1), n2z = S.at(tb, 2), rn2 = S.at(tb, 3);
        R c2 = rn2 * rn2 * S.at(tb, 10), Jl = S.at(tb, 11);
        R g2x = wij * (S.at(tb, 7) - c2 * n2x), g2y = wij * (S.at(tb, 8) - c2 * n2y), g2z = wij * (S.at(tb, 9) - c2 * n2z);
        R gbx = g2y * uz - g2z * uy, gby = g2z * ux - g2x * uz, gbz = g2x * uy - g2y * ux;
        gux += by * g2z - bz * g2y; guy += bz * g2x - bx * g2z; guz += bx * g2y - by * g2x;
        R eb = wij * G.dw[qb] * sj * Jl * inv_rb;
        gbx += eb * bx; gby += eb * by; gbz += eb * bz;
        R csj = -(ux * bx + uy * by + uz * bz) * inv_u * inv_rb;
        R dcj = wij * G.w[qb] * S.at(tb, 6) * Jl;
        R j1 = dcj * inv_u * inv_rb, j2 = dcj * csj * inv_rb * inv_rb, j3 = dcj * csj * inv_u * inv_u;
        gbx += -j1 * ux - j2 * bx; gby += -j1 * uy - j2 * by; gbz += -j1 * uz - j2 * bz;
        gux += -j1 * bx - j3 * ux; guy += -j1 * by - j3 * uy; guz += -j1 * bz - j3 * uz;
        sink.half(G.nj[qb], bx, by, bz, gbx, gby, gbz, fjx, fjy, fjz);
    }
    // the bond weight w_ij
    R em = dwij * (R)Ssum * inv_u;
    gux += em * ux; guy += em * uy; guz += em * uz;
    double gx = (double)gux, gy = (double)guy, gz = (double)guz;
    atomic_add(sink.f + i, fix + gx); atomic_add(sink.f + sink.n + i, fiy + gy); atomic_add(sink.f + 2 * sink.n + i, fiz + gz);
    atomic_add(sink.f + j, fjx - gx); atomic_add(sink.f + sink.n + j, fjy - gy); atomic_add(sink.f + 2 * sink.n + j, fjz - gz);
    if (sink.virial) {
        sink.W[0] -= (double)ux * gx; sink.W[1] -= (double)uy * gy; sink.W[2] -= (double)uz * gz;
        sink.W[3] -= (double)ux * gy; sink.W[4] -= (double)ux * gz; sink.W[5] -= (double)uy * gz;
    }
    return (double)wij * Ssum;
}

// ------------------------------------------------------------------ C_ij paths (Sec. 2.1.2, 4.3)
// A connectivity map of atom i holds, for every atom reachable over at most
// three REBO bonds (keyed by atom and periodic image), the largest path
// weight and the path realising it (slots of the bonds along the path).
HD long long map_key(int j, int img) { return ((long long)j << 24) | (long long)(img & 0xffffff); }
HD int path_pack(int len, int a, int b, int c) { return len | (a << 4) | (b << 8) | (c << 12); }
HD int path_len(int p) { return p & 15; }
HD int path_a(int p) { return (p >> 4) & 15; }
HD int path_b(int p) { return (p >> 8) & 15; }
HD int path_c(int p) { return (p >> 12) & 15; }

template <class R> struct PathMap {
    int cap;
    int* cnt;            // entries per atom
    R* wt;               // [n * cap]: C = 1 - largest path weight
    int* path;           // [n * cap]: the bonds of that path
    int hbits;           // the hash table of atom i: 2^hbits slots from (i << hbits)
    unsigned long long* ht;   // slot = ((key + 1) << MAP_IDX_BITS) | entry, 0 = empty
};

// The per-atom hash table of map keys (open addressing, linear probing): it
// has at least twice as many slots as entries, so every probe sequence meets
// an empty slot, after about 1.2 probes on average.  Keys are below 2^52
// (atoms below 2^28), entries below 2^12.
constexpr int MAP_IDX_BITS = 12;
constexpr int MAP_MAX_ATOMS = 1 << 28;
HD unsigned map_hash(long long key, int hbits) {
    return (unsigned)(((unsigned long long)key * 0x9E3779B97F4A7C15ull) >> (64 - hbits));
}
// the entry of (atom, image) in the map of atom i, or -1
template <class R> HD int map_find(const PathMap<R>& M, int i, long long key) {
    const unsigned long long* T = M.ht + ((size_t)i << M.hbits);
    unsigned mask = (1u << M.hbits) - 1, h = map_hash(key, M.hbits);
    unsigned long long want = (unsigned long long)(key + 1);
    for (unsigned probe = 0; probe <= mask; probe++) {
        unsigned long long slot = T[h];
        if (slot == 0ull) return -1;
        if ((slot >> MAP_IDX_BITS) == want) return (int)(slot & ((1u << MAP_IDX_BITS) - 1));
        h = (h + 1) & mask;
    }
    return -1;
}

// Ties: larger weight (smaller C), then the shorter path, then the smaller k,
// then the smaller l.  The map stores C = 1 - weight, formed from the 1 - w of
// each bond (1 - w1 w2 = (1 - w1) + w1 (1 - w2), and so on), which keeps the
// relative precision of small C in FP32.
HD bool path_better(double c, int len, int k, int l, double c0, int len0, int k0, int l0) {
    if (c != c0) return c < c0;
    if (len != len0) return len < len0;
    if (k != k0) return k < k0;
    return l < l0;
}

// 256-bit membership filter of the atoms already in a map (in registers
// while the map is built): a clear bit means a new atom
HD int map_bit(int atom) { return (int)(((unsigned)atom * 2654435761u) >> 24); }

template <class R>
HD int build_path_map(const Graph<R>& G, PathMap<R>& M, int i) {
    int base = i * M.cap;
    int count = 0, overflow = 0;
    unsigned long long* T = M.ht + ((size_t)i << M.hbits);      // cleared by the caller
    unsigned mask = (1u << M.hbits) - 1;
    // the filter, and for tables of up to 256 slots the occupied slots, in
    // registers: a new atom (most atoms: bonds form trees) then takes an empty
    // slot without reading the table back
    unsigned long long filt[4] = {0, 0, 0, 0}, occ[4] = {0, 0, 0, 0};
    bool occ_in_regs = M.hbits <= 8;
    auto insert = [&](int atom, int img, R c, int len, int k, int l, int code) {
        long long key = map_key(atom, img);
        unsigned long long want = (unsigned long long)(key + 1);
        unsigned h = map_hash(key, M.hbits);
        int bit = map_bit(atom);
        bool seen = (filt[bit >> 6] >> (bit & 63)) & 1ull;
        for (unsigned probe = 0; seen && probe <= mask; probe++) {
            unsigned long long slot = T[h];
            if (slot == 0ull) break;
            if ((slot >> MAP_IDX_BITS) == want) {          // seen: keep the better path
                int e = (int)(slot & ((1u << MAP_IDX_BITS) - 1));
                int p0 = M.path[base + e];
                int k0 = path_len(p0) >= 2 ? G.nj[i * G.stride + path_a(p0)] : -1;
                int l0 = -1;
                if (path_len(p0) == 3) l0 = G.nj[G.nj[i * G.stride + path_a(p0)] * G.stride + path_b(p0)];
                if (path_better((double)c, len, k, l, (double)M.wt[base + e], path_len(p0), k0, l0)) {
                    M.wt[base + e] = c;
                    M.path[base + e] = code;
                }
                return;
            }
            h = (h + 1) & mask;
        }
        if (count < M.cap) {
            if (occ_in_regs) {
                h = map_hash(key, M.hbits);
                while ((occ[h >> 6] >> (h & 63)) & 1ull) h = (h + 1) & mask;     // at most half full
                occ[h >> 6] |= 1ull << (h & 63);
            } else if (!seen) {
                for (unsigned probe = 0; probe <= mask && T[h] != 0ull; probe++) h = (h + 1) & mask;
            }
            T[h] = (want << MAP_IDX_BITS) | (unsigned long long)count;
            M.wt[base + count] = c;
            M.path[base + count] = code;
            count++;
            filt[bit >> 6] |= 1ull << (bit & 63);
        } else {
            overflow++;
        }
    };
    int ni = G.cnt[i];
    for (int a = 0; a < ni; a++) {
        int qa = i * G.stride + a;
        int k = G.nj[qa];
        int Sk = G.nimg[qa];
        R w1 = G.w[qa], c1 = G.omw[qa];
        insert(k, Sk, c1, 1, -1, -1, path_pack(1, a, 0, 0));
        int nk = G.cnt[k];
        for (int b = 0; b < nk; b++) {
            int qb = k * G.stride + b;
            int l = G.nj[qb];
            if (l == i) continue;
            int Sl = img_add(Sk, G.nimg[qb]);
            R w2 = w1 * G.w[qb];
            R c2 = c1 + w1 * G.omw[qb];
            insert(l, Sl, c2, 2, k, -1, path_pack(2, a, b, 0));
            int nl = G.cnt[l];
            for (int c = 0; c < nl; c++) {
                int qc = l * G.stride + c;
                int m = G.nj[qc];
                if (m == i || m == k) continue;
                int Sm = img_add(Sl, G.nimg[qc]);
                insert(m, Sm, c2 + w2 * G.omw[qc], 3, k, l, path_pack(3, a, b, c));
            }
        }
    }
    M.cnt[i] = count;
    return overflow;
}

// forces of dE/dwmax on the bonds of the path stored for atom i
template <class R, class SinkT = Sink>
HD void path_forces(const Graph<R>& G, int i, int code, R dEdw, SinkT& sink, double& fix, double& fiy, double& fiz) {
    int len = path_len(code);
    int q[3], from[3];
    q[0] = i * G.stride + path_a(code); from[0] = i;
    int k = G.nj[q[0]];
    if (len >= 2) { q[1] = k * G.stride + path_b(code); from[1] = k; }
    if (len == 3) { int l = G.nj[q[1]]; q[2] = l * G.stride + path_c(code); from[2] = l; }
    R w[3], dw[3];
    for (int s = 0; s < len; s++) { w[s] = G.w[q[s]]; dw[s] = G.dw[q[s]]; }
    for (int s = 0; s < len; s++) {
        if (is_zero(dw[s])) continue;
        R other = R(1);
        for (int t = 0; t < len; t++) if (t != s) other *= w[t];
        R c = dEdw * other * dw[s] * G.ir[q[s]];
        R gx = c * G.dx[q[s]], gy = c * G.dy[q[s]], gz = c * G.dz[q[s]];
        if (from[s] == i) sink.half(G.nj[q[s]], G.dx[q[s]], G.dy[q[s]], G.dz[q[s]], gx, gy, gz, fix, fiy, fiz);
        else sink.pair(from[s], G.nj[q[s]], G.dx[q[s]], G.dy[q[s]], G.dz[q[s]], gx, gy, gz);
    }
}

// ------------------------------------------------------------------ LJ (Alg. 3)
// V^LJ = 4 eps [(s/r)^12 - (s/r)^6] times the C^1 cubic cut-off, from r^2;
// dVr = (dV/dr)/r.  The cut-off switch is evaluated without a branch (t is
// clamped at 0, where it is the identity), so lanes of a warp never diverge.
// ir = 1/r is given.
template <class R> HD R vlj(const DevParams<R>& P, int p, R r2, R ir, R& dVr) {
    R r = r2 * ir;
    R v, dvr;
    if (P.kind == 0) {
        R ir2 = ir * ir;
        R s2 = P.sig2[p] * ir2;
        R s6 = s2 * s2 * s2;
        R t6 = P.eps4[p] * s6;
        v = t6 * s6 - t6;
        dvr = t6 * ir2 * (R(6) - R(12) * s6);
    } else {                         // Morse (AIREBO-M): eps (e^2 - 2 e), e = exp(-alpha (r - r_e))
        R e = exp_(-P.malpha[p] * (r - P.mre[p]));
        v = P.meps[p] * (e * e - R(2) * e);
        dvr = R(2) * P.malpha[p] * P.meps[p] * e * (R(1) - e) * ir;
    }
    R t = (r - P.swlo[p]) * P.swinv[p];
    t = gt_(t, R(0)) ? t : R(0);
    R so = R(1) - t * t * (R(3) - R(2) * t);
    R dso = R(-6) * t * (R(1) - t) * P.swinv[p];
    dVr = dvr * so + v * dso * ir;
    return v * so;
}
template <class R> HD R vlj(const DevParams<R>& P, int p, R r2, R& dVr) { return vlj<R>(P, p, r2, rsqrt_(r2), dVr); }

// dV/d(eps) and dV/d(sigma) of the inter-molecular pair term (with its cut-off
// switch) at r; eps is lj.epsilon (Lennard-Jones) or morse.epsilon (Morse).
template <class R> HD void vlj_param_grad(const DevParams<R>& P, int p, R r, R& dV_deps, R& dV_dsig) {
    R sg = P.sigma[p];
    R t = (r - P.swlo[p]) * P.swinv[p];
    t = gt_(t, R(0)) ? t : R(0);
    R so = R(1) - t * t * (R(3) - R(2) * t);
    R dso_dt = R(-6) * t * (R(1) - t);
    R dt_dsig = t > R(0) ? -r * P.swinv[p] / sg : R(0);        // t = (r/sigma - 2.7)/0.3
    R v, dv_dsig, eps;
    if (P.kind == 0) {
        R s6 = (sg / r) * (sg / r);
        s6 = s6 * s6 * s6;
        v = P.eps4[p] * (s6 * s6 - s6);
        dv_dsig = P.eps4[p] * (R(12) * s6 * s6 - R(6) * s6) / sg;
        eps = P.eps4[p] * R(0.25);
    } else {
        R e = exp_(-P.malpha[p] * (r - P.mre[p]));
        v = P.meps[p] * (e * e - R(2) * e);
        dv_dsig = R(0);
        eps = P.meps[p];
    }
    dV_deps = v * so / eps;
    dV_dsig = dv_dsig * so + v * dso_dt * dt_dsig;
}

// Energy and forces of one LJ pair with S_r = 0 (C and its path known).
template <class R>
HD void lj_eval(const DevParams<R>& P, const Graph<R>& G, int i, int p, int j, double dx, double dy, double dz,
                R C, int code, Sink& sink, double& fix, double& fiy, double& fiz, double& E) {
    R rx = (R)dx, ry = (R)dy, rz = (R)dz;
    R r2 = rx * rx + ry * ry + rz * rz;
    R dVr;
    R V = vlj<R>(P, p, r2, dVr);
    E += (double)(C * V);
    double c = (double)(C * dVr);
    sink.half(j, dx, dy, dz, c * dx, c * dy, c * dz, fix, fiy, fiz);
    if (code >= 0) path_forces<R>(G, i, code, -V, sink, fix, fiy, fiz);
    if (sink.pgrad) {
        R de, ds;
        vlj_param_grad<R>(P, p, sqrt_(r2), de, ds);
        sink.G[p] += (double)(C * de);
        sink.G[3 + p] += (double)(C * ds);
    }
}

// The Lennard-Jones pair in powers of 1/r^2, with A = 4 eps sigma^6 and
// B = 4 eps sigma^12 of one species pair: V = (1/r^6)(B/r^6 - A) and
// (dV/dr)/r = (1/r^8)(6 A - 12 B/r^6).  Written so, V and (dV/dr)/r take the
// fewest FP64 instructions (ten from 1/r^2 to both, with the energy sum).
struct LjPow {
    double A, B, A6, B12;        // A, B, 6 A, -12 B
};
HD LjPow lj_pow(double eps4, double sig2) {
    double A = eps4 * sig2 * sig2 * sig2, B = A * sig2 * sig2 * sig2;
    return LjPow{A, B, 6.0 * A, -12.0 * B};
}

// The common LJ pair: C = 1, no path, r inside 2.7 sigma (no cut-off switch):
// V and (dV/dr)/r from 1/r^2 alone.
template <class R>
HD void lj_eval_inner(const LjPow& K, int j, double dx, double dy, double dz, R r2, Sink& sink,
                      double& fix, double& fiy, double& fiz, double& E) {
    R ir2 = rcp_(r2);
    R ir6 = ir2 * ir2 * ir2;
    E += (double)(ir6 * ((R)K.B * ir6 - (R)K.A));
    double c = (double)(ir6 * ir2 * ((R)K.A6 + (R)K.B12 * ir6));
    sink.half(j, dx, dy, dz, c * dx, c * dy, c * dz, fix, fiy, fiz);
}

// C = 1, no path, r inside the cut-off switch (Lennard-Jones), or any
// C = 1 pair without a path (Morse).
template <class R>
HD void lj_eval_switch(const DevParams<R>& P, const LjPow& K, int p, int j, double dx, double dy, double dz, R r2,
                       Sink& sink, double& fix, double& fiy, double& fiz, double& E) {
    double c;
    if (P.kind == 0) {
        R ir = rsqrt_(r2);
        R ir2 = ir * ir;
        R ir6 = ir2 * ir2 * ir2;
        R v = ir6 * ((R)K.B * ir6 - (R)K.A);
        R dvr = ir6 * ir2 * ((R)K.A6 + (R)K.B12 * ir6);
        R t = (r2 * ir - P.swlo[p]) * P.swinv[p];          // > 0 in this class
        R so = R(1) - t * t * (R(3) - R(2) * t);
        R dso = R(-6) * t * (R(1) - t) * P.swinv[p];
        E += (double)(v * so);
        c = (double)(dvr * so + v * dso * ir);
    } else {
        R dVr;
        E += (double)vlj<R>(P, p, r2, dVr);
        c = (double)dVr;
    }
    sink.half(j, dx, dy, dz, c * dx, c * dy, c * dz, fix, fiy, fiz);
}

// The tests of one LJ pair i -> (j, image) with FP64 displacement d: the
// cut-off, and the C_ij lookup in i's connectivity map.  Returns
//   0: beyond the cut-off, or C = 0;
//   1: C = 1, no path, inside 2.7 sigma (lj_eval_inner);
//   2: to be queued for b* (S_r != 0);
//   3: C = 1, no path, inside the cut-off switch, or any such Morse pair (lj_eval_switch);
//   4: 0 < C < 1 along a path (lj_eval).
// C, the path code and the map entry are returned.
// The squared-distance thresholds of the pair tests for one species pair, in
// the type T of the squared distance that is tested against them.
template <class T> struct LjCuts {
    T rc2, rpath2, srhi2, swlo2;
};

template <class R, class T>
HD int lj_classify_c(const DevParams<R>& P, const PathMap<R>& M, int i, int j, int img, T r2, const LjCuts<T>& k,
                     R& C, int& code, int& mi, bool general) {
    mi = -1; code = -1; C = R(1);
    if (!lt_nonneg(r2, k.rc2)) return 0;
    if (lt_nonneg(r2, k.rpath2)) {
        mi = map_find<R>(M, i, map_key(j, img));
        if (mi >= 0) {
            C = M.wt[(size_t)i * M.cap + mi];
            if (!gt_(C, R(0))) return 0;
            code = M.path[(size_t)i * M.cap + mi];
        }
    }
    if (lt_nonneg(r2, k.srhi2)) return 2;
    if (mi >= 0 || general) return 4;
    return (P.kind != 0 || lt_nonneg(k.swlo2, r2)) ? 3 : 1;
}

template <class R>
HD int lj_classify(const DevParams<R>& P, const PathMap<R>& M, int i, int p, int j, int img, R r2,
                   R& C, int& code, int& mi, bool general = false) {
    LjCuts<R> k{P.rc2[p], P.rpath2, P.Srhi2[p], P.swlo2[p]};
    return lj_classify_c<R, R>(P, M, i, j, img, r2, k, C, code, mi, general);
}

// b* pair: (S_r S_b + 1 - S_r) C V for the pair i -> (j, image) with
// displacement d; C and its path given, and S_b(b*) with its derivative
// already known.  Applies every force except the one through db*, which the
// reverse bond order applies where dS_b != 0.  1/r, V and (dV/dr)/r of the
// pair are given, and S_r with dS_r/dr.
template <class R>
HD double bstar_finish_v(const DevParams<R>& P, const Graph<R>& G, int i, int j, R dx, R dy, R dz, R r2,
                         R inv_r, R V, R dVr, R Sr, R dSr, R C, int path_code, R Sb, R dSb, Sink& sink) {
    int p = pidx(G.type[i], G.type[j]);
    R r = r2 * inv_r;
    R factor = Sr * Sb + R(1) - Sr;
    R E = factor * C * V;
    R dEdr_r = (dSr * (Sb - R(1))) * C * V * inv_r + factor * C * dVr;   // (dE/dr)/r
    double gx = (double)(dEdr_r * dx), gy = (double)(dEdr_r * dy), gz = (double)(dEdr_r * dz);
    double fix = 0, fiy = 0, fiz = 0;
    if (path_code >= 0) path_forces<R>(G, i, path_code, -factor * V, sink, fix, fiy, fiz);
    if (sink.pgrad) {
        R de, ds;
        vlj_param_grad<R>(P, p, r, de, ds);
        // S_r = S((r/sigma - lo)/(hi - lo)) also depends on sigma
        R dSr_dsig = dSr * (-r / P.sigma[p]);
        sink.G[p] += (double)(C * factor * de);
        sink.G[3 + p] += (double)(C * (factor * ds + V * (Sb - R(1)) * dSr_dsig));
    }
    atomic_add(sink.f + i, fix + gx); atomic_add(sink.f + sink.n + i, fiy + gy); atomic_add(sink.f + 2 * sink.n + i, fiz + gz);
    atomic_add(sink.f + j, -gx); atomic_add(sink.f + sink.n + j, -gy); atomic_add(sink.f + 2 * sink.n + j, -gz);
    if (sink.virial) {
        sink.W[0] -= (double)dx * gx; sink.W[1] -= (double)dy * gy; sink.W[2] -= (double)dz * gz;
        sink.W[3] -= (double)dx * gy; sink.W[4] -= (double)dx * gz; sink.W[5] -= (double)dy * gz;
    }
    return (double)E;
}

// the same, with 1/r, V, (dV/dr)/r and S_r evaluated here
template <class R>
HD double bstar_finish(const DevParams<R>& P, const Graph<R>& G, int i, int j, R dx, R dy, R dz, R r2,
                       R C, int path_code, R Sb, R dSb, Sink& sink) {
    int p = pidx(G.type[i], G.type[j]);
    R inv_r = rsqrt_(r2);
    R dVr;
    R V = vlj<R>(P, p, r2, inv_r, dVr);
    R dSr;
    R Sr = Sw<R>((r2 * inv_r - P.Srlo[p]) * P.Srinv[p], dSr);
    return bstar_finish_v<R>(P, G, i, j, dx, dy, dz, r2, inv_r, V, dVr, Sr, dSr * P.Srinv[p], C, path_code, Sb, dSb,
                             sink);
}

// b* of the pair i -> (j, image) with displacement d: the bond order of
// Eq. 4 at the fixed length r* along d (value only)
template <class R>
HD R bstar_value(const DevParams<R>& P, const Graph<R>& G, int i, int j, R dx, R dy, R dz, R r2, Sink& sink) {
    int p = pidx(G.type[i], G.type[j]);
    R inv_r = rsqrt_(r2);
    R rs = P.rstar[p];
    R ux = dx * inv_r * rs, uy = dy * inv_r * rs, uz = dz * inv_r * rs;
    R gux = 0, guy = 0, guz = 0, gumag = 0;
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    return bond_order_c<R, false>(P, G, i, j, ux, uy, uz, rs, rcp_(rs), R(0), sink, gux, guy, guz, gumag,
                                fix, fiy, fiz, fjx, fjy, fjz);
}

// S_b from b*: 1 below the transition, 0 above it
template <class R> HD R bstar_switch(const DevParams<R>& P, int p, R bs, R& dSb) {
    R dS;
    R Sb = Sw<R>((bs - P.bmin[p]) * P.binv[p], dS);
    dSb = dS * P.binv[p];
    return Sb;
}

// The whole b* pair in one pass: b* and its reverse (where dS_b != 0) in one
// bond-order evaluation, then the pair term.  Returns the energy; sets dsb
// when dS_b != 0.
template <class R>
HD double bstar_full(const DevParams<R>& P, const Graph<R>& G, int i, int j, R dx, R dy, R dz, R r2,
                     R C, int path_code, Sink& sink, bool& dsb, SideCache<R> sc = SideCache<R>{nullptr, 0}) {
    int p = pidx(G.type[i], G.type[j]);
    R inv_r = rsqrt_(r2);
    R r = r2 * inv_r;
    R dVr;
    R V = vlj<R>(P, p, r2, inv_r, dVr);
    R dSr;
    R Sr = Sw<R>((r - P.Srlo[p]) * P.Srinv[p], dSr);
    R rs = P.rstar[p];
    R ux = dx * inv_r * rs, uy = dy * inv_r * rs, uz = dz * inv_r * rs;
    R gux = 0, guy = 0, guz = 0, gumag = 0;
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    BstarSwitch<R> bsw{P.bmin[p], P.binv[p], Sr * C * V, R(0), R(0)};
    bond_order_c<R, true>(P, G, i, j, ux, uy, uz, rs, rcp_(rs), R(0), sink, gux, guy, guz, gumag,
                          fix, fiy, fiz, fjx, fjy, fjz, &bsw, sc);
    dsb = !is_zero(bsw.dSb);
    if (dsb) {
        // u = r* d/|d|: only the direction of d carries a gradient
        R ud = (gux * dx + guy * dy + guz * dz) * inv_r;
        R sc = rs * inv_r;
        double gx = (double)(sc * (gux - ud * dx * inv_r));
        double gy = (double)(sc * (guy - ud * dy * inv_r));
        double gz = (double)(sc * (guz - ud * dz * inv_r));
        atomic_add(sink.f + i, fix + gx); atomic_add(sink.f + sink.n + i, fiy + gy); atomic_add(sink.f + 2 * sink.n + i, fiz + gz);
        atomic_add(sink.f + j, fjx - gx); atomic_add(sink.f + sink.n + j, fjy - gy); atomic_add(sink.f + 2 * sink.n + j, fjz - gz);
        if (sink.virial) {
            sink.W[0] -= (double)dx * gx; sink.W[1] -= (double)dy * gy; sink.W[2] -= (double)dz * gz;
            sink.W[3] -= (double)dx * gy; sink.W[4] -= (double)dx * gz; sink.W[5] -= (double)dy * gz;
        }
    }
    return bstar_finish_v<R>(P, G, i, j, dx, dy, dz, r2, inv_r, V, dVr, Sr, dSr * P.Srinv[p], C, path_code, bsw.Sb,
                             bsw.dSb, sink);
}

// ------------------------------------------------------------------ parameter derivatives of the forces
// A factor of the LJ pair energy as a function of r and sigma: value, d/dr,
// d/dsigma and d^2/(dr dsigma).
template <class R> struct Rs { R v, r, s, rs; };

// The product of three such factors.
template <class R> HD Rs<R> rs_mul3(const Rs<R>& x, const Rs<R>& y, const Rs<R>& z) {
    Rs<R> o;
    o.v = x.v * y.v * z.v;
    o.r = x.r * y.v * z.v + x.v * y.r * z.v + x.v * y.v * z.r;
    o.s = x.s * y.v * z.v + x.v * y.s * z.v + x.v * y.v * z.s;
    o.rs = x.rs * y.v * z.v + x.s * y.r * z.v + x.s * y.v * z.r + x.r * y.s * z.v + x.v * y.rs * z.v +
           x.v * y.s * z.r + x.r * y.v * z.s + x.v * y.r * z.s + x.v * y.v * z.rs;
    return o;
}

// A factor that depends on r and sigma through r/sigma only: from its first
// and second r-derivatives, d/dsigma = -(r/sigma) d/dr and
// d^2/(dr dsigma) = -(1/sigma) d/dr - (r/sigma) d^2/dr^2.
template <class R> HD Rs<R> rs_scaled(R v, R dr, R drr, R r, R inv_sigma) {
    return Rs<R>{v, dr, -r * inv_sigma * dr, -inv_sigma * dr - r * inv_sigma * drr};
}

// The radial factors of the LJ pair energy E = C (g1 + g2 S_b) (Alg. 3):
// g1 = V S_out (1 - S_r), g2 = V S_out S_r, with their sigma-derivatives h1,
// h2, and the r-derivatives of all four.  The Lennard-Jones core, the cut-off
// switch S_out and S_r are functions of r/sigma; the Morse core does not
// depend on sigma.
template <class R>
HD void lj_radial_sigma(const DevParams<R>& P, int p, R r, Rs<R>& g1, Rs<R>& g2) {
    R isg = rcp_(P.sigma[p]);
    Rs<R> A;
    if (P.kind == 0) {
        R ir = rcp_(r);
        R u2 = P.sig2[p] * ir * ir;
        R u6 = u2 * u2 * u2, u12 = u6 * u6;
        R e4 = P.eps4[p];
        A = rs_scaled<R>(e4 * (u12 - u6), -e4 * (R(12) * u12 - R(6) * u6) * ir,
                         e4 * (R(156) * u12 - R(42) * u6) * ir * ir, r, isg);
    } else {
        R e = exp_(-P.malpha[p] * (r - P.mre[p]));
        R a = P.malpha[p], em = P.meps[p];
        A = Rs<R>{em * (e * e - R(2) * e), R(2) * a * em * (e - e * e), R(0), R(0)};   // no sigma in the core
    }
    // cut-off switch 1 - 3t^2 + 2t^3, t = (r - 2.7 sigma) / (0.3 sigma)
    R t = (r - P.swlo[p]) * P.swinv[p];
    Rs<R> B{R(1), R(0), R(0), R(0)};
    if (gt_(t, R(0))) {
        R w = P.swinv[p];
        B = rs_scaled<R>(R(1) - t * t * (R(3) - R(2) * t), R(-6) * t * (R(1) - t) * w,
                         R(-6) * (R(1) - R(2) * t) * w * w, r, isg);
    }
    // S_r = S((r - sigma) / ((2^(1/6) - 1) sigma)), and 1 - S_r
    R ts = (r - P.Srlo[p]) * P.Srinv[p];
    Rs<R> S{R(1), R(0), R(0), R(0)};
    if (ge_(ts, R(1))) {
        S = Rs<R>{R(0), R(0), R(0), R(0)};
    } else if (gt_(ts, R(0))) {
        R sn, cs;
        sincospi_(ts, &sn, &cs);
        R w = P.Srinv[p];
        const R pi = R(3.14159265358979323846);
        S = rs_scaled<R>(R(0.5) * (R(1) + cs), R(-0.5) * pi * sn * w, R(-0.5) * pi * pi * cs * w * w, r, isg);
    }
    Rs<R> Sm{R(1) - S.v, -S.r, -S.s, -S.rs};
    g1 = rs_mul3<R>(A, B, Sm);
    g2 = rs_mul3<R>(A, B, S);
}

// v . dF/d(eps_p) and v . dF/d(sigma_p) of one LJ pair i -> (j, image) with
// displacement d, C and its path, S_b and dotSb = v . (-grad S_b) (zero where
// dS_b = 0), added to J[p] and J[3 + p].  The forces of E = C (g1 + g2 S_b)
// are linear in eps (so dF/deps = F / eps), and dE/dsigma = C (h1 + h2 S_b)
// has the same form, so dF/dsigma = -grad(dE/dsigma) follows from the same
// three parts: the radial force, the path forces of C (dotW = v . F of the
// energy w_max, with C = 1 - w_max) and the b* forces.
template <class R>
HD void lj_pair_jvp(const DevParams<R>& P, const Graph<R>& G, int i, int j, R dx, R dy, R dz, R r2, R C, int code,
                    R Sb, R dotSb, const double* v, int n, double* J) {
    int p = pidx(G.type[i], G.type[j]);
    R inv_r = rsqrt_(r2);
    R r = r2 * inv_r;
    Rs<R> g1, g2;
    lj_radial_sigma<R>(P, p, r, g1, g2);
    // (v_j - v_i) . r_hat
    double vr = ((v[j] - v[i]) * (double)dx + (v[n + j] - v[n + i]) * (double)dy +
                 (v[2 * n + j] - v[2 * n + i]) * (double)dz) * (double)inv_r;
    double dotW = 0;
    if (code >= 0) {
        JSink js{v, n, 0.0, false, {0, 0, 0, 0, 0, 0}};
        double fx = 0, fy = 0, fz = 0;
        path_forces<R, JSink>(G, i, code, R(1), js, fx, fy, fz);
        js.add(i, fx, fy, fz);
        dotW = js.jdot;
    }
    // v . F for E = C (a1 + a2 S_b): the radial force -(dE/dr) r_hat on j (and
    // its opposite on i), the path forces of C = 1 - w_max, and the b* forces
    auto vdotF = [&](R a1, R a1r, R a2, R a2r) {
        double c = (double)C;
        return -c * (double)(a1r + a2r * Sb) * vr - (double)(a1 + a2 * Sb) * dotW + c * (double)a2 * (double)dotSb;
    };
    double eps = (double)(P.kind == 0 ? P.eps4[p] * R(0.25) : P.meps[p]);
    J[p] += vdotF(g1.v, g1.r, g2.v, g2.r) / eps;
    J[3 + p] += vdotF(g1.s, g1.rs, g2.s, g2.rs);
}

// dotSb = v . (-grad S_b) of a b* pair in its transition: the reverse bond
// order with dE/db* = dS_b/db*, dotted with v instead of applied.
template <class R>
HD R bstar_jvp(const DevParams<R>& P, const Graph<R>& G, int i, int j, R dx, R dy, R dz, R r2, const double* v,
               int n, R& Sb) {
    int p = pidx(G.type[i], G.type[j]);
    R inv_r = rsqrt_(r2);
    R rs = P.rstar[p];
    R ux = dx * inv_r * rs, uy = dy * inv_r * rs, uz = dz * inv_r * rs;
    R gux = 0, guy = 0, guz = 0, gumag = 0;
    double fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    JSink js{v, n, 0.0, false, {0, 0, 0, 0, 0, 0}};
    BstarSwitch<R> bsw{P.bmin[p], P.binv[p], R(1), R(0), R(0)};
    bond_order_c<R, true, JSink>(P, G, i, j, ux, uy, uz, rs, rcp_(rs), R(0), js, gux, guy, guz, gumag,
                                 fix, fiy, fiz, fjx, fjy, fjz, &bsw);
    Sb = bsw.Sb;
    if (is_zero(bsw.dSb)) return R(0);
    R ud = (gux * dx + guy * dy + guz * dz) * inv_r;
    R sc = rs * inv_r;
    double gx = (double)(sc * (gux - ud * dx * inv_r));
    double gy = (double)(sc * (guy - ud * dy * inv_r));
    double gz = (double)(sc * (guz - ud * dz * inv_r));
    js.add(i, fix + gx, fiy + gy, fiz + gz);
    js.add(j, fjx - gx, fjy - gy, fjz - gz);
    return (R)js.jdot;
}

}  // namespace airebo

#ifdef __CUDACC__
#include "ef.cuh"          // the FP32 value with an error bound (R = ef: the b* screen of the FP64 path)
#endif

// FMA throughput probe: the ALU roofline denominator of the FP64 and mixed
// paths, measured on the device the library runs on; accuracy checks of the
// FP64 reciprocals and of the double-float operations.
#include <cstring>

#include "internal.h"

namespace airebo {

template <class T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[0] = s;   // keeps the chains alive
}

double alu_peak(int fp64) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* out = nullptr;
    if (cudaMalloc(&out, 64) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int blocks = sms * 8, threads = 256;
    int iters = fp64 ? 64 : 2048;
    double best = 0;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0);
        if (fp64) k_fma<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
        else k_fma<float><<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        double flops = 2.0 * 64.0 * iters * (double)blocks * threads;
        if (rep > 0 && ms > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return cudaGetLastError() == cudaSuccess ? best : -1.0;
}

// Accuracy of the FP64 reciprocal and reciprocal square root of the kernels
// (rcp_, rsqrt_) against CUDA's correctly rounded division and square root,
// over x = 2^t, t uniform in [-30, 30) (a counter-based hash picks t).
// out[0], out[1]: largest difference in units in the last place for 1/x and
// 1/sqrt(x) (the latter's reference, 1 / sqrt(x) with two correct roundings,
// is itself within 1 ulp); out[2], out[3]: the same for the hardware
// approximations alone.
__global__ void k_math_check(unsigned long long* out, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    unsigned long long h = (unsigned long long)k * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
    double t = -30.0 + 60.0 * (double)(h >> 11) * (1.0 / 9007199254740992.0);
    double x = exp2(t);
    double r1 = rcp_(x), q1 = __ddiv_rn(1.0, x);
    double r2 = rsqrt_(x), q2 = __ddiv_rn(1.0, __dsqrt_rn(x));
    long long d1 = __double_as_longlong(r1) - __double_as_longlong(q1);
    long long d2 = __double_as_longlong(r2) - __double_as_longlong(q2);
    atomicMax(out + 0, (unsigned long long)(d1 < 0 ? -d1 : d1));
    atomicMax(out + 1, (unsigned long long)(d2 < 0 ? -d2 : d2));
    // the hardware approximations alone, before the Newton step
    double a1, a2;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(a1) : "d"(x));
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(a2) : "d"(x));
    long long d3 = __double_as_longlong(a1) - __double_as_longlong(q1);
    long long d4 = __double_as_longlong(a2) - __double_as_longlong(q2);
    atomicMax(out + 2, (unsigned long long)(d3 < 0 ? -d3 : d3));
    atomicMax(out + 3, (unsigned long long)(d4 < 0 ? -d4 : d4));
}

// Accuracy of the double-float operations (dd.cuh) against FP64 on the same
// inputs, whose hi + lo sums are exact in FP64.  Operands a, b = +-m 2^t with
// m uniform in [1, 2), t uniform in [-20, 20) (counter-based hash), split into
// dd; t in [0, 2) for sin/cos of pi t.  out (as the bits of non-negative
// doubles, so that atomicMax orders them): the largest error of a + b
// relative to |a| + |b|; of a * b, a / b, 1 / a, 1 / sqrt(|a|) relative to
// the exact-input FP64 result; of sin(pi t) and cos(pi t) absolute; of the
// conversion from double relative.
__device__ __forceinline__ double dd_rand(unsigned long long k, int salt, double lo, double hi) {
    unsigned long long h = (k * 2 + salt) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
    return lo + (hi - lo) * (double)(h >> 11) * (1.0 / 9007199254740992.0);
}
__global__ void k_dd_check(unsigned long long* out, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    auto pick = [&](int salt) {
        double m = dd_rand(k, salt, 1.0, 2.0) * (dd_rand(k, salt + 7, 0.0, 1.0) < 0.5 ? -1.0 : 1.0);
        return m * exp2(floor(dd_rand(k, salt + 13, -20.0, 20.0)));
    };
    double x = pick(1), y = pick(2);
    dd a(x), b(y);
    double ea = (double)a, eb = (double)b;             // the exact values of the operands
    double t = dd_rand(k, 5, 0.0, 2.0);
    dd u(t);
    double eu = (double)u;
    double err[8];
    err[0] = fabs((double)(a + b) - (ea + eb)) / (fabs(ea) + fabs(eb));
    err[1] = fabs((double)(a * b) / (ea * eb) - 1.0);
    err[2] = fabs((double)(a / b) / (ea / eb) - 1.0);
    err[3] = fabs((double)rcp_(a) * ea - 1.0);
    dd aa = a.hi < 0.0f ? -a : a;
    err[4] = fabs((double)rsqrt_(aa) * sqrt(fabs(ea)) - 1.0);
    dd s, c;
    sincospi_(u, &s, &c);
    double rs, rc;
    sincospi(eu, &rs, &rc);
    err[5] = fabs((double)s - rs);
    err[6] = fabs((double)c - rc);
    err[7] = fabs(ea / x - 1.0);
    for (int q = 0; q < 8; q++) atomicMax(out + q, (unsigned long long)__double_as_longlong(err[q]));
}

int dd_check(double* out8) {
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 64) != cudaSuccess) return 1;
    cudaMemset(d, 0, 64);
    int n = 1 << 22;
    k_dd_check<<<(n + 255) / 256, 256>>>(d, n);
    unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(h, d, 64, cudaMemcpyDeviceToHost);
    cudaFree(d);
    for (int k = 0; k < 8; k++) memcpy(out8 + k, h + k, 8);
    return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? 0 : 1;
}

int math_check(long long* out4) {
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 32) != cudaSuccess) return 1;
    cudaMemset(d, 0, 32);
    int n = 1 << 22;
    k_math_check<<<(n + 255) / 256, 256>>>(d, n);
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(h, d, 32, cudaMemcpyDeviceToHost);
    cudaFree(d);
    for (int k = 0; k < 4; k++) out4[k] = (long long)h[k];
    return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? 0 : 1;
}

}  // namespace airebo

// Rebuild check that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they run -- code inside a
// framework that owns all device memory through its own pool, or code that
// must not allocate after its set-up phase -- yet still need to know when the
// neighbour lists are stale.  airebo_needs_rebuild_noalloc serves them: it is
// the displacement check of airebo_needs_rebuild (max |x - x_ref| against
// skin/2) computed by one kernel whose scratch is the file-scope device array
// below instead of a buffer owned by a handle, so the caller passes only its
// inputs and outputs and needs no handle at all.
//
// The array is part of the library image: every GPU that loads the library
// holds it (about 64 KB) until the process exits.  All calls share it and it
// keeps the last call's contents; the entry point clears the one word that
// must start at zero before each launch.  Calls whose kernels overlap on the
// GPU (different streams, or different host threads on one device) race on
// the array and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cmath>
#include <mutex>

#include "../../include/airebo.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 8192;                       // n <= 2,097,152 atoms
constexpr int NA_RESULT = NA_MAX_BLOCKS;                  // slot of the final maximum
constexpr int NA_COUNTER = NA_MAX_BLOCKS + 1;             // slot holding the blocks-done counter
constexpr int NA_WORDS = NA_MAX_BLOCKS + 32;

// per-block maxima of |dx|^2, the final maximum, and the blocks-done counter
static __device__ __align__(256) double g_noalloc_scratch[NA_WORDS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
// per device: the array's device address and the id of the context it was
// looked up in (a reset device gets a new context, and the array a new address)
double* g_scratch_ptr[NA_MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[NA_MAX_DEVICES] = {};

// One kernel: each block writes the maximum squared displacement of its atoms
// to scratch[block]; the last block to finish reduces those into
// scratch[NA_RESULT] and resets the counter.
__global__ void __launch_bounds__(NA_THREADS) k_max_disp_noalloc(const double* pos, const double* ref, int n,
                                                                 double* scratch) {
    __shared__ double red[NA_THREADS / 32];
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    if (i < n) {
        double ex = pos[i] - ref[i], ey = pos[n + i] - ref[n + i], ez = pos[2 * n + i] - ref[2 * n + i];
        d2 = ex * ex + ey * ey + ez * ez;
        if (!(d2 == d2)) d2 = 1e300;
    }
    for (int o = 16; o > 0; o >>= 1) d2 = fmax(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++) m = fmax(m, red[w]);
        scratch[blockIdx.x] = m;
        __threadfence();
        unsigned* counter = reinterpret_cast<unsigned*>(scratch + NA_COUNTER);
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        // the other blocks' maxima, read from L2 (where their writes went
        // before their fences), not from this SM's L1
        double m = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = fmax(m, __ldcg(scratch + b));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int w = 0; w < NA_THREADS / 32; w++) r = fmax(r, red[w]);
            scratch[NA_RESULT] = r;
            *reinterpret_cast<unsigned*>(scratch + NA_COUNTER) = 0u;
        }
    }
}

// Id of the current context (0 if the driver cannot tell), from the driver
// entry points the runtime hands out; the library does not link the driver.
unsigned long long current_context_id() {
    typedef CUresult (*get_current_t)(CUcontext*);
    typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<get_current_t>(f1);
            get_id = reinterpret_cast<get_id_t>(f2);
        }
        looked = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of the scratch array on the current device (host code may
// not pass the array's name to a kernel: on the host it is only a stand-in
// for the symbol).  Set-up: the first call made with a device current looks
// the address up and keeps it with the id of the device's context; it is
// looked up again only when that context has changed (after a
// cudaDeviceReset).  That first call should come before any stream capture.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    e = cudaSetDevice(dev);                    // makes the device's primary context current
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" airebo_status airebo_needs_rebuild_noalloc(const double* d_pos, const double* d_ref, int64_t n,
                                                      double skin, void* stream, int* h_flag,
                                                      double* h_max_disp) {
    if (!h_flag || n < 0 || !(skin >= 0.0)) return AIREBO_ERR_ARG;
    if (n > (int64_t)NA_MAX_BLOCKS * NA_THREADS) return AIREBO_ERR_ARG;   // beyond the scratch array
    if (n > 0 && (!d_pos || !d_ref)) return AIREBO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double d2 = 0.0;
    if (n > 0) {
        double* scratch = nullptr;
        if (scratch_address(&scratch) != cudaSuccess) return AIREBO_ERR_CUDA;
        if (cudaMemsetAsync(scratch + NA_COUNTER, 0, sizeof(double), s) != cudaSuccess) return AIREBO_ERR_CUDA;
        int blocks = (int)((n + NA_THREADS - 1) / NA_THREADS);
        k_max_disp_noalloc<<<blocks, NA_THREADS, 0, s>>>(d_pos, d_ref, (int)n, scratch);
        if (cudaGetLastError() != cudaSuccess) return AIREBO_ERR_CUDA;
        if (cudaMemcpyAsync(&d2, scratch + NA_RESULT, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return AIREBO_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return AIREBO_ERR_CUDA;
    }
    double half = 0.5 * skin;
    *h_flag = d2 > half * half ? 1 : 0;
    if (h_max_disp) *h_max_disp = std::sqrt(d2);
    return AIREBO_OK;
}

// noalloc.cu -- an energy reduction that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand
// out every byte of device memory from their own arena or a framework's
// caching allocator, and that budget memory up front.  For them
// fmm_energy_noalloc computes E = 1/2 sum_i q_i phi_i of caller arrays with the
// same two-kernel FP64 reduction as fmm_energy, but keeps its per-block partial
// sums in a fixed array in the library's own device memory (kNoAllocBlocks
// doubles, 64 KiB, present on every device that loads the library until the
// process exits) instead of in handle workspace.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress and caches it together with
// the current CUDA context; a later call in another context (after a device
// reset, or a context torn down and made again) looks it up again.  The first
// call on a device should be made before any stream capture.  All calls share
// the array and it keeps the last call's contents; every partial a call reads
// is written by that call, so nothing needs clearing.  Calls that overlap on
// the GPU (two streams, or two host threads) race on the array.
//
// q, phi and E must be device (or managed) memory that the current device can
// reach: each pointer's kind is looked up with cudaPointerGetAttributes
// (which allocates nothing) before anything is launched, and a host pointer is
// an argument error rather than a kernel writing to a host address.
#include <cuda_runtime.h>

#include <cuda.h>

#include <mutex>

#include "device_util.cuh"
#include "fmm_internal.cuh"

namespace fmm {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocItems = 8;                                  // per thread
constexpr int64_t kNoAllocChunk = kNoAllocThreads * kNoAllocItems;  // elements per block
constexpr int kNoAllocBlocks = 8192;                             // one FP64 partial per block
constexpr int64_t kNoAllocMaxN = kNoAllocChunk * kNoAllocBlocks;   // 16,777,216

static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks];

constexpr int kMaxDevices = 64;
static double *g_partials_addr[kMaxDevices] = {};
static CUcontext g_partials_ctx[kMaxDevices] = {};
static std::mutex g_partials_mutex;

__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_energy_partial(const float *q, const float *phi,
                                                                            int64_t n, double *partials)
{
    const int64_t base = (int64_t)blockIdx.x * kNoAllocChunk;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kNoAllocItems; ++k) {
        const int64_t i = base + (int64_t)k * kNoAllocThreads + threadIdx.x;
        if (i < n) s += (double)q[i] * (double)phi[i];
    }
    s = warp_sum(s);
    __shared__ double ws[kNoAllocThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_energy_final(const double *partials, int nblocks,
                                                                          double *E)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[b];
    s = warp_sum(s);
    __shared__ double ws[kNoAllocThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) t += ws[w];
        *E = 0.5 * t;
    }
}

// The current CUDA context (driver entry point, looked up once; no linking
// against libcuda).  Null if the entry point is unavailable.
static CUcontext current_context()
{
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<Fn>(f);
    }();
    CUcontext c = nullptr;
    if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

// Device address of the partials array on the current device, looked up once
// per device and context.
static int partials_address(double **out)
{
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fmm_energy_noalloc: device ordinal out of range");
        return FMM_ERR_ARG;
    }
    // the runtime has made the device's context current by now (the pointer
    // checks ran first); without a context handle the address is looked up on
    // every call
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lock(g_partials_mutex);
    if (!g_partials_addr[dev] || !ctx || g_partials_ctx[dev] != ctx) {
        void *p = nullptr;
        FMM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_partials_addr[dev] = static_cast<double *>(p);
        g_partials_ctx[dev] = ctx;
    }
    *out = g_partials_addr[dev];
    return FMM_OK;
}

// 0 if p is device memory of device dev or managed memory; an error code (and
// message naming the argument) otherwise.
static int check_device_pointer(const void *p, int dev, const char *name)
{
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // clear the sticky-free error of the lookup
        set_error(std::string("fmm_energy_noalloc: ") + name + " is not a CUDA pointer");
        return FMM_ERR_ARG;
    }
    if (a.type == cudaMemoryTypeManaged) return FMM_OK;
    if (a.type == cudaMemoryTypeDevice && a.device == dev) return FMM_OK;
    set_error(std::string("fmm_energy_noalloc: ") + name +
              (a.type == cudaMemoryTypeDevice ? " is device memory of another GPU than the current one"
                                              : " is host memory; it must be device memory of the current GPU"));
    return FMM_ERR_ARG;
}

}  // namespace fmm

using namespace fmm;

extern "C" int fmm_energy_noalloc(const float *q, const float *phi, int64_t n, double *E, void *stream)
{
    if (!q || !phi || !E) {
        set_error("fmm_energy_noalloc: null argument");
        return FMM_ERR_ARG;
    }
    if (n < 1 || n > kNoAllocMaxN) {
        set_error("fmm_energy_noalloc: n must be in [1, 16777216] (one FP64 partial per 2048 particles "
                  "in a fixed 64 KiB device array)");
        return FMM_ERR_ARG;
    }
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    FMM_TRY(check_device_pointer(q, dev, "q"));
    FMM_TRY(check_device_pointer(phi, dev, "phi"));
    FMM_TRY(check_device_pointer(E, dev, "E"));
    double *partials = nullptr;
    FMM_TRY(partials_address(&partials));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
    k_noalloc_energy_partial<<<nb, kNoAllocThreads, 0, s>>>(q, phi, n, partials);
    k_noalloc_energy_final<<<1, kNoAllocThreads, 0, s>>>(partials, nb, E);
    FMM_CHECK_LAUNCH("fmm_energy_noalloc");
    return FMM_OK;
}

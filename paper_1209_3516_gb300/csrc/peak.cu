// peak.cu -- the FP32 roofline denominators of this GPU, measured.
//
// The P2P and M2L kernels are bound by FP32 arithmetic (FMA pipe) and, for the
// P2P, one SFU reciprocal square root per particle pair.  Their roofline
// fractions need the chip's FP32 FMA rate and SFU rsqrt rate, which no
// vendor-measured figure here provides, so this file measures them with three
// launches of register-only chains, each over every SM:
//   - scalar FFMA: 8 independent chains a = a*m + c per thread;
//   - packed FFMA2: 8 independent float2 chains (two FMAs per instruction);
//   - MUFU rsqrt.approx.ftz: 8 independent chains x = rsqrt(x) + c.
// Each launch runs long enough (tens of ms) for the launch overhead to vanish;
// the best of several launches, timed with CUDA events on the caller's stream,
// is reported.  Flops count an FMA as two; the rsqrt rate counts operations.
// The paper has no counterpart (it quotes its CPU's peak from the data sheet).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"

namespace fmm {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;
constexpr int kPeakMaxBlocksPerSM = 2048 / kPeakThreads;

__device__ __forceinline__ float rsqrt_chain_step(float x, float c)
{
    float r;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r + c;
}

// kind 0: scalar FFMA, 1: packed FFMA2, 2: rsqrt.approx
template <int kKind>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float m, float c, float never, float *sink)
{
    float a[kPeakChains];
    float2 a2[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) {
        a[k] = 1.0f + 0.001f * (float)(threadIdx.x + k);
        a2[k] = make_float2(a[k], a[k] + 0.5f);
    }
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) {
                if (kKind == 0) a[k] = fmaf(a[k], m, c);
                else if (kKind == 1) a2[k] = __ffma2_rn(a2[k], m2, c2);
                else a[k] = rsqrt_chain_step(a[k], c);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += (kKind == 1) ? a2[k].x + a2[k].y : a[k];
    if (s == never) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true: keeps the chains live
}

// Times `reps` launches of one full wave (the occupancy limit of every SM) and
// keeps the fastest; *threads is the grid's thread count.
template <int kKind>
static int time_peak(int sms, int iters, cudaStream_t s, float *sink, int reps, double *best_ms, double *threads)
{
    int per_sm = 0;
    FMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak<kKind>, kPeakThreads, 0));
    const int blocks = sms * std::max(1, std::min(per_sm, kPeakMaxBlocksPerSM));
    *threads = (double)blocks * kPeakThreads;
    cudaEvent_t e0, e1;
    FMM_CUDA(cudaEventCreate(&e0));
    FMM_CUDA(cudaEventCreate(&e1));
    k_peak<kKind><<<blocks, kPeakThreads, 0, s>>>(iters / 8, 0.999f, 0.001f, -12345.0f, sink);   // warm-up
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        k_peak<kKind><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999f, 0.001f, -12345.0f, sink);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "k_peak", __FILE__, __LINE__);
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    FMM_CHECK_LAUNCH("k_peak");
    *best_ms = best;
    return FMM_OK;
}

}  // namespace fmm

using namespace fmm;

extern "C" int fmm_measure_peaks(fmm_peaks *out, void *stream)
{
    if (!out) {
        set_error("fmm_measure_peaks: null argument");
        return FMM_ERR_ARG;
    }
    int dev = 0, sms = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    FMM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // sink: never written (the guard is never true), but it must be a valid
    // address for every thread of the largest grid
    float *sink = nullptr;
    FMM_CUDA(cudaMallocAsync(&sink, (size_t)sms * 2048 * sizeof(float), s));
    const int iters[3] = {16384, 8192, 2048};   // ~10-30 ms per launch on a GB300
    double ms[3] = {0, 0, 0}, thr[3] = {0, 0, 0};
    int rc = time_peak<0>(sms, iters[0], s, sink, 5, &ms[0], &thr[0]);
    if (rc == FMM_OK) rc = time_peak<1>(sms, iters[1], s, sink, 5, &ms[1], &thr[1]);
    if (rc == FMM_OK) rc = time_peak<2>(sms, iters[2], s, sink, 5, &ms[2], &thr[2]);
    cudaFreeAsync(sink, s);
    if (rc != FMM_OK) return rc;
    const double per_thread[3] = {(double)iters[0] * kPeakUnroll * kPeakChains,
                                  (double)iters[1] * kPeakUnroll * kPeakChains * 2.0,
                                  (double)iters[2] * kPeakUnroll * kPeakChains};
    out->sms = sms;
    out->ffma_tflops = 2.0 * thr[0] * per_thread[0] / (ms[0] * 1e-3) / 1e12;
    out->ffma2_tflops = 2.0 * thr[1] * per_thread[1] / (ms[1] * 1e-3) / 1e12;
    out->rsqrt_per_s = thr[2] * per_thread[2] / (ms[2] * 1e-3);
    out->ms_ffma = ms[0];
    out->ms_ffma2 = ms[1];
    out->ms_rsqrt = ms[2];
    return FMM_OK;
}

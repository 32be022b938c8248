// Issue-rate microbenchmarks of the two pipes that bound the per-pixel and per-point kernels
// (include/sof.h, sof_measure_issue_peaks): the FP32 FMA pipe and the MUFU (special-function) pipe.
// They are the denominators of the roofline fractions of the composite, the replay and the query
// integration, measured on the device that runs them instead of taken from a data sheet.
//
// Each thread runs kChains independent dependency chains (enough independent work per warp that
// the pipe, not the latency, limits), 1024 threads per SM. An FFMA counts as one operation, as in
// the kernels' algorithmic operation counts.
#include <stdio.h>

#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;

// Written only when a chain ends on an impossible value: keeps every chain live.
__device__ float g_peak_sink;

__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)threadIdx.x * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.2345f) g_peak_sink = s;
}

__global__ void __launch_bounds__(kThreads) k_ex2_chains(int iters) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = -0.5f - (float)i * 1e-2f - (float)threadIdx.x * 1e-5f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 4
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                // 2^a of a negative a lies in (0, 1); its negation keeps the chain in (-1, 0)
                float y;
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
                a[i] = -y;
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == 1.2345f) g_peak_sink = s;
}

// Best of three timed launches (after one warm-up) in ms.
template <typename F>
cudaError_t time_best(F launch, cudaStream_t s, float *best_ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();
    *best_ms = 0.f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        float ms = 0.f;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        if ((e = launch()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (r == 0 || ms < *best_ms) *best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace sof

using namespace sof;

extern "C" int sof_measure_issue_peaks(double *fp32_tops, double *mufu_tops, void *stream) {
    if (!fp32_tops || !mufu_tops) return SOF_ERR_INVALID_ARG;
    *fp32_tops = *mufu_tops = 0.0;
    int dev = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return SOF_ERR_NO_DEVICE;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = device_sm_count() * kCtasPerSm;
    const int fma_iters = 1 << 14, ex2_iters = 1 << 13;  // about 8 ms each on GB300
    float ms = 0.f;
    cudaError_t e = time_best(
        [&]() {
            note_launches(1);
            k_fma_chains<<<grid, kThreads, 0, s>>>(fma_iters, 0.999f, 1e-3f);
            return cudaGetLastError();
        },
        s, &ms);
    if (e != cudaSuccess || ms <= 0.f) return SOF_ERR_CUDA;
    *fp32_tops = (double)grid * kThreads * kChains * 16.0 * fma_iters / (ms * 1e-3) / 1e12;
    e = time_best(
        [&]() {
            note_launches(1);
            k_ex2_chains<<<grid, kThreads, 0, s>>>(ex2_iters);
            return cudaGetLastError();
        },
        s, &ms);
    if (e != cudaSuccess || ms <= 0.f) return SOF_ERR_CUDA;
    *mufu_tops = (double)grid * kThreads * kChains * 4.0 * ex2_iters / (ms * 1e-3) / 1e12;
    return SOF_OK;
}

// peak.cu -- the measured FP32 throughput of this GPU: the denominator of the
// step kernels' ALU roofline. Nothing on the tracking path calls it.
//
// Every thread runs kChains independent FMA chains (x <- x a + b), so each
// scheduler always has an independent FMA to issue; the grid holds 2048
// threads on every SM (the most it can keep resident), sized from the SM count
// that the device reports.
#include <cuda_runtime.h>

#include "../../include/inhand.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;   // 8 x 256 = 2048 resident threads per SM

__global__ void __launch_bounds__(kThreads) ffma_chains_kernel(float *sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) sink[blockIdx.x] = s;   // never true for a in (0, 1): keeps the chains live
}

}  // namespace

extern "C" ih_status ih_fp32_peak(int32_t iters, int32_t reps, void *stream, double *tflops,
                                  double *ms_per_launch, int32_t *sm_count) {
    if (iters < 1 || reps < 1 || !tflops) return IH_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IH_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return IH_ERR_CUDA;
    const int grid = sms * kBlocksPerSm;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, grid * sizeof(float)) != cudaSuccess) return IH_ERR_OOM;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {   // warm-up
        ffma_chains_kernel<<<grid, kThreads, 0, s>>>(sink, iters, 0.999f, 1e-4f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        ffma_chains_kernel<<<grid, kThreads, 0, s>>>(sink, iters, 0.999f, 1e-4f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || !(ms > 0.0f)) return IH_ERR_CUDA;
    const double per_launch = (double)ms / reps;
    const double flop = 2.0 * kChains * kUnroll * (double)iters * (double)grid * kThreads;
    *tflops = flop / (per_launch * 1e-3) / 1e12;
    if (ms_per_launch) *ms_per_launch = per_launch;
    if (sm_count) *sm_count = sms;
    return IH_OK;
}

// cg_diag.cu -- measured FP32 throughput of the device, the denominator of
// the ALU roofline of the LM kernels (a diagnostic of this library; the paper
// has no counterpart).
//
// Every thread runs 16 independent chains a <- a * m + c (packed: 8 chains of
// FP32x2 pairs, each instruction two fused multiply-adds), enough independent
// work per warp that the FMA pipes, not latency, set the rate.  The launches
// are timed with CUDA events on the caller's stream.
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_internal.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

// written only if the chains reach an impossible value: keeps them live
__device__ float g_fma_sink;

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(int iters, float seed)
{
    const float m = 0.99999f, c = 1.0e-7f;
    float total = 0.f;
    if constexpr (PACKED) {
        float2 a[kChains / 2];
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i)
            a[i] = make_float2(seed + 1e-3f * i + 1e-7f * threadIdx.x, seed - 1e-3f * i);
        const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains / 2; ++i) a[i] = __ffma2_rn(a[i], m2, c2);
        }
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i) total += a[i].x + a[i].y;
    } else {
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = seed + 1e-3f * i + 1e-7f * threadIdx.x;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) total += a[i];
    }
    if (total == -1.0f) g_fma_sink = total;
}

}  // namespace

extern "C" cg_status cg_fp32_peak(int packed, int reps, double* tflops_host, void* cuda_stream)
{
    cg::set_last_error("");
    if (!tflops_host || reps < 1 || (packed != 0 && packed != 1)) {
        cg::set_last_error("packed must be 0 or 1, reps >= 1, tflops_host non-NULL");
        return CG_ERR_ARG;
    }
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int iters = 4096;
    const dim3 grid(sms * kBlocksPerSM), block(kThreads);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto launch = [&] {
        if (packed) fma_peak_kernel<true><<<grid, block, 0, s>>>(iters, 1.0f);
        else fma_peak_kernel<false><<<grid, block, 0, s>>>(iters, 1.0f);
        return cudaGetLastError();
    };
    // one warm-up launch, then the timed ones
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cg::set_last_error(cudaGetErrorString(e));
        return CG_ERR_CUDA;
    }
    const double flop = 2.0 * kChains * static_cast<double>(iters) * grid.x * block.x * reps;
    *tflops_host = flop / (ms * 1e-3) / 1e12;
    return CG_OK;
}

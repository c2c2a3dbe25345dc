// bf_probe.cu -- bf_measure_fp32_peak: the FP32 fused multiply-add rate of the
// CUDA cores, measured on the current device. It is the roofline denominator
// of the plain FP32 product form (BF_FP32), whose 22.4 flop per byte at f = 36
// puts it above the CUDA-core ridge point: its bound is FMA issue, not HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "bf.h"
#include "bf_plan.h"

namespace {

constexpr int CHAINS = 8;    // independent FMA chains per thread (covers the FMA latency)
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 4;

// MODE 0 / 1: every thread runs CHAINS independent chains a <- a * b + c for
// `iters` rounds of 4: 2 * 4 * CHAINS * iters flop per thread (twice that
// with packed FP32x2 FMAs, MODE 1). b and c are the same for every thread
// (kernel arguments), so only a is read from the register file: the FMA
// pipe's own limit. b is just below 1 and c small, so the values stay finite
// and normal. The final store is conditional on a value no chain reaches, so
// the compiler cannot drop the loop, and it never writes in practice.
template <int MODE>
__global__ void __launch_bounds__(THREADS) bf_ffma_peak_kernel(float *sink, int iters, float b, float c) {
    using V = typename std::conditional<MODE == 1, float2, float>::type;
    V a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) {
        const float x = (float)(threadIdx.x + k) * 1e-3f;
        if constexpr (MODE == 1) a[k] = make_float2(x, x + 0.5f);
        else a[k] = x;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) {
                if constexpr (MODE == 1) a[k] = __ffma2_rn(a[k], make_float2(b, b), make_float2(c, c));
                else a[k] = __fmaf_rn(a[k], b, c);
            }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) {
        if constexpr (MODE == 1) s += a[k].x + a[k].y;
        else s += a[k];
    }
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// MODE 2: packed FP32x2 FMAs in the operand pattern of an outer-product
// (register-blocked matrix product) loop: 16 accumulator pairs acc[e][q] +=
// x[e] * y[q] over 4 x 4 operand pairs held in registers, 4 * 16 * iters
// flop per thread. Each instruction reads two register pairs that the
// previous one did not (one operand is shared with it), as every such loop
// must; the rate is the ceiling of an FP32 product kernel, below the MODE 1
// rate. Operands are built from the thread index (no memory traffic) and the
// increments are small, so the accumulators stay finite.
__global__ void __launch_bounds__(THREADS) bf_ffma_outer_kernel(float *sink, int iters, float b, float c) {
    float2 acc[4][4], x[4], y[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float t = (float)(threadIdx.x + e) * 1e-3f;
        x[e] = make_float2(t * b, t * c + 1e-3f);
        y[e] = make_float2(0.5f + t, 0.25f + t);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[e][q] = make_float2(t, -t);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[e][q] = __ffma2_rn(x[e], y[q], acc[e][q]);
    }
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) s += acc[e][q].x + acc[e][q].y;
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" bf_status bf_measure_fp32_peak(int32_t iters, int32_t reps, int32_t mode, double *tflops_host,
                                          double *ms_host, void *stream) {
    if (!tflops_host || iters < 1 || iters > (1 << 24) || reps < 1 || reps > 1000 || mode < 0 || mode > 2)
        return bf_fail(nullptr, BF_EINVAL, "bf_measure_fp32_peak: iters in [1, 2^24], reps in [1, 1000], "
                                           "mode 0, 1 or 2, tflops_host not NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "device query: %s", cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = sms * CTAS_PER_SM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return bf_fail(nullptr, BF_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
    }
    float best_ms = 0.f;
    // one warm-up launch, then the best of `reps` timed launches
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        if (mode == 2)
            bf_ffma_outer_kernel<<<grid, THREADS, 0, s>>>(nullptr, iters, 0.9999999f, 1e-7f);
        else if (mode == 1)
            bf_ffma_peak_kernel<1><<<grid, THREADS, 0, s>>>(nullptr, iters, 0.9999999f, 1e-7f);
        else
            bf_ffma_peak_kernel<0><<<grid, THREADS, 0, s>>>(nullptr, iters, 0.9999999f, 1e-7f);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0) best_ms = (best_ms == 0.f) ? ms : std::min(best_ms, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "FMA probe: %s", cudaGetErrorString(e));
    const double per_iter = mode == 2 ? 4.0 * 16 : (mode == 1 ? 4.0 : 2.0) * CHAINS * 4;
    const double flop = per_iter * (double)iters * (double)grid * THREADS;
    *tflops_host = flop / (best_ms * 1e-3) / 1e12;
    if (ms_host) *ms_host = best_ms;
    return BF_OK;
}

// Throughput micro-benchmark of the two SIMT pipes the MPPI step is bound
// by: FP32 fused multiply-add (the FMA pipe) and the multi-function unit
// (MUFU: ex2, lg2, rsqrt, sin, cos).  It gives the roofline its measured
// denominators on the GPU the step runs on.
//
// Each kernel keeps kChains independent dependency chains per thread (so
// that latency is hidden by the chains and the resident warps, and the
// pipe, not the chain, is the limit), runs a fixed number of iterations
// and writes one value per thread only when a test the data never passes
// succeeds, so that nothing is eliminated.  The grid fills every SM with
// 1024 threads.  Each rate is the best of several launches timed with CUDA
// events on the caller's stream.
#include <cuda_runtime.h>

#include "mppi_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) ffma_kernel(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)threadIdx.x + (float)c;
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
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One MUFU operation per chain step; the chains stay bounded (ex2 of a
// non-positive value, lg2 of a value >= 1, rsqrt of a positive value,
// sine and cosine of a value in [-1, 1]).
enum MufuOp { kEx2 = 0, kLg2 = 1, kRsqrt = 2, kSin = 3, kCos = 4 };

template <int OP>
__device__ __forceinline__ float mufu_step(float x) {
    float y;
    if (OP == kEx2) {
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return -y;
    } else if (OP == kLg2) {
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y + 1.0f;
    } else if (OP == kRsqrt) {
        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else if (OP == kSin) {
        asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else {
        asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
}

template <int OP>
__global__ void __launch_bounds__(kThreads) mufu_kernel(float* out, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v = 1e-4f * (float)threadIdx.x + 0.05f * (float)c;
        x[c] = OP == kEx2 ? -v : OP == kLg2 ? 1.0f + v : OP == kRsqrt ? 0.5f + v : v;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = mufu_step<OP>(x[c]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.0e30f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best (shortest) time of `reps` launches of `launch` [ms].
template <typename F>
int best_ms(F launch, cudaStream_t st, int reps, float* best) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MPPI_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MPPI_ECUDA;
    }
    int rc = MPPI_OK;
    *best = 1e30f;
    launch();  // warm-up
    for (int r = 0; r < reps && rc == MPPI_OK; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = MPPI_ECUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < *best) *best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int mppi_measure_peaks(mppi_peaks* out, void* stream) {
    if (!out) return MPPI_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = mppi::sm_count();
    const int grid = sms * kBlocksPerSm;
    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)grid * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return MPPI_ENOMEM;
    }
    // About 4 ms per launch at 2 GHz: iters * kUnroll * kChains FMAs per
    // thread, 1024 threads per SM, 128 FP32 lanes per SM.
    const int iters_fma = 4096, iters_mufu = 512;
    const double threads = (double)grid * kThreads;
    mppi_peaks p = {};
    p.sm_count = sms;
    float ms = 0.0f;
    int rc = best_ms([&] { ffma_kernel<<<grid, kThreads, 0, st>>>(sink, iters_fma, 0.999999f, 1e-6f); }, st, 5,
                     &ms);
    if (!rc) {
        p.fp32_ms = ms;
        p.fp32_flops = threads * iters_fma * kUnroll * kChains * 2.0 / (ms * 1e-3);
    }
    auto mufu = [&](auto kernel, double* rate) {
        if (rc) return;
        float t = 0.0f;
        rc = best_ms([&] { kernel<<<grid, kThreads, 0, st>>>(sink, iters_mufu); }, st, 3, &t);
        if (!rc) *rate = threads * iters_mufu * kUnroll * kChains / (t * 1e-3);
    };
    mufu(mufu_kernel<kEx2>, &p.ex2_ops);
    mufu(mufu_kernel<kLg2>, &p.lg2_ops);
    mufu(mufu_kernel<kRsqrt>, &p.rsqrt_ops);
    mufu(mufu_kernel<kSin>, &p.sin_ops);
    mufu(mufu_kernel<kCos>, &p.cos_ops);
    cudaFree(sink);
    if (rc) return rc;
    *out = p;
    return MPPI_OK;
}

// Throughput probes of the arithmetic units the integration kernels use
// (a measurement program of bench.py's roofline, built apart from the
// library by bench_peaks.py):
// FP64 FMA (with all or some lanes of a warp active), FP32 FMA, FP64
// tensor-core MMA (mma.sync m8n8k4), the double exponential and the double
// reciprocal. They measure the denominators of the kernels' ALU roofline;
// none of them is part of the method. Each thread runs independent chains
// held in registers for a fixed number of iterations (no memory traffic in
// the loop, every launch ends) and stores one value so that nothing is
// optimised away.

#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;

// FP64 FMA on the first `active` lanes of every warp (the others idle)
__global__ void probe_dfma(int active, int64_t iters, double* out) {
    const int lane = threadIdx.x & 31;
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    if (lane < active) {
        const double m = 0.9999999, s = 1e-7;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, s);
        }
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void probe_ffma(int64_t iters, double* out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    const float m = 0.9999f, s = 1e-4f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, s);
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// D = A B + C with 8 x 4 FP64 A and 4 x 8 B, one element of each per lane,
// accumulators of two elements per lane; 4 independent accumulators
__global__ void probe_dmma(int64_t iters, double* out) {
    const double a = 1e-3 * (threadIdx.x & 31), b = 1e-3;
    double d[4][2];
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c][0] = d[c][1] = 0.0;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) t += d[c][0] + d[c][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// y <- exp(-y): a contraction towards 0.567, so values stay in range
__global__ void probe_exp(int64_t iters, double* out) {
    double y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) y[c] = 0.5 + 1e-3 * c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) y[c] = exp(-y[c]);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += y[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// y <- 1 / (1 + y): a contraction towards 0.618
__global__ void probe_rcp(int64_t iters, double* out) {
    double y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) y[c] = 0.5 + 1e-3 * c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) y[c] = 1.0 / (1.0 + y[c]);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += y[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

cudaError_t launch_one(int kind, int active, int64_t iters, int blocks, int threads, double* out,
                       cudaStream_t st) {
    switch (kind) {
        case 0: probe_dfma<<<blocks, threads, 0, st>>>(active, iters, out); break;
        case 1: probe_ffma<<<blocks, threads, 0, st>>>(iters, out); break;
        case 2: probe_dmma<<<blocks, threads, 0, st>>>(iters, out); break;
        case 3: probe_exp<<<blocks, threads, 0, st>>>(iters, out); break;
        default: probe_rcp<<<blocks, threads, 0, st>>>(iters, out); break;
    }
    return cudaGetLastError();
}

}  // namespace

// Runs probe `kind` (0 FP64 FMA on the first `active` lanes of every warp,
// 1 FP32 FMA, 2 FP64 MMA m8n8k4, 3 exp(double), 4 1/x (double)) on 8 blocks
// of 256 threads per SM for `iters` iterations, once to warm up and once
// timed with CUDA events; *rate receives FLOP/s for kinds 0-2 (an FMA
// counts 2) and evaluations/s for kinds 3-4. Returns a cudaError_t code.
extern "C" int peak_probe(int kind, int active, long long iters, double* rate) {
    if (kind < 0 || kind > 4 || active < 1 || active > 32 || iters < 1 || !rate) return (int)cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int threads = 256, blocks = 8 * sms;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_one(kind, active, iters, blocks, threads, out, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = launch_one(kind, active, iters, blocks, threads, out, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double warps = 8.0 * blocks, lanes = 32.0 * warps, it = (double)iters;
    const double ops[5] = {warps * active * it * kChains * 2,   // FP64 FMA
                           lanes * it * kChains * 2,              // FP32 FMA
                           warps * it * 4 * 2 * 8 * 8 * 4,        // 4 MMA of m8n8k4 per warp
                           lanes * it * kChains,                  // exp
                           lanes * it * kChains};                 // reciprocal
    *rate = ops[kind] / (ms * 1e-3);
    return 0;
}

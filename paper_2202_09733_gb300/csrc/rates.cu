// Arithmetic-pipe microbenchmarks behind the design choices of the residual kernels:
// FP64 scalar fused multiply-add chains (DFMA) against the FP64 tensor-core instruction
// (DMMA, mma.sync m8n8k4 f64), and FP32 scalar fma chains.  Each kernel keeps many
// independent accumulators per thread (or per warp) in flight so that the pipe, not the
// dependency latency, bounds it; the host times a launch with CUDA events.
//
// Exported (C ABI): frr_rate(kind, iters, &tflops, &checksum) with kind 0 DFMA, 1 DMMA,
// 2 FFMA.  Built into its own library (librates.so), not part of the solver.
#include <cuda_runtime.h>
#include <stdio.h>

#define NCHAIN 8

__global__ void __launch_bounds__(256) k_dfma(double *out, int iters, double a, double b) {
    double x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = 1e-3 * threadIdx.x + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ffma(float *out, int iters, float a, float b) {
    float x[2 * NCHAIN];
#pragma unroll
    for (int c = 0; c < 2 * NCHAIN; ++c) x[c] = 1e-3f * threadIdx.x + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < 2 * NCHAIN; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 2 * NCHAIN; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one m8n8k4 FP64 MMA per accumulator pair: D(8x8) = A(8x4) B(4x8) + C; each thread
// holds one element of A and of B and two of C/D; NACC independent accumulators per warp
#define NACC 8
__global__ void __launch_bounds__(256) k_dmma(double *out, int iters, double a0, double b0) {
    double a = a0 + 1e-3 * threadIdx.x, b = b0 - 1e-3 * threadIdx.x;
    double d[NACC][2];
#pragma unroll
    for (int c = 0; c < NACC; ++c) { d[c][0] = c; d[c][1] = -c; }
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < NACC; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[c][0]), "+d"(d[c][1]) : "d"(a), "d"(b));
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NACC; ++c) s += d[c][0] + d[c][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" int frr_rate(int kind, int iters, double *tflops, double *checksum) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = nsm * 8;
    const size_t n = (size_t)threads * blocks;
    void *out = nullptr;
    if (cudaMalloc(&out, n * sizeof(double)) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double flops = 0.0;
    for (int rep = 0; rep < 2; ++rep) {          // the first launch warms up, the second is timed
        cudaEventRecord(e0);
        if (kind == 0) {
            k_dfma<<<blocks, threads>>>((double *)out, iters, 0.999999, 1e-7);
            flops = 2.0 * NCHAIN * iters * (double)n;
        } else if (kind == 1) {
            k_dmma<<<blocks, threads>>>((double *)out, iters, 0.5, 0.25);
            flops = 2.0 * 8 * 8 * 4 * NACC * (double)iters * (double)(n / 32);
        } else {
            k_ffma<<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
            flops = 2.0 * 2 * NCHAIN * iters * (double)n;
        }
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int rc = cudaGetLastError() == cudaSuccess ? 0 : -1;
    double h = 0.0;
    if (kind == 2) {
        float hf = 0.f;
        cudaMemcpy(&hf, out, sizeof(float), cudaMemcpyDeviceToHost);
        h = hf;
    } else {
        cudaMemcpy(&h, out, sizeof(double), cudaMemcpyDeviceToHost);
    }
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = flops / (ms * 1e-3) / 1e12;
    *checksum = h;
    return rc;
}

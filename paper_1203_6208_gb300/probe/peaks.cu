// peaks.cu -- arithmetic-pipe throughput probes used as roofline
// denominators for the ALU-bound kernels (FP64 DFMA, FP64 DMMA m8n8k4, FP32
// FFMA, MUFU ex2).  Each kernel runs independent dependency chains long
// enough to hide latency; the result is written so nothing is optimised out.
#include <cuda_runtime.h>
#include <stdint.h>

__global__ void k_dfma(double *out, int iters, double b, double c)
{
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma(float *out, int iters, float b, float c)
{
    float a[16];
#pragma unroll
    for (int j = 0; j < 16; j++) a[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 16; j++) a[j] = fmaf(a[j], b, c);
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < 16; j++) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ex2(float *out, int iters)
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] = -(threadIdx.x & 7) * 1e-3f - j * 1e-4f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[j]));
            a[j] = y - 1.0f;
        }
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// DMMA: D(8x8) = A(8x4) B(4x8) + C, FP64; 4 independent accumulators
__global__ void k_dmma(double *out, int iters)
{
    double a = 1.0 + threadIdx.x * 1e-6, b = 1.0 - threadIdx.x * 1e-6;
    double d[4][2];
#pragma unroll
    for (int j = 0; j < 4; j++) { d[j][0] = 0.0; d[j][1] = 0.0; }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            asm volatile(
                "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                : "+d"(d[j][0]), "+d"(d[j][1])
                : "d"(a), "d"(b));
        }
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) s += d[j][0] + d[j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// which: 0 DFMA, 1 DMMA, 2 FFMA, 3 MUFU ex2.  Returns operations per second
// (flops for 0-2, ex2 results for 3) or a negative value on error.
extern "C" double bd_probe_peak(int which, int iters, int blocks, int threads)
{
    void *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)blocks * threads * 8) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double ops = 0;
    for (int rep = 0; rep < 2; rep++) {      // first launch warms up
        cudaEventRecord(e0);
        switch (which) {
        case 0:
            k_dfma<<<blocks, threads>>>((double *)buf, iters, 0.999999, 1e-7);
            ops = 2.0 * 8 * (double)iters * blocks * threads;
            break;
        case 1:
            k_dmma<<<blocks, threads>>>((double *)buf, iters);
            ops = 2.0 * 8 * 8 * 4 * 4 * (double)iters * blocks * (threads / 32);
            break;
        case 2:
            k_ffma<<<blocks, threads>>>((float *)buf, iters, 0.999999f, 1e-7f);
            ops = 2.0 * 16 * (double)iters * blocks * threads;
            break;
        default:
            k_ex2<<<blocks, threads>>>((float *)buf, iters);
            ops = 8.0 * (double)iters * blocks * threads;
            break;
        }
        cudaEventRecord(e1);
    }
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess || ms <= 0) return -2.0;
    return ops / (ms * 1e-3);
}

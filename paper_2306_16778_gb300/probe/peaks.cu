// peaks.cu -- measurement probe (not part of the method): FMA throughput of the
// FP64 and FP32 pipes, used as the denominator of the "alu" rooflines, and of the
// packed two-lane binary32 FMA (fma.rn.f32x2, sm_100 and later).
// Each thread runs 8 independent FMA chains so that issue, not latency, binds.
#include <cuda_runtime.h>
#include <stdint.h>

template <class T>
__global__ void fma_chains(T *out, int iters, T a, T b) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)12345.678) out[0] = s;  // keeps the chains alive
}

// Packed binary32 pairs: one fma.rn.f32x2 performs two binary32 FMAs.
__global__ void fma_chains_x2(float *out, int iters, float a, float b) {
    unsigned long long x[8], av, bv;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b), "f"(b));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float v = (float)(threadIdx.x + k);
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(v), "f"(v + 0.5f));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < 8; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
        s += lo + hi;
    }
    if (s == 12345.678f) out[0] = s;
}

// kind 0: binary64, kind 1: binary32, kind 2: packed binary32 pairs (2 FMAs per instruction).  Returns achieved TFLOP/s (2 flops per FMA),
// best of `reps` launches, or a negative value on a CUDA error.
extern "C" double expm_probe_fma_tflops(int kind, int iters, int blocks_per_sm, int reps) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *out = nullptr;
    if (cudaMalloc(&out, 64) != cudaSuccess) return -1.0;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int threads = 256;
    const int blocks = sms * blocks_per_sm;
    double best = 0.0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a);
        if (kind == 0)
            fma_chains<double><<<blocks, threads>>>((double *)out, iters, 0.999999, 1e-7);
        else if (kind == 1)
            fma_chains<float><<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
        else
            fma_chains_x2<<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double flops = (kind == 2 ? 2.0 : 1.0) * 2.0 * 8 * 16 * (double)iters * threads * blocks;
        if (ms > 0) best = best > flops / (ms * 1e-3) ? best : flops / (ms * 1e-3);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    return e == cudaSuccess ? best / 1e12 : -1.0;
}

// peak_probe.cu -- live throughput probe of the FP64 and FP32 FMA pipes
// (libplk_probe.so).  Used by the benchmark to state its roofline denominator
// for FP64-pipe-bound kernels: MEASURED_PEAKS-style numbers exist only for HBM
// copy and bf16 GEMM, not for FP64.  Not part of the paper's method.
#include <cuda_runtime.h>
#include <stdint.h>

template <class T, int ITERS>
__global__ void fma_chain(T *out, T a, T b) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
#pragma unroll 4
    for (int i = 0; i < ITERS; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class T>
static double run(int reps) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    constexpr int IT = 4096;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chain<T, IT><<<blocks, threads>>>(out, (T)0.999, (T)0.001);
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        fma_chain<T, IT><<<blocks, threads>>>(out, (T)0.999, (T)0.001);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return 2.0 * 8 * IT * (double)blocks * threads / (best * 1e-3) / 1e12;
}

extern "C" double plk_probe_fp64_fma_tflops(int reps) { return run<double>(reps); }
extern "C" double plk_probe_fp32_fma_tflops(int reps) { return run<float>(reps); }

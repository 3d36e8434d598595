// peak_probe.cu -- live throughput probes of the FP64 and FP32 FMA pipes, the
// FP64 tensor MMA (DMMA) and the tcgen05 bf16 MMA, and the FP64 issue cost
// against active lanes
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

// ---------------------------------------------------------------------------
// FP64 issue cost against active lanes: one block of `warps` warps, in each
// warp the lanes below `active` run a dependent chain of ITERS FP64 FMAs,
// timed by clock64 between two block barriers.  Returns SM cycles per warp
// FMA instruction (per warp: the chain length over ITERS).
// ---------------------------------------------------------------------------
template <int ITERS>
__global__ void fp64_lane_chain(double *out, int active, long long *cyc) {
    const int lane = threadIdx.x & 31;
    double a = 1.0 + threadIdx.x * 1e-9;
    const double b = 0.999999, c = 1e-7;
    __syncthreads();
    const long long t0 = clock64();
    if (lane < active) {
#pragma unroll 16
        for (int i = 0; i < ITERS; ++i) a = fma(a, b, c);
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) *cyc = t1 - t0;
    out[threadIdx.x] = a;
}

extern "C" double plk_probe_fp64_cycles_per_warp_fma(int warps, int active) {
    if (warps < 1 || warps > 16 || active < 1 || active > 32) return -1.0;
    constexpr int IT = 4096;
    double *out = nullptr;
    long long *cyc = nullptr, h = 0;
    if (cudaMalloc(&out, sizeof(double) * 32 * 16) != cudaSuccess) return -1.0;
    if (cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) {
        cudaFree(out);
        return -1.0;
    }
    fp64_lane_chain<IT><<<1, 32 * warps>>>(out, active, cyc);   // warm-up
    fp64_lane_chain<IT><<<1, 32 * warps>>>(out, active, cyc);
    const bool ok = cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(out);
    cudaFree(cyc);
    if (!ok || cudaGetLastError() != cudaSuccess) return -1.0;
    return (double)h / IT;
}

// ---------------------------------------------------------------------------
// FP64 tensor-core MMA (DMMA, mma.sync m8n8k4 f64): eight independent
// accumulator chains per warp, 8 warps per block, 4 blocks per SM.
// ---------------------------------------------------------------------------
template <int ITERS>
__global__ void dmma_chain(double *out, double a0, double b0) {
    double acc[8][2];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double a = a0 + 1e-3 * threadIdx.x, b = b0;
#pragma unroll 2
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(acc[c][0]), "+d"(acc[c][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c][0] + acc[c][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" double plk_probe_fp64_mma_tflops(int reps) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 4, threads = 256;
    constexpr int IT = 1024;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dmma_chain<IT><<<blocks, threads>>>(out, 0.5, 1e-3);
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        dmma_chain<IT><<<blocks, threads>>>(out, 0.5, 1e-3);
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
    // one m8n8k4 MMA per warp = 2 * 8 * 8 * 4 flops
    const double warps = (double)blocks * threads / 32;
    return 2.0 * 8 * 8 * 4 * 8.0 * IT * warps / (best * 1e-3) / 1e12;
}

// ---------------------------------------------------------------------------
// tcgen05 bf16 MMA from shared memory (kind::f16, M = 128, K = 16 per
// instruction, FP32 accumulator in TMEM), one CTA per SM, one issuing thread:
// the rate the 5th-generation tensor core reaches with both operands read
// from shared memory, for N = 64, 128 and 256.  The operands are zeros (the
// rate does not depend on the values).  Every wait is bounded.
// ---------------------------------------------------------------------------
#include "../csrc/plk_tc.cuh"

namespace {
constexpr int TC_SMEM = 120 * 1024;   // > half the SM's shared memory: one CTA per SM

__global__ void __launch_bounds__(128, 1) tc_mma_probe(int N, int iters, int *err) {
    using namespace plk;
    extern __shared__ uint8_t smraw[];
    uint8_t *sA = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t *sB = sA + 16384;                       // up to 256 rows x 128 bytes
    __shared__ uint64_t done;
    __shared__ uint32_t tmem;
    const int tid = threadIdx.x;
    for (int i = tid; i < (16384 + 32768) / 16; i += blockDim.x) reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
    }
    if (tid < 32) {
        tc::tmem_alloc(&tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
        const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(sA)), b0 = tc::sdesc_sw128(tc::smem_u32(sB));
        const uint32_t idesc = tc::idesc_bf16_f32(128, N);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(tmem + 256 * (it & 1), a0 + 2 * kk, b0 + 2 * kk, idesc, (it > 1 || kk) ? 1u : 0u);
        tc::mma_commit(&done);
        if (!tc::mbar_wait(&done, 0)) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(tmem, 512);
}
}  // namespace

// bf16 TFLOP/s of tcgen05.mma with N columns (64, 128 or 256); -1 on error.
extern "C" double plk_probe_tcgen05_bf16_tflops(int N, int reps) {
    if (N != 64 && N != 128 && N != 256) return -1.0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(tc_mma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess)
        return -1.0;
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return -1.0;
    cudaMemset(err, 0, sizeof(int));
    const int iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    tc_mma_probe<<<sms, 128, TC_SMEM>>>(N, iters, err);
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        tc_mma_probe<<<sms, 128, TC_SMEM>>>(N, iters, err);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    int h = 0;
    cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(err);
    if (cudaGetLastError() != cudaSuccess || h) return -1.0;
    return 2.0 * 128 * N * 16 * 4.0 * iters * sms / (best * 1e-3) / 1e12;
}

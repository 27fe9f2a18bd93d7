// bench_fma_peak.cu -- measurement tooling for bench.py, built into its own
// libps_bench.so and not part of the solver library's ABI (include/ps.h).
// It measures the fused multiply-add rate of the current device, the ALU
// ceiling that the FP64 step is held against (the FP64 path moves half the
// bytes per second of the FP32 path but runs several times slower, so on
// this part it is bound by FP64 arithmetic, not by HBM).
//
// Each thread runs 8 independent FMA chains for `iters` iterations (8
// chains hide the FMA latency); the grid is 8 blocks of 256 threads per SM.
// FLOPs = 2 x 8 x iters x threads. The only memory access is one store to a
// fixed device sink in a branch that no run takes, which keeps the chains
// live.
#include <cuda_runtime.h>

#include <stdint.h>

// status codes as in include/ps.h
enum { kOk = 0, kEinval = 1, kEcuda = 3 };
enum { kFp32 = 0, kFp64 = 1 };

static __device__ double ps_peak_sink;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T seed) {
    T a[8];
    const T b = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < 8; ++i) a[i] = seed + (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    T s = a[0] + a[1] + a[2] + a[3] + a[4] + a[5] + a[6] + a[7];
    if (s == (T)-1.2345e30) ps_peak_sink = (double)s;
}

// FLOP/s (an FMA counts 2) of k_fma_chains in `precision` (0 FP32, 1 FP64):
// 8 blocks of 256 threads per SM, timed with CUDA events on cuda_stream
// after one warm-up launch. Synchronises.
extern "C" int32_t bench_fma_peak(int32_t precision, int32_t iters, void* cuda_stream, double* flops_per_s) {
    if (!flops_per_s || iters < 1 || (precision != kFp32 && precision != kFp64)) return kEinval;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return kEcuda;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = 8 * nsm, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return kEcuda;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return kEcuda;
    }
    float ms = 0.0f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, s);
        if (precision == kFp64) k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 1.0);
        else k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 1.0f);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || !(ms > 0.0f)) return kEcuda;
    *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
    return kOk;
}

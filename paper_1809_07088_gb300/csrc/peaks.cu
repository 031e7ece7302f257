// Throughput of the arithmetic pipes the ALU-bound kernels use, measured on the device (no
// counterpart in the paper; the denominators of the ALU rooflines of the benchmark).
//
// Each kernel keeps 8 independent dependency chains per thread for ITER iterations on a grid of
// 8 CTAs of 256 threads per SM, times the launch with CUDA events and reports operations per second:
//   0  FP32 fused multiply-add (FFMA), in flop (2 per FMA)
//   1  FP32 paired fused multiply-add on float2 (FFMA2), in flop (4 per instruction)
//   2  FP64 fused multiply-add, in flop
//   3  FP32 base-2 exponential of the SFU (ex2.approx), in operations
//   4  FP32 sine and cosine of the SFU (__sincosf), in (sin, cos) pairs
// The chain values are stored only if a runtime flag (never set) asks for it, so the compiler keeps
// the arithmetic.
#include <cuda_runtime.h>

#include "../../include/ds.h"
#include "internal.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;
constexpr int PK_ITER = 4096;

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(float seed, int store, float *sink) {
    float v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = seed + threadIdx.x * 1e-7f + c;
    const float a = 0.999999f, b = 1e-7f;
    for (int i = 0; i < PK_ITER; ++i)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = fmaf(v[c], a, b);
    if (store) {
        float t = 0.f;
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) t += v[c];
        sink[blockIdx.x * PK_THREADS + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma2(float seed, int store, float *sink) {
    float2 v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = make_float2(seed + threadIdx.x * 1e-7f + c, seed - c);
    const float2 a = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < PK_ITER; ++i)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = __ffma2_rn(v[c], a, b);
    if (store) {
        float t = 0.f;
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) t += v[c].x + v[c].y;
        sink[blockIdx.x * PK_THREADS + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(double seed, int store, double *sink) {
    double v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = seed + threadIdx.x * 1e-9 + c;
    const double a = 0.999999999, b = 1e-9;
    for (int i = 0; i < PK_ITER / 16; ++i)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = fma(v[c], a, b);
    if (store) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) t += v[c];
        sink[blockIdx.x * PK_THREADS + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_ex2(float seed, int store, float *sink) {
    float v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = -1e-3f * (threadIdx.x & 7) - 1e-4f * c + seed;
    for (int i = 0; i < PK_ITER / 4; ++i)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = ds::exp2_w(v[c]) - 1.0f;
    if (store) {
        float t = 0.f;
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) t += v[c];
        sink[blockIdx.x * PK_THREADS + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_sincos(float seed, int store, float *sink) {
    float v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = 1e-3f * (threadIdx.x & 7) + 1e-4f * c + seed;
    for (int i = 0; i < PK_ITER / 8; ++i)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) {
            float s, co;
            __sincosf(v[c], &s, &co);
            v[c] = s + co;
        }
    if (store) {
        float t = 0.f;
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) t += v[c];
        sink[blockIdx.x * PK_THREADS + threadIdx.x] = t;
    }
}

template <typename F> float time_kernel(F launch, cudaEvent_t e0, cudaEvent_t e1) {
    launch();  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 5.f;
}

}  // namespace

extern "C" ds_status ds_measure_peaks(int device, double out[5]) {
    if (!out) return DS_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DS_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return DS_ERR_CUDA;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int nblk = 8 * nsm;
    const double threads = (double)nblk * PK_THREADS;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return DS_ERR_CUDA;
    float ms;
    ms = time_kernel([&] { k_peak_ffma<<<nblk, PK_THREADS>>>(0.5f, 0, nullptr); }, e0, e1);
    out[0] = threads * PK_CHAINS * PK_ITER * 2.0 / (ms * 1e-3) / 1e12;
    ms = time_kernel([&] { k_peak_ffma2<<<nblk, PK_THREADS>>>(0.5f, 0, nullptr); }, e0, e1);
    out[1] = threads * PK_CHAINS * PK_ITER * 4.0 / (ms * 1e-3) / 1e12;
    ms = time_kernel([&] { k_peak_dfma<<<nblk, PK_THREADS>>>(0.5, 0, nullptr); }, e0, e1);
    out[2] = threads * PK_CHAINS * (PK_ITER / 16) * 2.0 / (ms * 1e-3) / 1e12;
    ms = time_kernel([&] { k_peak_ex2<<<nblk, PK_THREADS>>>(0.0f, 0, nullptr); }, e0, e1);
    out[3] = threads * PK_CHAINS * (PK_ITER / 4) / (ms * 1e-3) / 1e12;
    ms = time_kernel([&] { k_peak_sincos<<<nblk, PK_THREADS>>>(0.1f, 0, nullptr); }, e0, e1);
    out[4] = threads * PK_CHAINS * (PK_ITER / 8) / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ds::count_launches(30);
    return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ERR_CUDA;
}

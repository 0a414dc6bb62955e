// Arithmetic-rate probe (md_fma_rate): the measured peak that the FP64
// solver form's roofline is reported against.  Every thread runs 8
// independent fused multiply-add chains of a fixed length, so the pipe, not
// the dependency latency, sets the time; the grid fills every SM.  Bounded:
// the chain length is fixed (about 1e10 FP64 or 8e10 FP32 multiply-adds on
// 152 SMs, some 20 ms and 3 ms on GB300).
#include <cuda_runtime.h>

#include <string>

#include "md_internal.h"

namespace md {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b, T* out) {
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = v[c] * a + b;
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == (T)-1) out[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

template <class T>
md_status fma_rate(int iters, cudaStream_t s, double* tflops) {
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_sm * 8;
    T* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, grid * sizeof(T));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fma_chains<T><<<grid, kThreads, 0, s>>>(iters / 8, (T)0.999999, (T)1e-7, out);   // warm-up
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<grid, kThreads, 0, s>>>(iters, (T)0.999999, (T)1e-7, out);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    const double fmas = (double)grid * kThreads * kChains * (double)iters;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return MD_OK;
}

}  // namespace

md_status fma_rate_probe(int precision, cudaStream_t s, double* tflops) {
    if (precision == MD_PREC_FP64) return fma_rate<double>(1 << 12, s, tflops);
    return fma_rate<float>(1 << 15, s, tflops);
}

}  // namespace md

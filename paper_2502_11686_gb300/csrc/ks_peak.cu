// ks_peak.cu -- ks_measure_fma_rate: the FP64 / FP32 FMA rate of the device, measured.
//
// The rooflines of the arithmetic-bound kernels (whitening, levels and SelInv at every state
// dimension in FP64) are taken against the rate the FMA pipe actually sustains, measured here
// rather than read from a datasheet.  Every thread runs eight independent FMA chains (enough
// to cover the pipe latency at eight warps per SM); two launches, the second timed with CUDA
// events on a private stream.
#include <cuda_runtime.h>

#include "../../include/ks.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* sink, int iters) {
    T a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    const T b = (T)0.999, d = (T)1e-4;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == (T)12345.678) sink[0] = s;   // never true; keeps the chains live
}

template <typename T>
ks_status measure(int sms, double* tflops) {
    const int threads = 256, iters = T(0.5) == 0.5f ? 4000 : 20000;
    const int blocks = sms * 4;   // 32 warps per SM
    T* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ks_status rc = KS_ERR_CUDA;
    float ms = 0.f;
    if (cudaMalloc(&sink, 16) != cudaSuccess) { rc = KS_ERR_OOM; goto out; }
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) goto out;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto out;
    fma_rate_kernel<T><<<blocks, threads, 0, st>>>(sink, iters / 10);
    cudaEventRecord(e0, st);
    fma_rate_kernel<T><<<blocks, threads, 0, st>>>(sink, sizeof(T) == 4 ? iters * 25 : iters);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) goto out;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) goto out;
    *tflops = 2.0 * 8.0 * (double)blocks * threads * (sizeof(T) == 4 ? iters * 25.0 : iters) /
              (ms * 1e-3) / 1e12;
    rc = KS_OK;
out:
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    return rc;
}

}  // namespace

extern "C" ks_status ks_measure_fma_rate(int device, int precision, double* tflops) {
    if (!tflops || (precision != KS_FP64 && precision != KS_FP32_REFINE)) return KS_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return KS_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const ks_status rc = precision == KS_FP64 ? measure<double>(sms > 0 ? sms : 1, tflops)
                                              : measure<float>(sms > 0 ? sms : 1, tflops);
    cudaSetDevice(prev);
    return rc;
}

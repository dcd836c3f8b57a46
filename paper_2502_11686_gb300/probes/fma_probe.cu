// fma_probe.cu -- FMA issue rates of the GPU: DFMA and FFMA, full vs partially active warps,
// warps per SM.  Gives the FP64 / FP32 rates the kernels are measured against.
// Build and run: python -m paper_2502_11686_gb300.probes
#include <cstdio>
#include <cuda_runtime.h>
template <typename T, int CH>
__global__ void fma_kernel(T* out, int iters, int active_lanes) {
    T a[CH];
    for (int c = 0; c < CH; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    const T b = (T)0.999, d = (T)1e-4;
    if ((threadIdx.x & 31) < active_lanes) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < CH; ++c) a[c] = fma(a[c], b, d);
        }
    }
    T s = 0;
    for (int c = 0; c < CH; ++c) s += a[c];
    if (s == (T)12345.678) out[0] = s;
}
template <typename T, int CH>
double run(int blocks, int threads, int iters, int active) {
    T* out; cudaMalloc(&out, 16);
    fma_kernel<T, CH><<<blocks, threads>>>(out, 10, active);
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0);
    fma_kernel<T, CH><<<blocks, threads>>>(out, iters, active);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(out);
    double lanes = (double)blocks * threads * active / 32.0;
    return 2.0 * lanes * iters * CH / (ms * 1e-3) / 1e12;  // TFLOP/s of useful lanes
}
int main() {
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    printf("SMs %d clock %d kHz\n", sms, clk);
    for (int wps : {1, 2, 4, 8, 16}) {
        double t = run<double, 8>(sms, 32 * wps, 20000, 32);
        printf("DFMA ILP8 warps/SM %2d : %.3f TFLOP/s\n", wps, t);
    }
    for (int act : {32, 16, 8, 1}) {
        double t = run<double, 8>(sms, 32 * 8, 20000, act);
        printf("DFMA ILP8 8 warps/SM active lanes %2d : useful %.3f TFLOP/s\n", act, t);
    }
    for (int wps : {1, 4, 8}) {
        double t = run<double, 1>(sms, 32 * wps, 20000, 32);
        printf("DFMA ILP1 (dependent chain) warps/SM %2d : %.3f TFLOP/s\n", wps, t);
    }
    for (int wps : {4, 8, 16, 32}) {
        double t = run<float, 8>(sms, 32 * wps, 20000, 32);
        printf("FFMA ILP8 warps/SM %2d : %.2f TFLOP/s\n", wps, t);
    }
    return 0;
}

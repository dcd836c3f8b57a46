// tc_probe.cu -- checks the tcgen05 conventions of csrc/ks_tc.cuh on the GPU.  One block of
// four warps computes D = A B^T (M = 128 rows, N columns, depth K) as 3xTF32 twice -- A from
// shared memory and A from tensor memory, B from shared memory -- and the host compares both
// with an FP64 product.  Every index stays inside its buffer; the MMA completion wait is
// bounded.  Build and run: python -m paper_2502_11686_gb300.probes tc
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../csrc/ks_tc.cuh"

using namespace ks::tc;
constexpr int M = 128;

__global__ void __launch_bounds__(128) probe_k(int N, int K, const float* A, const float* B,
                                               float* Dss, float* Dts, int* status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float* Ahi = reinterpret_cast<float*>(sm);   // M x K, tile layout
    float* Alo = Ahi + M * K;
    float* Bhi = Alo + M * K;                     // N x K, tile layout
    float* Blo = Bhi + N * K;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + N * K);
    uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tmem_alloc(slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) mbar_init(mbar, 1);
    for (int e = tid; e < M * K; e += blockDim.x) {
        const int m = e / K, k = e - m * K;
        const float x = A[e], h = tf32_hi(x);
        const uint32_t off = tile_off(M, m, k) >> 2;
        Ahi[off] = h;
        Alo[off] = x - h;
    }
    for (int e = tid; e < N * K; e += blockDim.x) {
        const int n = e / K, k = e - n * K;
        const float x = B[e], h = tf32_hi(x);
        const uint32_t off = tile_off(N, n, k) >> 2;
        Bhi[off] = h;
        Blo[off] = x - h;
    }
    fence_proxy_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *slot;
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    {   // A into TMEM: row 32 warp + lane; hi at columns [0, K), lo at [K, 2K)
        const int m = 32 * warp + lane;
        for (int c0 = 0; c0 < K; c0 += 32) {
            float h[32], l[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float x = A[m * K + c0 + j];
                h[j] = tf32_hi(x);
                l[j] = x - h[j];
            }
            tmem_st32(tbase + lanes + (uint32_t)c0, h);
            tmem_st32(tbase + lanes + (uint32_t)(K + c0), l);
        }
    }
    fence_before();
    __syncthreads();
    const uint32_t dss = tbase + (uint32_t)(2 * K), dts = dss + (uint32_t)N;
    if (tid == 0) {
        fence_after();
        const uint32_t id = idesc_tf32(M, N);
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
        for (int s = 0; s < K / 8; ++s) {
            mma_ss(dss, tile_desc(al, M, s), tile_desc(bh, N, s), id, s > 0 ? 1u : 0u);
            mma_ss(dss, tile_desc(ah, M, s), tile_desc(bl, N, s), id, 1u);
            mma_ss(dss, tile_desc(ah, M, s), tile_desc(bh, N, s), id, 1u);
        }
        for (int s = 0; s < K / 8; ++s) {
            mma_ts(dts, tbase + (uint32_t)(K + 8 * s), tile_desc(bh, N, s), id, s > 0 ? 1u : 0u);
            mma_ts(dts, tbase + (uint32_t)(8 * s), tile_desc(bl, N, s), id, 1u);
            mma_ts(dts, tbase + (uint32_t)(8 * s), tile_desc(bh, N, s), id, 1u);
        }
        commit(mbar);
    }
    __syncwarp();
    if (!mbar_wait(mbar, 0, 1u << 22) && lane == 0) atomicExch(status, 1);
    fence_after();
    {
        const int m = 32 * warp + lane;
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tmem_ld32(dss + lanes + (uint32_t)c0, v);
            for (int j = 0; j < 32; ++j) Dss[m * N + c0 + j] = v[j];
            tmem_ld32(dts + lanes + (uint32_t)c0, v);
            for (int j = 0; j < 32; ++j) Dts[m * N + c0 + j] = v[j];
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

static int run(int N, int K) {
    std::vector<float> A(M * K), B(N * K), Dss(M * N), Dts(M * N);
    srand(1234 + N + K);
    for (auto& x : A) x = 2.0f * (float)rand() / (float)RAND_MAX - 1.0f;
    for (auto& x : B) x = 2.0f * (float)rand() / (float)RAND_MAX - 1.0f;
    float *dA, *dB, *dss, *dts;
    int* dst;
    cudaMalloc(&dA, A.size() * 4);
    cudaMalloc(&dB, B.size() * 4);
    cudaMalloc(&dss, Dss.size() * 4);
    cudaMalloc(&dts, Dts.size() * 4);
    cudaMalloc(&dst, 4);
    cudaMemset(dst, 0, 4);
    cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice);
    const size_t smem = (size_t)(2 * M * K + 2 * N * K) * 4 + 16;
    cudaFuncSetAttribute(probe_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    probe_k<<<1, 128, smem>>>(N, K, dA, dB, dss, dts, dst);
    cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        printf("N=%d K=%d: CUDA error %s\n", N, K, cudaGetErrorString(err));
        return 1;
    }
    int st = 0;
    cudaMemcpy(&st, dst, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(Dss.data(), dss, Dss.size() * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(Dts.data(), dts, Dts.size() * 4, cudaMemcpyDeviceToHost);
    double emax_ss = 0, emax_ts = 0, ref = 0;
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            double s = 0;
            for (int k = 0; k < K; ++k) s += (double)A[m * K + k] * (double)B[n * K + k];
            ref = fmax(ref, fabs(s));
            emax_ss = fmax(emax_ss, fabs(Dss[m * N + n] - s));
            emax_ts = fmax(emax_ts, fabs(Dts[m * N + n] - s));
        }
    printf("M=128 N=%d K=%d: wait %s; max |D - A B^T| / max |A B^T|: A in smem %.2e, A in TMEM %.2e\n",
           N, K, st ? "TIMED OUT" : "ok", emax_ss / ref, emax_ts / ref);
    cudaFree(dA); cudaFree(dB); cudaFree(dss); cudaFree(dts); cudaFree(dst);
    return (st || emax_ss / ref > 1e-5 || emax_ts / ref > 1e-5) ? 1 : 0;
}

int main() {
    int bad = 0;
    bad |= run(32, 128);
    bad |= run(128, 64);
    bad |= run(128, 32);
    bad |= run(96, 32);
    printf(bad ? "tc probe: MISMATCH\n" : "tc probe: ok\n");
    return bad;
}

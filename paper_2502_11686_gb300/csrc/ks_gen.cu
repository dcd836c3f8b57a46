// ks_gen.cu -- synthetic smoothing problems generated on the device (input generation only; none
// of the smoother's arithmetic).  The serving loop uses it to create requests at admission
// without moving their inputs across the host link.
//
// Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): a counter-based generator, 10 rounds of the Philox S-box on a 128-bit
// counter with a 64-bit key bumped by the Weyl constants after each round.  Normals by the
// Box-Muller transform.  Stream layout: key = seed; counter = (element index, array tag).
//
// The problem (time invariant: one matrix each, used at every step):
//   F = f * Q with Q = (I - 2 v1 v1^T / |v1|^2)(I - 2 v2 v2^T / |v2|^2)(I - 2 v3 v3^T / |v3|^2),
//       v_j ~ N(0, I) (orthogonal by construction);
//   H = I;  K = L_K L_K^T,  C = L_C L_C^T with L lower triangular, diagonal U[0.5, 1.5],
//       off-diagonal N(0, 0.1^2);  G ~ N(0, 1/n) (m x n);  o_i ~ N(0, 1) per step.
#include "ks_internal.cuh"

namespace ks {

struct Philox {
    __device__ static void round(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        const uint32_t hi0 = __umulhi(m0, c[0]), lo0 = m0 * c[0];
        const uint32_t hi1 = __umulhi(m1, c[2]), lo1 = m1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    // Four 32-bit words for counter (idx, tag) under key seed.
    __device__ static void draw(uint64_t seed, uint64_t idx, uint32_t tag, uint32_t (&out)[4]) {
        uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), tag, 0x243F6A88u};
        uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        for (int r = 0; r < 10; ++r) {
            round(c, k0, k1);
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
    }
};

__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {   // (0, 1], 53 bits
    const uint64_t x = ((uint64_t)a << 21) ^ (uint64_t)b;
    return ((double)(x & ((1ULL << 53) - 1)) + 1.0) * (1.0 / 9007199254740992.0);
}

// Standard normal number `idx` of array `tag`.
__device__ double gauss(uint64_t seed, uint32_t tag, uint64_t idx) {
    uint32_t w[4];
    Philox::draw(seed, idx, tag, w);
    const double r = sqrt(-2.0 * log(u01(w[0], w[1])));
    return r * cospi(2.0 * u01(w[2], w[3]));
}

__device__ double uniform(uint64_t seed, uint32_t tag, uint64_t idx) {
    uint32_t w[4];
    Philox::draw(seed, idx, tag, w);
    return u01(w[0], w[1]);
}

enum { TAG_V = 1, TAG_LK = 2, TAG_DK = 3, TAG_LC = 4, TAG_DC = 5, TAG_G = 6, TAG_O = 7,
       TAG_LKS = 8, TAG_DKS = 9, TAG_LCS = 10, TAG_DCS = 11, TAG_GS = 12 };

// One block builds the time-invariant matrices.  Shared memory: the three reflection vectors
// and the packed lower factor L of K or C (max(n, m)^2 / 2 doubles); F is formed in place in
// device memory, one row per thread (each reflection only mixes the entries of a row).
__global__ void gen_model_kernel(int n, int m, uint64_t seed, double f_scale, double* F, double* H,
                                 double* K, double* G, double* C) {
    extern __shared__ double sh[];
    double* V = sh;              // 3 x n reflection vectors
    double* Lp = sh + 3 * n;     // packed lower factor, row r at r (r + 1) / 2
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < 3 * n; e += nth) V[e] = gauss(seed, TAG_V, e);
    __syncthreads();
    double vv[3];
    for (int j = 0; j < 3; ++j) {
        vv[j] = 0.0;
        for (int p = 0; p < n; ++p) vv[j] = fma(V[j * n + p], V[j * n + p], vv[j]);
    }
    // F <- I (I - 2 v1 v1^T / |v1|^2)(I - 2 v2 v2^T / |v2|^2)(I - 2 v3 v3^T / |v3|^2), row by row.
    for (int r = tid; r < n; r += nth) {
        double* Fr = F + (int64_t)r * n;
        for (int p = 0; p < n; ++p) Fr[p] = (p == r) ? 1.0 : 0.0;
        for (int j = 0; j < 3; ++j) {
            const double* v = V + j * n;
            double s = 0.0;
            for (int p = 0; p < n; ++p) s = fma(Fr[p], v[p], s);
            s *= 2.0 / vv[j];
            for (int p = 0; p < n; ++p) Fr[p] = fma(-s, v[p], Fr[p]);
        }
        for (int p = 0; p < n; ++p) {
            Fr[p] *= f_scale;
            H[(int64_t)r * n + p] = (p == r) ? 1.0 : 0.0;
        }
    }
    // K = L L^T and C = L L^T.
    for (int which = 0; which < 2; ++which) {
        const int d = which == 0 ? n : m;
        double* out = which == 0 ? K : C;
        if (d == 0) continue;
        const uint32_t tl = which == 0 ? TAG_LK : TAG_LC, td = which == 0 ? TAG_DK : TAG_DC;
        __syncthreads();
        for (int e = tid; e < d * d; e += nth) {
            const int r = e / d, c = e % d;
            if (c <= r) Lp[r * (r + 1) / 2 + c] = c < r ? 0.1 * gauss(seed, tl, e) : 0.5 + uniform(seed, td, r);
        }
        __syncthreads();
        for (int e = tid; e < d * d; e += nth) {
            const int r = e / d, c = e % d;
            const double* Lr = Lp + r * (r + 1) / 2;
            const double* Lc = Lp + c * (c + 1) / 2;
            double s = 0.0;
            for (int p = 0; p <= (r < c ? r : c); ++p) s = fma(Lr[p], Lc[p], s);
            out[e] = s;
        }
    }
    const double gs = sqrt(1.0 / n);
    for (int e = tid; e < m * n; e += nth) G[e] = gs * gauss(seed, TAG_G, e);
}

__global__ void gen_obs_kernel(int64_t count, uint64_t seed, double* o) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        o[e] = gauss(seed, TAG_O, (uint64_t)e);
}

cudaError_t launch_generate(int64_t k, int n, int m, uint64_t seed, double f_scale, double* F,
                            double* H, double* K, double* G, double* C, double* o,
                            cudaStream_t st) {
    const int d = n > m ? n : m;
    const size_t smem = sizeof(double) * (size_t)(3 * n + d * (d + 1) / 2);
    if (smem > (size_t)SMEM_OPTIN_SM103) return cudaErrorInvalidValue;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(gen_model_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gen_model_kernel<<<1, 256, smem, st>>>(n, m, seed, f_scale, F, H, K, G, C);
    ++t_launches;
    const int64_t count = k * (int64_t)m;
    if (count > 0) {
        int64_t b = (count + 255) / 256;
        gen_obs_kernel<<<(unsigned)(b > 8192 ? 8192 : b), 256, 0, st>>>(count, seed, o);
        ++t_launches;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Per-step draws (the batched-benchmark recipe): F_i = f Q for every step (Q as above, one draw
// per problem, stored for every step so that its traffic is real), H_i = I, and K_i, C_i = L L^T
// and G_i ~ N(0, 1/n) drawn independently for every step; o_i ~ N(0, 1).  Counters: array tag,
// element index step * (matrix size) + entry.  Persistent blocks; each forms Q once in shared
// memory and then writes the steps it owns.
__device__ void gen_spd_into(double* out, double* Lp, int d, uint64_t seed, uint32_t tl,
                             uint32_t td, uint64_t base) {
    const int tid = threadIdx.x, nth = blockDim.x;
    __syncthreads();
    for (int e = tid; e < d * d; e += nth) {
        const int r = e / d, c = e % d;
        if (c <= r)
            Lp[r * (r + 1) / 2 + c] = c < r ? 0.1 * gauss(seed, tl, base * d + e)
                                            : 0.5 + uniform(seed, td, base + r);
    }
    __syncthreads();
    for (int e = tid; e < d * d; e += nth) {
        const int r = e / d, c = e % d;
        const double* Lr = Lp + r * (r + 1) / 2;
        const double* Lc = Lp + c * (c + 1) / 2;
        double s = 0.0;
        for (int p = 0; p <= (r < c ? r : c); ++p) s = fma(Lr[p], Lc[p], s);
        out[e] = s;
    }
}

__global__ void gen_steps_kernel(int64_t k, int n, int m, uint64_t seed, double f_scale, double* F,
                                 double* H, double* K, double* G, double* C, double* o) {
    extern __shared__ double sh[];
    double* V = sh;                         // 3 x n reflection vectors
    double* Q = sh + 3 * n;                 // f Q, n x n
    double* Lp = Q + (size_t)n * n;         // packed lower factor
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t nn = (int64_t)n * n;
    for (int e = tid; e < 3 * n; e += nth) V[e] = gauss(seed, TAG_V, e);
    __syncthreads();
    double vv[3];
    for (int j = 0; j < 3; ++j) {
        vv[j] = 0.0;
        for (int p = 0; p < n; ++p) vv[j] = fma(V[j * n + p], V[j * n + p], vv[j]);
    }
    for (int r = tid; r < n; r += nth) {
        double* Qr = Q + (int64_t)r * n;
        for (int p = 0; p < n; ++p) Qr[p] = (p == r) ? 1.0 : 0.0;
        for (int j = 0; j < 3; ++j) {
            const double* v = V + j * n;
            double s = 0.0;
            for (int p = 0; p < n; ++p) s = fma(Qr[p], v[p], s);
            s *= 2.0 / vv[j];
            for (int p = 0; p < n; ++p) Qr[p] = fma(-s, v[p], Qr[p]);
        }
        for (int p = 0; p < n; ++p) Qr[p] *= f_scale;
    }
    __syncthreads();
    const double gs = sqrt(1.0 / n);
    for (int64_t i = blockIdx.x; i < k; i += gridDim.x) {
        if (i + 1 < k) {
            for (int e = tid; e < n * n; e += nth) {
                F[i * nn + e] = Q[e];
                H[i * nn + e] = (e / n == e % n) ? 1.0 : 0.0;
            }
            gen_spd_into(K + i * nn, Lp, n, seed, TAG_LKS, TAG_DKS, (uint64_t)i * n);
        }
        if (m > 0) {
            for (int e = tid; e < m * n; e += nth)
                G[i * m * n + e] = gs * gauss(seed, TAG_GS, (uint64_t)i * m * n + e);
            for (int e = tid; e < m; e += nth) o[i * m + e] = gauss(seed, TAG_O, (uint64_t)i * m + e);
            gen_spd_into(C + i * (int64_t)m * m, Lp, m, seed, TAG_LCS, TAG_DCS, (uint64_t)i * m);
        }
    }
}

cudaError_t launch_generate_steps(int64_t k, int n, int m, uint64_t seed, double f_scale, double* F,
                                  double* H, double* K, double* G, double* C, double* o,
                                  cudaStream_t st) {
    const int d = n > m ? n : m;
    const size_t smem = sizeof(double) * (size_t)(3 * n + n * n + d * (d + 1) / 2);
    if (smem > (size_t)SMEM_OPTIN_SM103) return cudaErrorInvalidValue;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(gen_steps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 4;
    gen_steps_kernel<<<(unsigned)(k < cap ? k : cap), 128, smem, st>>>(k, n, m, seed, f_scale, F, H, K,
                                                                         G, C, o);
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

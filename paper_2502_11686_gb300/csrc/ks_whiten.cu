// ks_whiten.cu -- whitening of every step (Section 2: V_i^T V_i = K_i^{-1}, W_i^T W_i = C_i^{-1}),
// producing the level-0 problem of the odd-even factorization.
//
// Per step i (one thread block): K_i = L_K L_K^T and C_i = L_C L_C^T by Cholesky in FP64 (the
// whitening factors are V_i = L_K^{-1}, W_i = L_C^{-1}); then
//     [-B | D | rE] = L_K^{-1} [-F_i | H_i | c_i]     (coupling row of column i+1)
//     [Chat | rC]   = L_C^{-1} [G_i | o_i]            (m_i x n observation block of column i)
// and the observation block is reduced to an n x n upper-triangular block by a Householder QR of
// [0 ; Chat] (the triangular-over-full routine with a zero triangle), so every level-0 column has
// the same shape whatever m_i is (m_i = 0 gives Chat = 0).  The rhs rows the reduction discards
// go to resid[i].  In KS_FP32_REFINE mode the Cholesky factors are also stored (FP64) for the
// refinement step and the level-0 blocks are rounded to FP32.
#include "ks_generic.cuh"

namespace ks {

template <typename T>
__global__ void __launch_bounds__(256) whiten_kernel(WhitenArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sm = reinterpret_cast<double*>(smem_raw);
    for (int64_t i = blockIdx.x; i < a.k; i += gridDim.x) whiten_cta_step<T>(a, i, sm);
}

cudaError_t launch_whiten(const WhitenArgs& a, bool fp32, cudaStream_t st) {
    if (!use_large(a.n, fp32))
        if (const MedOps* m = med_whiten_ops(a.n, a.mmax, fp32)) return m->whiten(a, fp32, st);
    if (use_large(a.n, fp32) || !generic_whiten_fits(a.n, a.mmax)) return launch_whiten_large(a, fp32, st);
    const WhitenLayout L = whiten_layout(a.n, a.mmax);
    const size_t smem = sizeof(double) * (size_t)L.total;
    int threads = 3 * a.n + 2;
    if (a.n + a.mmax > threads) threads = a.n + a.mmax;
    threads = ((threads + 31) / 32) * 32;
    if (threads > 256) return cudaErrorInvalidValue;
    const int64_t blocks = a.k < (1LL << 30) ? a.k : (1LL << 30);
    if (fp32) {
        cudaFuncSetAttribute(whiten_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        whiten_kernel<float><<<(unsigned)blocks, threads, smem, st>>>(a);
        ++t_launches;
    } else {
        cudaFuncSetAttribute(whiten_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        whiten_kernel<double><<<(unsigned)blocks, threads, smem, st>>>(a);
        ++t_launches;
    }
    return cudaGetLastError();
}

// Non-finite inputs.  NaN or Inf in F_i, H_{i-1} or G_i reaches the column norms cn2 / cd2 of
// state i through the whitening (a non-finite K_i or C_i is already caught by its Cholesky
// factorization); o_i and c_i enter only the right-hand side and are checked directly.
__global__ void check_finite_kernel(WhitenArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    const int64_t kn = a.k * n;
    for (int64_t e = t0; e < kn; e += stride)
        if (!isfinite(a.cn2[e]) || !isfinite(a.cd2[e])) flag_error(a.bad, ST_NONFINITE, e / n);
    if (a.c != nullptr)
        for (int64_t e = t0; e < (a.k - 1) * n; e += stride)
            if (!isfinite(a.c[e])) flag_error(a.bad, ST_NONFINITE, e / n);
    if (a.o != nullptr) {
        const int64_t tot = a.m_uniform >= 0 ? a.k * a.m_uniform : a.goff[a.k];
        for (int64_t e = t0; e < tot; e += stride) {
            if (isfinite(a.o[e])) continue;
            int64_t i;
            if (a.m_uniform >= 0) {
                i = e / a.m_uniform;
            } else {   // the step whose rows hold entry e: goff[i] <= e < goff[i + 1]
                int64_t lo = 0, hi = a.k;
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (a.goff[mid] <= e) lo = mid; else hi = mid;
                }
                i = lo;
            }
            flag_error(a.bad, ST_NONFINITE, i);
        }
    }
}

cudaError_t launch_check_finite(const WhitenArgs& a, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (a.k * a.n + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    const unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    check_finite_kernel<<<grid, 256, 0, st>>>(a);
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

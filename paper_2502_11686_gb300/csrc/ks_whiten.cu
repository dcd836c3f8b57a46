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

}  // namespace ks

// ks_level.cu -- one level of the odd-even block QR factorization (Section 3).
//
// At a level with nc alive block columns (j = 0..nc-1; original index c = (j+1) 2^l - 1), the
// even columns are eliminated and the odd ones survive.  One thread block handles tile t: the
// eliminated column j = 2t and its right neighbour s = 2t+1, plus -- when nc is odd and t is the
// last tile -- the last column e = nc-1, which has no right neighbour.  Tiles touch disjoint
// block rows, so the whole level is one launch (the parallelism argument of Section 3).
//
//   step 1 (Section 3, first QR):   [Chat_j ; -B_s] -> Rtilde_j, applied to [0 ; D_s] and the rhs
//                                   giving X_j (fill in column s), Dtilde_s and t_j, s_s;
//   step 2 (second QR, j >= 1):     [Rtilde_j ; D_j] -> R_j, applied to [0 ; -B_j], [X_j ; 0] and
//                                   the rhs: the top rows are block row j of R (R_j, -Btilde_j,
//                                   Y_j, y_j), the bottom rows [Z_j | Xtilde_j | z_j] are the
//                                   coupling row of the reduced problem between j-1 and s;
//                                   for j = 0 there is no step 2 and R_0 = Rtilde_0, Rr = X_0;
//   tail (nc odd): column e has no step 1; its step 2 is [Chat_e ; D_e] applied to [0 ; -B_e],
//                                   giving block row e of R and a block Z_e in column s only;
//   step 3 (invariant restoring):   [Chat_s ; Dtilde_s (; Z_e)] -> Chat'_s, the reduced problem's
//                                   diagonal block; discarded rhs rows go to the residual.
//
// Shared memory (TileLayout): TOP2 / BOT2 hold the step-2 working matrix
// [n factor | n left companion | n right companion | rhs] (top rows, bottom rows); step 1 writes
// its top rows straight into TOP2 (factor -> cols 0..n-1, companion -> cols 2n..3n-1, rhs -> col
// 3n) and its bottom companion rows into BOT3 (cols 0..n-1, rhs col n), where step 3 reads them;
// BF holds the bottom of step 1's factor columns.
#include "ks_generic.cuh"

namespace ks {

template <typename T, typename IO>
__global__ void __launch_bounds__(256) level_kernel(int n, int64_t nc, int level, int64_t k,
                                                    const T* __restrict__ in, T* __restrict__ out,
                                                    T* __restrict__ R, double* __restrict__ resid,
                                                    const double* __restrict__ cn2,
                                                    const double* __restrict__ cd2,
                                                    unsigned long long* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const IO io(n, nc, level, k, in, out, R);
    for (int64_t t = blockIdx.x; t < nc / 2; t += gridDim.x)
        level_cta_tile<T, IO>(io, n, nc, level, t, resid, cn2, cd2, bad, sm);
}

template <typename T>
__global__ void base_kernel(int n, int64_t k, int L, const T* __restrict__ in, T* __restrict__ R,
                            const double* __restrict__ cn2, const double* __restrict__ cd2,
                            unsigned long long* bad) {
    base_block<T>(n, k, L, in, R, cn2, cd2, bad);
}

template <template <typename> class IO>
static cudaError_t launch_level_io(int n, int64_t nc, int level, int64_t k, const void* in,
                                   void* out, void* R, double* resid, const double* cn2,
                                   const double* cd2, unsigned long long* bad, bool fp32,
                                   cudaStream_t st) {
    const int64_t nt = nc / 2;
    if (nt <= 0) return cudaSuccess;
    const TileLayout L = tile_layout(n);
    int threads = ((3 * n + 1 + 31) / 32) * 32;
    if (threads > 256) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)(nt < (1LL << 30) ? nt : (1LL << 30));
    if (fp32) {
        const size_t smem = sizeof(float) * (size_t)L.total;
        cudaFuncSetAttribute(level_kernel<float, IO<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        level_kernel<float, IO<float>><<<blocks, threads, smem, st>>>(
            n, nc, level, k, (const float*)in, (float*)out, (float*)R, resid, cn2, cd2, bad);
    } else {
        const size_t smem = sizeof(double) * (size_t)L.total;
        cudaFuncSetAttribute(level_kernel<double, IO<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        level_kernel<double, IO<double>><<<blocks, threads, smem, st>>>(
            n, nc, level, k, (const double*)in, (double*)out, (double*)R, resid, cn2, cd2, bad);
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_level(int n, int64_t nc, int level, int64_t k, const void* in, void* out,
                         void* R, double* resid, const double* cn2, const double* cd2,
                         unsigned long long* bad, bool fp32, cudaStream_t st) {
    if (use_large(n, fp32))   // works in place: each input record is read by one tile only
        return launch_level_large(n, nc, level, const_cast<void*>(in), out, R, resid, cn2, cd2, bad, fp32, st);
    return launch_level_io<AosIO>(n, nc, level, k, in, out, R, resid, cn2, cd2, bad, fp32, st);
}

cudaError_t launch_level_soa(int n, int64_t nc, int level, int64_t k, const void* in, void* out,
                             void* R, double* resid, const double* cn2, const double* cd2,
                             unsigned long long* bad, bool fp32, cudaStream_t st) {
    return launch_level_io<SoaIO>(n, nc, level, k, in, out, R, resid, cn2, cd2, bad, fp32, st);
}

cudaError_t launch_base(int n, int64_t k, int L, const void* in, void* R, const double* cn2,
                        const double* cd2, unsigned long long* bad, bool fp32, cudaStream_t st) {
    if (fp32)
        base_kernel<float><<<1, 128, 0, st>>>(n, k, L, (const float*)in, (float*)R, cn2, cd2, bad);
    else
        base_kernel<double><<<1, 128, 0, st>>>(n, k, L, (const double*)in, (double*)R, cn2, cd2, bad);
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

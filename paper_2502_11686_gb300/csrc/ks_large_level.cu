// ks_large_level.cu -- launcher of the large-state level kernels (kernels and device code in
// ks_large.cuh).
#include "ks_large.cuh"

namespace ks {
namespace large {

// FP32 tensor-core level kernel with two blocks per SM: the compact layout (QrSmemTc) and TMEM
// taken per trailing update, so one block's panel factorization on the CUDA cores overlaps the
// other block's tensor-core update.
__global__ void __launch_bounds__(NTH, 2) level_tc2_k(int n, int64_t nc, int level, float* in,
                                                      float* out, float* R, double* resid,
                                                      const double* cn2, const double* cd2,
                                                      unsigned long long* bad, int stall) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcState tcs;
    tc_setup(tcs, smem_raw + QrSmemTc::TC_BYTES, bad, stall, 1);
    for (int64_t t = blockIdx.x; t < nc / 2; t += gridDim.x)
        level_tile<float, QrSmemTc>(n, nc, level, t, in, out, R, resid, cn2, cd2, bad,
                                    reinterpret_cast<float*>(smem_raw), &tcs);
    tc_teardown(tcs);
}

}  // namespace large

cudaError_t launch_level_large(int n, int64_t nc, int level, void* in, void* out, void* R,
                               double* resid, const double* cn2, const double* cd2,
                               unsigned long long* bad, bool fp32, cudaStream_t st) {
    using namespace large;
    if (nc < 2) return cudaSuccess;
    if (n > PMAX) {
        const unsigned grid = grid_of(nc / 2, 1);
        if (fp32) {
            const size_t smem = BigSmem<float>::bytes(n);
            set_smem(level_k<float>, smem);
            level_k<float><<<grid, NTH, smem, st>>>(n, nc, level, (float*)in, (float*)out, (float*)R, resid, cn2, cd2, bad, -1, 0);
        } else {
            const size_t smem = BigSmem<double>::bytes(n);
            set_smem(level_k<double>, smem);
            level_k<double><<<grid, NTH, smem, st>>>(n, nc, level, (double*)in, (double*)out, (double*)R, resid, cn2, cd2, bad, -1, 0);
        }
        ++t_launches;
        return cudaGetLastError();
    }
    int tc_off = -1;
    const size_t smem = with_tc(qr_bytes(fp32), fp32, &tc_off);
    if (tc_off >= 0 && tc_blocks_per_sm() == 2) {
        const unsigned grid = grid_of(nc / 2, 2);
        set_smem(level_tc2_k, QrSmemTc::BYTES);
        cudaFuncSetAttribute(level_tc2_k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);   // room for two blocks per SM
        level_tc2_k<<<grid, NTH, QrSmemTc::BYTES, st>>>(n, nc, level, (float*)in, (float*)out, (float*)R,
                                                        resid, cn2, cd2, bad, tc_stall_test());
        ++t_launches;
        return cudaGetLastError();
    }
    const unsigned grid = grid_of(nc / 2, tc_off >= 0 ? 1 : 2);
    if (fp32) {
        set_smem(level_k<float>, smem);
        const int stall = tc_off >= 0 ? tc_stall_test() : 0;
        level_k<float><<<grid, NTH, smem, st>>>(n, nc, level, (float*)in, (float*)out, (float*)R, resid, cn2, cd2, bad, tc_off, stall);
    } else {
        set_smem(level_k<double>, smem);
        level_k<double><<<grid, NTH, smem, st>>>(n, nc, level, (double*)in, (double*)out, (double*)R, resid, cn2, cd2, bad, -1, 0);
    }
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

// ks_large_selinv.cu -- launchers of the large-state SelInv kernels (kernels and device code in
// ks_large.cuh).
#include "ks_large.cuh"

namespace ks {

namespace large {

// FP32 SelInv with the products on the tensor cores (selinv_row_tc): two blocks per SM, each
// holding 256 TMEM columns for its life.
// ri_scratch (state dimensions above PMAX): per-block slices of 2 n^2 floats for Rd^{-1} and M.
__global__ void __launch_bounds__(NTH, 2) selinv_tc_k(int n, int64_t k, int level, const float* R,
                                                      float* Sx, double* Sd, unsigned long long* bad,
                                                      float* ri_scratch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SelTc st;
    sel_tc_setup(st, smem_raw, bad);
    float* ri = ri_scratch ? ri_scratch + blockIdx.x * 2 * (int64_t)n * n : nullptr;
    const int64_t rows = (k >> level) - (k >> (level + 1));
    for (int64_t q = blockIdx.x; q < rows; q += gridDim.x)
        selinv_row_tc(n, k, level, q, R, Sx, Sd, bad, st, ri);
    sel_tc_teardown(st);
}

static void selinv_tc_attrs() {
    set_smem(selinv_tc_k, SelTcSmem::BYTES);
    cudaFuncSetAttribute(selinv_tc_k, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);   // room for two blocks per SM
}

}  // namespace large

cudaError_t launch_selinv_large(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                                unsigned long long* bad, bool fp32, cudaStream_t st) {
    using namespace large;
    const int64_t rows = (k >> level) - (k >> (level + 1));
    if (rows <= 0) return cudaSuccess;
    if (fp32 && n <= PMAX && tc_enabled()) {
        const unsigned grid = grid_of(rows, 2);
        selinv_tc_attrs();
        selinv_tc_k<<<grid, NTH, SelTcSmem::BYTES, st>>>(n, k, level, (const float*)R, (float*)Sx, Sd, bad,
                                                         nullptr);
        ++t_launches;
        return cudaGetLastError();
    }
    const size_t smem = SelSmem::bytes(n, fp32);
    const unsigned grid = grid_of(rows, fp32 ? 2 : 1);
    if (fp32) {
        set_smem(selinv_k<float>, smem);
        selinv_k<float><<<grid, NTH, smem, st>>>(n, k, level, (const float*)R, (float*)Sx, Sd, bad, nullptr);
    } else {
        set_smem(selinv_k<double>, smem);
        selinv_k<double><<<grid, NTH, smem, st>>>(n, k, level, (const double*)R, (double*)Sx, Sd, bad, nullptr);
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_selinv_huge(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                               void* ri_scratch, unsigned long long* bad, bool fp32, cudaStream_t st) {
    using namespace large;
    const int64_t rows = (k >> level) - (k >> (level + 1));
    if (rows <= 0) return cudaSuccess;
    if (ri_scratch == nullptr) return cudaErrorInvalidValue;
    const unsigned grid = huge_grid(rows);   // the scratch holds huge_grid(...) slices of 2 n x n
    if (fp32 && tc_enabled()) {
        selinv_tc_attrs();
        selinv_tc_k<<<grid, NTH, SelTcSmem::BYTES, st>>>(n, k, level, (const float*)R, (float*)Sx, Sd, bad,
                                                         (float*)ri_scratch);
        ++t_launches;
        return cudaGetLastError();
    }
    const size_t smem = (size_t)(GK * GM + GK * GN) * (fp32 ? sizeof(float) : sizeof(double));
    if (fp32) {
        set_smem(selinv_k<float>, smem);
        selinv_k<float><<<grid, NTH, smem, st>>>(n, k, level, (const float*)R, (float*)Sx, Sd, bad,
                                                 (float*)ri_scratch);
    } else {
        set_smem(selinv_k<double>, smem);
        selinv_k<double><<<grid, NTH, smem, st>>>(n, k, level, (const double*)R, (double*)Sx, Sd, bad,
                                                  (double*)ri_scratch);
    }
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

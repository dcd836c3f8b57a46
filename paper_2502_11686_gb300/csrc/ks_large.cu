// ks_large.cu -- launchers of the large-state whitening (kernels and device code in ks_large.cuh).
#include "ks_large.cuh"

namespace ks {

// Largest dynamic shared memory a large-state launch of this n requests (with the tensor-core
// region of the FP32 whitening and level kernels).
size_t large_smem_bytes(int n, bool fp32) {
    using namespace large;
    if (n > PMAX) {   // QR panel in shared memory; factors and Rd^{-1} in global scratch
        const size_t q = fp32 ? BigSmem<float>::bytes(n) : BigSmem<double>::bytes(n);
        const size_t sel = (size_t)(GK * GM + GK * GN) * (fp32 ? sizeof(float) : sizeof(double));
        return q > sel ? q : sel;
    }
    int off = -1;
    size_t m = with_tc(WhitenSmem::bytes(n, fp32), fp32, &off);
    const size_t q = with_tc(qr_bytes(fp32), fp32, &off);
    if (q > m) m = q;
    if (SelSmem::bytes(n, fp32) > m) m = SelSmem::bytes(n, fp32);
    return m;
}

size_t huge_whiten_scratch_bytes(int n) {
    const size_t tri = (size_t)n * (n + 1) / 2;
    return ((tri * sizeof(double) + tri * sizeof(float)) + 255) & ~(size_t)255;
}

unsigned huge_grid(int64_t units) { return large::grid_of(units, 1); }

cudaError_t launch_whiten_large(const WhitenArgs& a, bool fp32, cudaStream_t st) {
    using namespace large;
    if (a.n > PMAX) {   // one block per SM: its slice of a.cta_scratch holds the factors
        if (a.cta_scratch == nullptr) return cudaErrorInvalidValue;
        const unsigned grid = huge_grid(a.k);
        if (fp32) {
            const size_t smem = BigSmem<float>::bytes(a.n);
            set_smem(whiten_k<float>, smem);
            whiten_k<float><<<grid, NTH, smem, st>>>(a, -1);
        } else {
            const size_t smem = BigSmem<double>::bytes(a.n);
            set_smem(whiten_k<double>, smem);
            whiten_k<double><<<grid, NTH, smem, st>>>(a, -1);
        }
        ++t_launches;
        return cudaGetLastError();
    }
    int tc_off = -1;
    const size_t smem = with_tc(WhitenSmem::bytes(a.n, fp32), fp32, &tc_off);
    const unsigned grid = grid_of(a.k, tc_off >= 0 ? 1 : 2);
    if (fp32) {
        set_smem(whiten_k<float>, smem);
        whiten_k<float><<<grid, NTH, smem, st>>>(a, tc_off);
    } else {
        set_smem(whiten_k<double>, smem);
        whiten_k<double><<<grid, NTH, smem, st>>>(a, -1);
    }
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

// ks_large_batch.cu -- launcher of the batched large-state kernels (kernels and device code in
// ks_large.cuh).
#include "ks_large.cuh"

namespace ks {
namespace large {

// Batched FP32 SelInv with the products on the tensor cores (selinv_row_tc), two blocks per SM.
__global__ void __launch_bounds__(NTH, 2) batch_selinv_tc_k(const BatchWork* wk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchWork w = *wk;
    const int64_t total = w.off[w.np];
    SelTc st;
    sel_tc_setup(st, smem_raw, w.np > 0 ? w.desc[w.probs[0]].bad : nullptr);
    for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
        const int pi = batch_find(w.off, w.np, u);
        const ProbDesc& P = w.desc[w.probs[pi]];
        st.bad = P.bad;
        selinv_row_tc(P.n, P.k, work_level(w, P), u - w.off[pi], reinterpret_cast<const float*>(P.R),
                      reinterpret_cast<float*>(P.Sx), P.cov, P.bad, st);
    }
    sel_tc_teardown(st);
}

}  // namespace large

cudaError_t launch_batch_large(int op, int n, const BatchWork* wk, bool fp32, unsigned grid,
                               cudaStream_t st) {
    using namespace large;
    if (op == B_SELINV && fp32 && n <= PMAX && tc_enabled()) {
        const unsigned two = grid_of(1LL << 40, 2);   // two blocks per SM hold all of the TMEM
        if (grid > two) grid = two;
        set_smem(batch_selinv_tc_k, SelTcSmem::BYTES);
        cudaFuncSetAttribute(batch_selinv_tc_k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        batch_selinv_tc_k<<<grid, NTH, SelTcSmem::BYTES, st>>>(wk);
        ++t_launches;
        return cudaGetLastError();
    }
    size_t smem = 0;
    int tc_off = -1;
    if (op == B_WHITEN) smem = with_tc(WhitenSmem::bytes(n, fp32), fp32, &tc_off);
    else if (op == B_LEVEL) smem = with_tc(qr_bytes(fp32), fp32, &tc_off);
    else if (op == B_SELINV) smem = SelSmem::bytes(n, fp32);
    else return cudaErrorInvalidValue;
    if (tc_off >= 0) {   // one block per SM holds the whole TMEM
        const unsigned one = grid_of(1LL << 40, 1);
        if (grid > one) grid = one;
    }
#define KS_LARGE_BATCH(TT, OPV)                               \
    do {                                                      \
        set_smem(batch_k<TT, OPV>, smem);                     \
        batch_k<TT, OPV><<<grid, NTH, smem, st>>>(wk, tc_off); \
    } while (0)
    if (fp32) {
        if (op == B_WHITEN) KS_LARGE_BATCH(float, B_WHITEN);
        else if (op == B_LEVEL) KS_LARGE_BATCH(float, B_LEVEL);
        else KS_LARGE_BATCH(float, B_SELINV);
    } else {
        if (op == B_WHITEN) KS_LARGE_BATCH(double, B_WHITEN);
        else if (op == B_LEVEL) KS_LARGE_BATCH(double, B_LEVEL);
        else KS_LARGE_BATCH(double, B_SELINV);
    }
#undef KS_LARGE_BATCH
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace ks

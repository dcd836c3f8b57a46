// ks_med_n.cu -- launches of the register-column level and whitening kernels for one
// compile-time N (the build compiles this file once per N in {12, 16, 24, 32, 48, 64} with
// -DKS_MED_N=N).  Levels: FP32 for every N, FP64 up to N = 32, where a thread's two columns of
// N doubles still fit in registers.  Whitening (every m_i <= N): FP32 for every N, FP64 up to
// N = 48.
#include "ks_med.cuh"

#ifndef KS_MED_N
#error "compile with -DKS_MED_N=<12|16|24|32|48|64>"
#endif
#define KS_CAT2(a, b) a##b
#define KS_CAT(a, b) KS_CAT2(a, b)

namespace ks {
namespace med {
namespace {

constexpr int NN = KS_MED_N;
constexpr int THREADS = ((3 * NN + 1 + 31) / 32) * 32;
constexpr bool FP64_OK = NN <= 32;
constexpr int WTHREADS = ((3 * NN + 2 + 31) / 32) * 32;
constexpr bool WFP64_OK = NN <= 48;
// Blocks per SM the whitening is compiled for: a register cap of 128 (FP32) or 168 (FP64) per
// thread, which the live column (N values) fits without spilling; FP64 at N = 48 and FP32 at
// N = 64 need more.
template <typename T>
constexpr int wminb() {
    const int cap = sizeof(T) == 4 ? 128 : 168;
    const int b = ((sizeof(T) == 8 && NN >= 48) || NN >= 64) ? 1 : 65536 / (WTHREADS * cap);
    return b < 1 ? 1 : b;
}

// Blocks per SM the level kernel is compiled for: 2 for FP32 at N = 48 (168 registers, a small
// spill) so that ten warps share an SM instead of five; 1 otherwise.
template <typename T>
constexpr int lminb() { return (sizeof(T) == 4 && NN == 48) ? 2 : 1; }

template <typename T>
__global__ void __launch_bounds__(THREADS, lminb<T>()) level_med_k(int64_t nc, int level, int64_t k, const T* in,
                                                           T* out, T* R, double* resid, const double* cn2,
                                                           const double* cd2, unsigned long long* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AosIO<T> io(NN, nc, level, k, in, out, R);
    for (int64_t t = blockIdx.x; t < nc / 2; t += gridDim.x)
        level_med_tile<T, NN>(io, nc, level, t, resid, cn2, cd2, bad, reinterpret_cast<T*>(smem_raw));
}

template <typename T>
__global__ void __launch_bounds__(THREADS, lminb<T>()) batch_level_med_k(const BatchWork* wk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchWork w = *wk;
    const int64_t total = w.off[w.np];
    for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
        const int pi = batch_find(w.off, w.np, u);
        const ProbDesc& P = w.desc[w.probs[pi]];
        const int l = work_level(w, P);
        const int64_t nc = P.k >> l;
        const AosIO<T> io(NN, nc, l, P.k, reinterpret_cast<const T*>(P.lvl[l & 1]),
                          reinterpret_cast<T*>(P.lvl[(l + 1) & 1]), reinterpret_cast<T*>(P.R));
        level_med_tile<T, NN>(io, nc, l, u - w.off[pi], P.resid, P.cn2, P.cd2, P.bad,
                              reinterpret_cast<T*>(smem_raw));
    }
}

template <typename T>
__global__ void __launch_bounds__(WTHREADS, wminb<T>()) whiten_med_k(WhitenArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int64_t i = blockIdx.x; i < a.k; i += gridDim.x) whiten_med_step<T, NN>(a, i, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(WTHREADS, wminb<T>()) batch_whiten_med_k(const BatchWork* wk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchWork w = *wk;
    const int64_t total = w.off[w.np];
    for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
        const int pi = batch_find(w.off, w.np, u);
        const ProbDesc& P = w.desc[w.probs[pi]];
        whiten_med_step<T, NN>(whiten_args_of(P), u - w.off[pi], smem_raw);
    }
}

template <typename T>
int smem_bytes() { return MedSmem<T, NN>::TOTAL * (int)sizeof(T); }

template <typename T>
cudaError_t whiten_t(const WhitenArgs& a, const BatchWork* wk, unsigned grid, cudaStream_t st) {
    const int smem = MedWhitenSmem<T, NN>::BYTES;
    if (wk != nullptr) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(batch_whiten_med_k<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        batch_whiten_med_k<T><<<grid, WTHREADS, smem, st>>>(wk);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(whiten_med_k<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        const unsigned blocks = (unsigned)(a.k < (1LL << 30) ? a.k : (1LL << 30));
        whiten_med_k<T><<<blocks, WTHREADS, smem, st>>>(a);
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t whiten(const WhitenArgs& a, bool fp32, cudaStream_t st) {
    if (a.n != NN || a.mmax > NN) return cudaErrorInvalidValue;
    if (fp32) return whiten_t<float>(a, nullptr, 0, st);
    if constexpr (WFP64_OK) return whiten_t<double>(a, nullptr, 0, st);
    return cudaErrorInvalidValue;
}

cudaError_t batch_whiten(const BatchWork* wk, bool fp32, unsigned grid, cudaStream_t st) {
    const WhitenArgs none{};
    if (fp32) return whiten_t<float>(none, wk, grid, st);
    if constexpr (WFP64_OK) return whiten_t<double>(none, wk, grid, st);
    return cudaErrorInvalidValue;
}

cudaError_t level(int64_t nc, int lvl, int64_t k, const void* in, void* out, void* R, double* resid,
                  const double* cn2, const double* cd2, unsigned long long* bad, bool fp32,
                  cudaStream_t st) {
    const int64_t nt = nc >> 1;
    if (nt <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(nt < (1LL << 30) ? nt : (1LL << 30));
    if (fp32) {
        cudaFuncSetAttribute(level_med_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<float>());
        level_med_k<float><<<blocks, THREADS, smem_bytes<float>(), st>>>(
            nc, lvl, k, (const float*)in, (float*)out, (float*)R, resid, cn2, cd2, bad);
    } else {
        if constexpr (FP64_OK) {
            cudaFuncSetAttribute(level_med_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<double>());
            level_med_k<double><<<blocks, THREADS, smem_bytes<double>(), st>>>(
                nc, lvl, k, (const double*)in, (double*)out, (double*)R, resid, cn2, cd2, bad);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t batch_level(const BatchWork* wk, bool fp32, unsigned grid, cudaStream_t st) {
    if (fp32) {
        cudaFuncSetAttribute(batch_level_med_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<float>());
        batch_level_med_k<float><<<grid, THREADS, smem_bytes<float>(), st>>>(wk);
    } else {
        if constexpr (FP64_OK) {
            cudaFuncSetAttribute(batch_level_med_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<double>());
            batch_level_med_k<double><<<grid, THREADS, smem_bytes<double>(), st>>>(wk);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace
}  // namespace med

extern const MedOps KS_CAT(med_ops_, KS_MED_N);
const MedOps KS_CAT(med_ops_, KS_MED_N) = {KS_MED_N,          med::FP64_OK,      med::level,
                                           med::batch_level, med::WFP64_OK,     med::whiten,
                                           med::batch_whiten};

}  // namespace ks

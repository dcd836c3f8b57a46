// ks_small_n.cu -- kernels of the small-state path for one compile-time N (the build compiles
// this file once per N = 1..8 with -DKS_SMALL_N=N).  Each kernel maps one thread to one unit:
// a step (whitening), a column pair / tail triple (level), a block row (back substitution,
// SelInv), an alive column (R^T w = g).
#include <cstdlib>

#include "ks_small.cuh"

#ifndef KS_SMALL_N
#error "compile with -DKS_SMALL_N=<1..8>"
#endif
#define KS_CAT2(a, b) a##b
#define KS_CAT(a, b) KS_CAT2(a, b)

namespace ks {
namespace small {
namespace {

constexpr int NN = KS_SMALL_N;
constexpr int BLK = 64;

template <typename T>
__global__ void __launch_bounds__(BLK) whiten_k(WhitenArgs a) {
    const int64_t i = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (i < a.k) whiten_step<T, NN>(a, i, reinterpret_cast<T*>(a.level0));
}

template <typename T>
__global__ void __launch_bounds__(BLK) level_k(int64_t nc, int level, int64_t k, const T* in, T* out,
                                               T* R, double* resid, const double* cn2,
                                               const double* cd2, unsigned long long* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stash<T> st{reinterpret_cast<T*>(smem_raw), BLK, (int)threadIdx.x};
    const int64_t t = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (t < (nc >> 1)) level_tile<T, NN>(nc, level, k, t, in, out, R, resid, cn2, cd2, bad, st);
}

template <typename T>
__global__ void base_k(int64_t k, int L, const T* in, T* R, const double* cn2, const double* cd2,
                       unsigned long long* bad) {
    using D = Dims<NN>;
    if (threadIdx.x != 0) return;
    const LevelView<const T, NN> I(in, 1);
    const RowView<T> RV(R, k, L, D::RS);
    const int64_t c = (1LL << L) - 1;
    T Tm[NN][NN];
    load_upper<T, NN>(I, 0, Tm);
    check_diag<T, NN>(Tm, cn2, cd2, c, bad);
    for (int r = 0; r < NN; ++r) {
        for (int cc = r; cc < NN; ++cc) *RV.at(0, D::ORD + tri(NN, r, cc)) = Tm[r][cc];
        for (int cc = 0; cc < NN; ++cc) {
            *RV.at(0, D::ORL + r * NN + cc) = T(0);
            *RV.at(0, D::ORR + r * NN + cc) = T(0);
        }
        *RV.at(0, D::OY + r) = *I.at(0, D::ORC + r);
    }
}

template <typename T>
__global__ void __launch_bounds__(BLK) backsub_k(int64_t k, int level, const T* R, const double* w,
                                                 double* u) {
    const int64_t q = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (q < (k >> level) - (k >> (level + 1))) backsub_row<T, NN>(k, level, q, R, w, u);
}

template <typename T>
__global__ void __launch_bounds__(BLK) selinv_k(int64_t k, int level, const T* R, T* Sx, double* Sd,
                                                unsigned long long* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stash<T> st{reinterpret_cast<T*>(smem_raw), BLK, (int)threadIdx.x};
    const int64_t q = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (q < (k >> level) - (k >> (level + 1))) selinv_row<T, NN>(k, level, q, R, Sx, Sd, bad, st);
}

template <typename T>
__global__ void __launch_bounds__(BLK) cross_k(int64_t k, const T* Sx, double* cross) {
    using D = Dims<NN>;
    const int64_t i = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (i + 1 >= k) return;
    const RowView<const T> SV(Sx, k, 0, D::SS);
    if ((i & 1) == 0) {  // i eliminated at level 0 with right neighbour i+1: Sr_i
        const int64_t q = i >> 1;
        for (int e = 0; e < NN * NN; ++e) cross[i * NN * NN + e] = (double)*SV.at(q, NN * NN + e);
    } else {             // i+1 eliminated at level 0 with left neighbour i: Sl_{i+1}^T
        const int64_t q = (i + 1) >> 1;
        for (int r = 0; r < NN; ++r)
            for (int c = 0; c < NN; ++c)
                cross[i * NN * NN + r * NN + c] = (double)*SV.at(q, c * NN + r);
    }
}

__global__ void __launch_bounds__(BLK) refine_q_k(RefineArgs a, float* q) {
    const int64_t i = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (i + 1 < a.k) refine_q_step<NN>(a, i, q);
}

__global__ void __launch_bounds__(BLK) refine_g_k(RefineArgs a, const float* q, float* g) {
    const int64_t c = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (c < a.k) refine_g_col<NN>(a, c, q, g);
}

__global__ void __launch_bounds__(BLK) rt_solve_k(int64_t k, int level, const float* R, float* g,
                                                  float* w) {
    const int64_t j = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (j < (k >> level)) rt_solve_col<float, float, NN>(k, level, j, R, g, w);
}

__global__ void __launch_bounds__(BLK) backsub_f_k(int64_t k, int level, const float* R,
                                                   const float* w, float* d) {
    const int64_t q = blockIdx.x * (int64_t)BLK + threadIdx.x;
    if (q < (k >> level) - (k >> (level + 1))) backsub_row_f<NN>(k, level, q, R, w, d);
}

__global__ void __launch_bounds__(256) add_k(double* u, const float* d, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256)
        u[i] += (double)d[i];
}

// Below this many units per launch the level / SelInv launches use one thread block per unit
// (column-owner kernels, all lanes of a warp share a unit) instead of one thread per unit: a
// lone lane pays the full cost of every warp instruction, which dominates when a level has too
// few units to fill the GPU.  KS_TAIL_UNITS overrides the default.
int64_t tail_units(bool fp32) {
    const char* v = getenv("KS_TAIL_UNITS");
    if (v && *v) return atoll(v);
    return fp32 ? 1024 : 2048;
}

// ---- batched form: one launch covers one operation for every problem of a class ----------
template <typename T>
__device__ void base_one(int64_t k, int L, const T* in, T* R, const double* cn2,
                         const double* cd2, unsigned long long* bad) {
    using D = Dims<NN>;
    const LevelView<const T, NN> I(in, 1);
    const RowView<T> RV(R, k, L, D::RS);
    const int64_t c = (1LL << L) - 1;
    T Tm[NN][NN];
    load_upper<T, NN>(I, 0, Tm);
    check_diag<T, NN>(Tm, cn2, cd2, c, bad);
    for (int r = 0; r < NN; ++r) {
        for (int cc = r; cc < NN; ++cc) *RV.at(0, D::ORD + tri(NN, r, cc)) = Tm[r][cc];
        for (int cc = 0; cc < NN; ++cc) {
            *RV.at(0, D::ORL + r * NN + cc) = T(0);
            *RV.at(0, D::ORR + r * NN + cc) = T(0);
        }
        *RV.at(0, D::OY + r) = *I.at(0, D::ORC + r);
    }
}

template <typename T, int OP>
__global__ void __launch_bounds__(BLK) batch_k(const BatchWork* wk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stash<T> st{reinterpret_cast<T*>(smem_raw), BLK, (int)threadIdx.x};
    const BatchWork w = *wk;
    const int64_t total = w.off[w.np];
    for (int64_t u = blockIdx.x * (int64_t)BLK + threadIdx.x; u < total;
         u += (int64_t)gridDim.x * BLK) {
        const int pi = batch_find(w.off, w.np, u);
        const ProbDesc& P = w.desc[w.probs[pi]];
        const int64_t x = u - w.off[pi];
        const int l = work_level(w, P);
        if constexpr (OP == B_WHITEN) {
            whiten_step<T, NN>(whiten_args_of(P), x, reinterpret_cast<T*>(P.lvl[0]));
        } else if constexpr (OP == B_LEVEL) {
            level_tile<T, NN>(P.k >> l, l, P.k, x, reinterpret_cast<const T*>(P.lvl[l & 1]),
                              reinterpret_cast<T*>(P.lvl[(l + 1) & 1]), reinterpret_cast<T*>(P.R),
                              P.resid, P.cn2, P.cd2, P.bad, st);
        } else if constexpr (OP == B_BASE) {
            base_one<T>(P.k, P.L, reinterpret_cast<const T*>(P.lvl[P.L & 1]),
                        reinterpret_cast<T*>(P.R), P.cn2, P.cd2, P.bad);
        } else if constexpr (OP == B_BACKSUB) {
            backsub_row<T, NN>(P.k, l, x, reinterpret_cast<const T*>(P.R), nullptr, P.u);
        } else if constexpr (OP == B_SELINV) {
            selinv_row<T, NN>(P.k, l, x, reinterpret_cast<const T*>(P.R), reinterpret_cast<T*>(P.Sx),
                              P.cov, P.bad, st);
        } else if constexpr (OP == B_REFINE_Q) {
            refine_q_step<NN>(refine_args_of(P), x, reinterpret_cast<float*>(P.q));
        } else if constexpr (OP == B_REFINE_G) {
            refine_g_col<NN>(refine_args_of(P), x, reinterpret_cast<const float*>(P.q),
                             reinterpret_cast<float*>(P.g));
        } else if constexpr (OP == B_RT_SOLVE) {
            rt_solve_col<float, float, NN>(P.k, l, x, reinterpret_cast<const float*>(P.R),
                                           reinterpret_cast<float*>(P.g), reinterpret_cast<float*>(P.w));
        } else if constexpr (OP == B_BACKSUB_W) {
            backsub_row_f<NN>(P.k, l, x, reinterpret_cast<const float*>(P.R),
                              reinterpret_cast<const float*>(P.w), reinterpret_cast<float*>(P.d));
        } else if constexpr (OP == B_ADD) {
            P.u[x] += (double)reinterpret_cast<const float*>(P.d)[x];
        }
    }
}

template <typename T, int OP>
cudaError_t batch_launch(const BatchWork* wk, unsigned grid, int smem, cudaStream_t st) {
    if (smem > 0) cudaFuncSetAttribute(batch_k<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    batch_k<T, OP><<<grid, BLK, smem, st>>>(wk);
    ++t_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_t(int op, const BatchWork* wk, unsigned grid, cudaStream_t st) {
    const int lvl_smem = TileSlots<NN>::COUNT * BLK * (int)sizeof(T);
    const int sel_smem = SelinvSlots<NN>::COUNT * BLK * (int)sizeof(T);
    switch (op) {
        case B_WHITEN: return batch_launch<T, B_WHITEN>(wk, grid, 0, st);
        case B_LEVEL: return batch_launch<T, B_LEVEL>(wk, grid, lvl_smem, st);
        case B_BASE: return batch_launch<T, B_BASE>(wk, grid, 0, st);
        case B_BACKSUB: return batch_launch<T, B_BACKSUB>(wk, grid, 0, st);
        case B_SELINV: return batch_launch<T, B_SELINV>(wk, grid, sel_smem, st);
        case B_REFINE_Q: return batch_launch<T, B_REFINE_Q>(wk, grid, 0, st);
        case B_REFINE_G: return batch_launch<T, B_REFINE_G>(wk, grid, 0, st);
        case B_RT_SOLVE: return batch_launch<T, B_RT_SOLVE>(wk, grid, 0, st);
        case B_BACKSUB_W: return batch_launch<T, B_BACKSUB_W>(wk, grid, 0, st);
        case B_ADD: return batch_launch<T, B_ADD>(wk, grid, 0, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch(int op, const BatchWork* wk, bool fp32, unsigned grid, cudaStream_t st) {
    if (fp32) return batch_t<float>(op, wk, grid, st);
    // FP64 mode has no refinement operations.
    if (op >= B_REFINE_Q) return cudaErrorInvalidValue;
    return batch_t<double>(op, wk, grid, st);
}

unsigned grid(int64_t work) {
    int64_t b = (work + BLK - 1) / BLK;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t whiten(const WhitenArgs& a, bool fp32, cudaStream_t st) {
    if (fp32)
        whiten_k<float><<<grid(a.k), BLK, 0, st>>>(a);
    else
        whiten_k<double><<<grid(a.k), BLK, 0, st>>>(a);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t level(int64_t nc, int lvl, int64_t k, const void* in, void* out, void* R, double* resid,
                  const double* cn2, const double* cd2, unsigned long long* bad, bool fp32,
                  cudaStream_t st) {
    const int64_t nt = nc >> 1;
    if (nt <= 0) return cudaSuccess;
    if (nt < tail_units(fp32))
        return launch_level_soa(NN, nc, lvl, k, in, out, R, resid, cn2, cd2, bad, fp32, st);
    const int stash = TileSlots<NN>::COUNT;
    if (fp32) {
        const int smem = stash * BLK * (int)sizeof(float);
        cudaFuncSetAttribute(level_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        level_k<float><<<grid(nt), BLK, smem, st>>>(nc, lvl, k, (const float*)in, (float*)out,
                                                   (float*)R, resid, cn2, cd2, bad);
    } else {
        const int smem = stash * BLK * (int)sizeof(double);
        cudaFuncSetAttribute(level_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        level_k<double><<<grid(nt), BLK, smem, st>>>(nc, lvl, k, (const double*)in, (double*)out,
                                                    (double*)R, resid, cn2, cd2, bad);
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t base(int64_t k, int L, const void* in, void* R, const double* cn2, const double* cd2,
                 unsigned long long* bad, bool fp32, cudaStream_t st) {
    if (fp32)
        base_k<float><<<1, 32, 0, st>>>(k, L, (const float*)in, (float*)R, cn2, cd2, bad);
    else
        base_k<double><<<1, 32, 0, st>>>(k, L, (const double*)in, (double*)R, cn2, cd2, bad);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t backsub(int64_t k, int lvl, const void* R, const double* w, double* u, bool fp32,
                    cudaStream_t st) {
    const int64_t rows = (k >> lvl) - (k >> (lvl + 1));
    if (fp32)
        backsub_k<float><<<grid(rows), BLK, 0, st>>>(k, lvl, (const float*)R, w, u);
    else
        backsub_k<double><<<grid(rows), BLK, 0, st>>>(k, lvl, (const double*)R, w, u);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t selinv(int64_t k, int lvl, const void* R, void* Sx, double* Sd, unsigned long long* bad,
                   bool fp32, cudaStream_t st) {
    const int64_t rows = (k >> lvl) - (k >> (lvl + 1));
    if (rows < tail_units(fp32)) return launch_selinv_soa(NN, k, lvl, R, Sx, Sd, bad, fp32, st);
    const int stash = SelinvSlots<NN>::COUNT;
    if (fp32) {
        const int smem = stash * BLK * (int)sizeof(float);
        cudaFuncSetAttribute(selinv_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        selinv_k<float><<<grid(rows), BLK, smem, st>>>(k, lvl, (const float*)R, (float*)Sx, Sd, bad);
    } else {
        const int smem = stash * BLK * (int)sizeof(double);
        cudaFuncSetAttribute(selinv_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        selinv_k<double><<<grid(rows), BLK, smem, st>>>(k, lvl, (const double*)R, (double*)Sx, Sd, bad);
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t cross(int64_t k, const void* Sx, double* out, bool fp32, cudaStream_t st) {
    if (k < 2) return cudaSuccess;
    if (fp32)
        cross_k<float><<<grid(k - 1), BLK, 0, st>>>(k, (const float*)Sx, out);
    else
        cross_k<double><<<grid(k - 1), BLK, 0, st>>>(k, (const double*)Sx, out);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t refine(const RefineArgs& a, float* q, float* g, float* w, float* d, const void* R,
                   int L, cudaStream_t st) {
    const int64_t k = a.k;
    const float* Rf = static_cast<const float*>(R);
    if (k > 1) {
        refine_q_k<<<grid(k - 1), BLK, 0, st>>>(a, q);
        ++t_launches;
    }
    refine_g_k<<<grid(k), BLK, 0, st>>>(a, q, g);
    ++t_launches;
    for (int l = 0; l <= L; ++l) {
        rt_solve_k<<<grid(k >> l), BLK, 0, st>>>(k, l, Rf, g, w);
        ++t_launches;
    }
    for (int l = L; l >= 0; --l) {
        backsub_f_k<<<grid((k >> l) - (k >> (l + 1))), BLK, 0, st>>>(k, l, Rf, w, d);
        ++t_launches;
    }
    const int64_t cnt = k * NN;
    int64_t b = (cnt + 255) / 256;
    add_k<<<(unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), 256, 0, st>>>(const_cast<double*>(a.u), d, cnt);
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace
}  // namespace small

extern const SmallOps KS_CAT(small_ops_, KS_SMALL_N);
const SmallOps KS_CAT(small_ops_, KS_SMALL_N) = {
    KS_SMALL_N, small::whiten, small::level, small::base, small::backsub,
    small::selinv, small::cross, small::refine, small::batch};

}  // namespace ks

// ks_solve.cu -- everything that runs on the finished R factor.
//
//  * back substitution through the recursion (Section 3.1): levels from the top down; at level l
//    every column c with ctz(c+1) = l solves Rd_c u_c = y_c - Rl_c u_{c-2^l} - Rr_c u_{c+2^l};
//  * odd-even block SelInv (Section 4, Algorithm 2), levels from the top down: with
//    T = Rd_c^{-1} [Rl_c | Rr_c] and I = {c-2^l, c+2^l},
//        S_{c,I} = -T S_{I,I},   S_cc = Rd_c^{-1} Rd_c^{-T} - S_{c,I} T^T.
//    S_{I,I} needs the cross block of the two neighbours a < b; they are adjacent at level l+1,
//    so the one of them eliminated there holds it (S_ab = Sr_a if ctz(a+1) = l+1, else Sl_b^T);
//  * the refinement of KS_FP32_REFINE (not in the paper): g = (UA)^T U (b - A u) in FP64, then
//    the corrected semi-normal equations R^T R d = g with the FP32 R: R^T w = g level by level
//    from the bottom (column c pulls the blocks of the rows eliminated below it that touch it),
//    then R d = w by back substitution, u += d.
#include <algorithm>

#include "ks_generic.cuh"
#include "ks_warp.cuh"

namespace ks {

// R and SelInv-store access of the column-owner SelInv kernel: AoS rows by original index, or
// the small-state path's per-level element-major rows.  part 0/1/2 = Rd/Rl/Rr; S part 0/1 = Sl/Sr.
template <typename T>
struct SelAos {
    int n;
    int64_t k;
    __device__ SelAos(int n_, int64_t k_) : n(n_), k(k_) {}
    __device__ T R(const T* Rs, int, int64_t, int64_t c, int part, int r, int cc) const {
        return Rs[c * rstore_rs(n) + part * n * n + r * n + cc];
    }
    __device__ T S(const T* Sx, int, int64_t, int64_t c, int part, int r, int cc) const {
        return Sx[c * 2 * n * n + part * n * n + r * n + cc];
    }
    __device__ void setS(T* Sx, int, int64_t, int64_t c, int part, int r, int cc, T v) const {
        Sx[c * 2 * n * n + part * n * n + r * n + cc] = v;
    }
};

template <typename T>
struct SelSoa {
    int n, nt;
    int64_t k;
    __device__ SelSoa(int n_, int64_t k_) : n(n_), nt(n_ * (n_ + 1) / 2), k(k_) {}
    __device__ int64_t rows(int l) const { return (k >> l) - (k >> (l + 1)); }
    __device__ T R(const T* Rs, int l, int64_t q, int64_t, int part, int r, int cc) const {
        const int64_t RS = nt + 2 * n * n + n;
        const int64_t base = (k - (k >> l)) * RS;
        if (part == 0) return cc >= r ? Rs[base + (int64_t)(r * n - r * (r - 1) / 2 + cc - r) * rows(l) + q] : T(0);
        return Rs[base + (int64_t)(nt + (part - 1) * n * n + r * n + cc) * rows(l) + q];
    }
    __device__ T S(const T* Sx, int l, int64_t q, int64_t, int part, int r, int cc) const {
        return Sx[(k - (k >> l)) * 2 * n * n + (int64_t)(part * n * n + r * n + cc) * rows(l) + q];
    }
    __device__ void setS(T* Sx, int l, int64_t q, int64_t, int part, int r, int cc, T v) const {
        Sx[(k - (k >> l)) * 2 * n * n + (int64_t)(part * n * n + r * n + cc) * rows(l) + q] = v;
    }
};

// Row q of level `level` (Algorithm 2 body), column-owner scheme: every thread of the block
// must call it.
template <typename T, typename IO>
__device__ void selinv_cta_row(int n, int64_t k, int level, int64_t q, const T* __restrict__ R,
                               T* __restrict__ Sx, double* __restrict__ Sd,
                               unsigned long long* bad, T* sm) {
    const SelinvLayout L = selinv_layout(n);
    T* RD = sm + L.rd;
    T* TT = sm + L.tt;
    T* RI = sm + L.ri;
    T* SII = sm + L.sii;
    T* SL = sm + L.sl;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nn = n * n;
    const int64_t c = ((2 * q + 1) << level) - 1;
    if (c >= k) return;
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    const bool ha = a >= 0, hb = b < k;
    const IO io(n, k);
    // The cross block S_ab: a and b are adjacent one level up, where one of them is eliminated.
    int sab_src = 0;  // 0 none, 1 Sr_a = S_{a,b}, 2 Sl_b = S_{b,a}
    if (ha && hb) sab_src = (ctz64(a + 1) == level + 1) ? 1 : 2;
    const int64_t qa = (a + 1) >> (level + 2), qb = (b + 1) >> (level + 2);
    for (int e = tid; e < nn; e += nth) {
        const int r = e / n, cc = e - r * n;
        RD[r * L.ldr + cc] = io.R(R, level, q, c, 0, r, cc);
        TT[r * L.ldt + cc] = ha ? io.R(R, level, q, c, 1, r, cc) : T(0);
        TT[r * L.ldt + n + cc] = hb ? io.R(R, level, q, c, 2, r, cc) : T(0);
        RI[r * L.ldr + cc] = (r == cc) ? T(1) : T(0);
        SII[r * L.lds + cc] = ha ? (T)Sd[a * nn + e] : T(0);
        SII[(n + r) * L.lds + n + cc] = hb ? (T)Sd[b * nn + e] : T(0);
        T x = T(0);
        if (sab_src == 1) x = io.S(Sx, level + 1, qa, a, 1, r, cc);
        else if (sab_src == 2) x = io.S(Sx, level + 1, qb, b, 0, cc, r);
        SII[r * L.lds + n + cc] = x;          // S_ab
        SII[(n + cc) * L.lds + r] = x;        // S_ba = S_ab^T
    }
    __syncthreads();
    // X <- Rd^{-1} X for the 3n columns of [TT | RI] (one thread per column).
    for (int col = tid; col < 3 * n; col += nth) {
        T* X = col < 2 * n ? TT + col : RI + (col - 2 * n);
        const int ldx = col < 2 * n ? L.ldt : L.ldr;
        for (int i = n - 1; i >= 0; --i) {
            T s = X[i * ldx];
            for (int p = i + 1; p < n; ++p) s = fma(-RD[i * L.ldr + p], X[p * ldx], s);
            X[i * ldx] = s / RD[i * L.ldr + i];
        }
    }
    __syncthreads();
    // [Sl | Sr] = -T S_II
    for (int e = tid; e < 2 * nn; e += nth) {
        const int r = e / (2 * n), cc = e - r * 2 * n;
        T s = T(0);
        for (int p = 0; p < 2 * n; ++p) s = fma(TT[r * L.ldt + p], SII[p * L.lds + cc], s);
        SL[r * L.ldt + cc] = -s;
    }
    __syncthreads();
    // S_cc = Rd^{-1} Rd^{-T} - [Sl | Sr] T^T   (into RD, no longer needed)
    for (int e = tid; e < nn; e += nth) {
        const int r = e / n, cc = e - r * n;
        T s = T(0);
        for (int p = 0; p < n; ++p) s = fma(RI[r * L.ldr + p], RI[cc * L.ldr + p], s);
        for (int p = 0; p < 2 * n; ++p) s = fma(-SL[r * L.ldt + p], TT[cc * L.ldt + p], s);
        RD[r * L.ldr + cc] = s;
    }
    __syncthreads();
    for (int e = tid; e < nn; e += nth) {
        const int r = e / n, cc = e - r * n;
        const T v = T(0.5) * (RD[r * L.ldr + cc] + RD[cc * L.ldr + r]);
        Sd[c * nn + e] = (double)v;
        io.setS(Sx, level, q, c, 0, r, cc, SL[r * L.ldt + cc]);
        io.setS(Sx, level, q, c, 1, r, cc, SL[r * L.ldt + n + cc]);
        if (r == cc && !(v > T(0))) flag_error(bad, ST_SINGULAR, c);
    }
    __syncthreads();
}

template <typename T, typename IO>
__global__ void __launch_bounds__(128) selinv_kernel(int n, int64_t k, int level,
                                                     const T* __restrict__ R, T* __restrict__ Sx,
                                                     double* __restrict__ Sd,
                                                     unsigned long long* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    selinv_cta_row<T, IO>(n, k, level, blockIdx.x, R, Sx, Sd, bad, reinterpret_cast<T*>(smem_raw));
}

template <typename T>
__global__ void cross_kernel(int n, int64_t k, const T* __restrict__ Sx, double* __restrict__ cross) {
    const int nn = n * n;
    const int64_t total = (k - 1) * nn;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nn;
        const int rc = (int)(e - i * nn), r = rc / n, cc = rc - r * n;
        double v;
        if ((i & 1) == 0)
            v = (double)Sx[i * 2 * nn + nn + rc];              // Sr_i = S_{i,i+1}
        else
            v = (double)Sx[(i + 1) * 2 * nn + cc * n + r];     // Sl_{i+1}^T
        cross[e] = v;
    }
}

__global__ void sum_kernel(const double* __restrict__ x, int64_t count, double* out) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

static unsigned grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1LL << 30)) b = 1LL << 30;
    return (unsigned)b;
}

template <template <typename> class IO>
static cudaError_t launch_selinv_io(int n, int64_t k, int level, const void* R, void* Sx,
                                    double* Sd, unsigned long long* bad, bool fp32,
                                    cudaStream_t st) {
    const int64_t cols = ((k >> level) + 1) / 2;
    const SelinvLayout L = selinv_layout(n);
    const int threads = 128;
    const unsigned blocks = (unsigned)cols;
    if (fp32) {
        const size_t smem = sizeof(float) * (size_t)L.total;
        cudaFuncSetAttribute(selinv_kernel<float, IO<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        selinv_kernel<float, IO<float>><<<blocks, threads, smem, st>>>(n, k, level, (const float*)R, (float*)Sx, Sd, bad);
    } else {
        const size_t smem = sizeof(double) * (size_t)L.total;
        cudaFuncSetAttribute(selinv_kernel<double, IO<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        selinv_kernel<double, IO<double>><<<blocks, threads, smem, st>>>(n, k, level, (const double*)R, (double*)Sx, Sd, bad);
    }
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_selinv(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                          unsigned long long* bad, bool fp32, cudaStream_t st) {
    if (use_large(n, fp32)) return launch_selinv_large(n, k, level, R, Sx, Sd, bad, fp32, st);
    return launch_selinv_io<SelAos>(n, k, level, R, Sx, Sd, bad, fp32, st);
}

cudaError_t launch_selinv_soa(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                              unsigned long long* bad, bool fp32, cudaStream_t st) {
    return launch_selinv_io<SelSoa>(n, k, level, R, Sx, Sd, bad, fp32, st);
}

cudaError_t launch_cross(int n, int64_t k, const void* Sx, double* cross, bool fp32,
                         cudaStream_t st) {
    if (k < 2) return cudaSuccess;
    const int64_t total = (k - 1) * (int64_t)n * n;
    if (fp32)
        cross_kernel<float><<<grid_for(total, 256), 256, 0, st>>>(n, k, (const float*)Sx, cross);
    else
        cross_kernel<double><<<grid_for(total, 256), 256, 0, st>>>(n, k, (const double*)Sx, cross);
    ++t_launches;
    return cudaGetLastError();
}

thread_local uint64_t t_launches = 0;

cudaError_t launch_sum(const double* x, int64_t count, double* out, cudaStream_t st) {
    sum_kernel<<<1, 1024, 0, st>>>(x, count, out);
    ++t_launches;
    return cudaGetLastError();
}

// ---- warp-per-unit kernels of the column-owner path -----------------------------------------
// One warp per block row / column / step; lane l owns rows l, l+32, ... (ks_warp.cuh).  Triangular
// substitutions proceed one unknown at a time: its owner lane divides and broadcasts it with a
// shuffle, and every lane updates its own rows.  In FP32 + refinement mode the vectors are FP32
// except the residuals of the refinement, which are formed in FP64.

template <int NR, typename TR, typename TV, typename TO>
__global__ void __launch_bounds__(128) backsub_warp_kernel(int n, int64_t k, int level, const TR* R,
                                                           const TV* w, TO* u) {
    const int64_t q = blockIdx.x * 4LL + (threadIdx.x >> 5);
    if (q < (k >> level) - (k >> (level + 1))) backsub_warp<NR, TR, TV, TO>(n, k, level, q, R, w, u);
}

template <int NR, typename TR, typename TV>
__global__ void __launch_bounds__(128) rt_solve_warp_kernel(int n, int64_t k, int level, const TR* R,
                                                            TV* g, TV* w) {
    rt_solve_warp<NR, TR, TV>(n, k, level, blockIdx.x * 4LL + (threadIdx.x >> 5), R, g, w);
}

template <int NR, typename TV>
__global__ void __launch_bounds__(128) refine_qg_warp_kernel(RefineArgs a, int which, TV* q, TV* g) {
    const int64_t x = blockIdx.x * 4LL + (threadIdx.x >> 5);
    if (which == 0) refine_q_warp<NR, TV>(a, x, q);
    else refine_g_warp<NR, TV>(a, x, q, g);
}

template <typename TV>
__global__ void add_kernel(double* __restrict__ u, const TV* __restrict__ d, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        u[i] += (double)d[i];
}

static unsigned warps_grid(int64_t units) {
    int64_t b = (units + 3) / 4;
    return (unsigned)(b < 1 ? 1 : (b > (1LL << 30) ? (1LL << 30) : b));
}

template <int NR>
static cudaError_t backsub_warp_nr(int n, int64_t k, int level, const void* R, bool fp32, double* u,
                                   cudaStream_t st) {
    const int64_t rows = (k >> level) - (k >> (level + 1));
    if (fp32)  // FP32 first solve; the refinement corrects it
        backsub_warp_kernel<NR, float, float, double><<<warps_grid(rows), 128, 0, st>>>(
            n, k, level, (const float*)R, (const float*)nullptr, u);
    else
        backsub_warp_kernel<NR, double, double, double><<<warps_grid(rows), 128, 0, st>>>(
            n, k, level, (const double*)R, (const double*)nullptr, u);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_backsub_warp(int n, int64_t k, int level, const void* R, bool fp32,
                                double* u, cudaStream_t st) {
    return n <= 64 ? backsub_warp_nr<2>(n, k, level, R, fp32, u, st)
           : n <= 128 ? backsub_warp_nr<4>(n, k, level, R, fp32, u, st)
                      : backsub_warp_nr<16>(n, k, level, R, fp32, u, st);
}

template <int NR>
static cudaError_t refine_warp_nr(const RefineArgs& a, float* q, float* g, float* w, float* d,
                                  const void* R, int L, cudaStream_t st) {
    const int64_t k = a.k;
    const float* Rf = static_cast<const float*>(R);
    if (k > 1) {
        refine_qg_warp_kernel<NR, float><<<warps_grid(k - 1), 128, 0, st>>>(a, 0, q, g);
        ++t_launches;
    }
    refine_qg_warp_kernel<NR, float><<<warps_grid(k), 128, 0, st>>>(a, 1, q, g);
    ++t_launches;
    for (int l = 0; l <= L; ++l) {
        rt_solve_warp_kernel<NR, float, float><<<warps_grid(k >> l), 128, 0, st>>>(a.n, k, l, Rf, g, w);
        ++t_launches;
    }
    for (int l = L; l >= 0; --l) {
        backsub_warp_kernel<NR, float, float, float><<<warps_grid((k >> l) - (k >> (l + 1))), 128, 0, st>>>(
            a.n, k, l, Rf, w, d);
        ++t_launches;
    }
    const int64_t cnt = k * a.n;
    int64_t b = (cnt + 255) / 256;
    add_kernel<float><<<(unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), 256, 0, st>>>(
        const_cast<double*>(a.u), d, cnt);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_refine_warp(const RefineArgs& a, float* q, float* g, float* w, float* d,
                               const void* R, int L, cudaStream_t st) {
    return a.n <= 64 ? refine_warp_nr<2>(a, q, g, w, d, R, L, st)
           : a.n <= 128 ? refine_warp_nr<4>(a, q, g, w, d, R, L, st)
                        : refine_warp_nr<16>(a, q, g, w, d, R, L, st);
}

// ---- batched column-owner launches ----------------------------------------------------------
template <typename T, int OP, int NR>
__global__ void __launch_bounds__(256) batch_generic_k(const BatchWork* wk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchWork w = *wk;
    const int64_t total = w.off[w.np];
    constexpr bool per_block = (OP == B_WHITEN || OP == B_LEVEL || OP == B_BASE || OP == B_SELINV);
    constexpr bool per_warp = (OP == B_BACKSUB || OP == B_REFINE_Q || OP == B_REFINE_G ||
                               OP == B_RT_SOLVE || OP == B_BACKSUB_W);
    const int64_t first = per_block ? blockIdx.x
                          : per_warp ? blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)
                                     : blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = per_block ? gridDim.x
                           : per_warp ? (int64_t)gridDim.x * (blockDim.x >> 5)
                                      : (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = first; u < total; u += stride) {
        const int pi = batch_find(w.off, w.np, u);
        const ProbDesc& P = w.desc[w.probs[pi]];
        const int64_t x = u - w.off[pi];
        const int n = P.n;
        const int l = work_level(w, P);
        if constexpr (OP == B_WHITEN) {
            whiten_cta_step<T>(whiten_args_of(P), x, reinterpret_cast<double*>(smem_raw));
        } else if constexpr (OP == B_LEVEL) {
            const int64_t nc = P.k >> l;
            const AosIO<T> io(n, nc, l, P.k, reinterpret_cast<const T*>(P.lvl[l & 1]),
                              reinterpret_cast<T*>(P.lvl[(l + 1) & 1]), reinterpret_cast<T*>(P.R));
            level_cta_tile<T, AosIO<T>>(io, n, nc, l, x, P.resid, P.cn2, P.cd2, P.bad,
                                        reinterpret_cast<T*>(smem_raw));
        } else if constexpr (OP == B_BASE) {
            base_block<T>(n, P.k, P.L, reinterpret_cast<const T*>(P.lvl[P.L & 1]),
                          reinterpret_cast<T*>(P.R), P.cn2, P.cd2, P.bad);
            __syncthreads();
        } else if constexpr (OP == B_BACKSUB) {
            backsub_warp<NR, T, T, double>(n, P.k, l, x, reinterpret_cast<const T*>(P.R), (const T*)nullptr, P.u);
        } else if constexpr (OP == B_SELINV) {
            selinv_cta_row<T, SelAos<T>>(n, P.k, l, x, reinterpret_cast<const T*>(P.R),
                                         reinterpret_cast<T*>(P.Sx), P.cov, P.bad,
                                         reinterpret_cast<T*>(smem_raw));
        } else if constexpr (OP == B_REFINE_Q) {
            refine_q_warp<NR, float>(refine_args_of(P), x, reinterpret_cast<float*>(P.q));
        } else if constexpr (OP == B_REFINE_G) {
            refine_g_warp<NR, float>(refine_args_of(P), x, reinterpret_cast<const float*>(P.q),
                                 reinterpret_cast<float*>(P.g));
        } else if constexpr (OP == B_RT_SOLVE) {
            rt_solve_warp<NR, float, float>(n, P.k, l, x, reinterpret_cast<const float*>(P.R),
                                        reinterpret_cast<float*>(P.g), reinterpret_cast<float*>(P.w));
        } else if constexpr (OP == B_BACKSUB_W) {
            backsub_warp<NR, float, float, float>(n, P.k, l, x, reinterpret_cast<const float*>(P.R),
                                              reinterpret_cast<const float*>(P.w),
                                              reinterpret_cast<float*>(P.d));
        } else if constexpr (OP == B_ADD) {
            P.u[x] += (double)reinterpret_cast<const float*>(P.d)[x];
        }
    }
}

template <typename T, int OP, int NR>
static cudaError_t batch_generic_launch(const BatchWork* wk, unsigned grid, int threads, size_t smem,
                                        cudaStream_t st) {
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(batch_generic_k<T, OP, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_generic_k<T, OP, NR><<<grid, threads, smem, st>>>(wk);
    ++t_launches;
    return cudaGetLastError();
}

// NR = 2: state dimensions up to 64 (every operation); NR = 4: up to 128 (the vector
// operations only -- whitening, levels and SelInv of those sizes run the large-state kernels).
template <typename T, int NR>
static cudaError_t batch_generic_t(int op, int n, int mmax, const BatchWork* wk, unsigned grid,
                                   cudaStream_t st) {
    if constexpr (NR == 2) {
        const int wthreads = ((std::max(3 * n + 2, n + mmax) + 31) / 32) * 32;
        const int lthreads = ((3 * n + 1 + 31) / 32) * 32;
        switch (op) {
            case B_WHITEN:
                return batch_generic_launch<T, B_WHITEN, NR>(wk, grid, wthreads,
                                                             sizeof(double) * (size_t)whiten_layout(n, mmax).total, st);
            case B_LEVEL:
                return batch_generic_launch<T, B_LEVEL, NR>(wk, grid, lthreads, sizeof(T) * (size_t)tile_layout(n).total, st);
            case B_SELINV:
                return batch_generic_launch<T, B_SELINV, NR>(wk, grid, 128, sizeof(T) * (size_t)selinv_layout(n).total, st);
            default: break;
        }
    }
    switch (op) {
        case B_BASE: return batch_generic_launch<T, B_BASE, NR>(wk, grid, 128, 0, st);
        case B_BACKSUB: return batch_generic_launch<T, B_BACKSUB, NR>(wk, grid, 128, 0, st);
        case B_REFINE_Q: return batch_generic_launch<T, B_REFINE_Q, NR>(wk, grid, 128, 0, st);
        case B_REFINE_G: return batch_generic_launch<T, B_REFINE_G, NR>(wk, grid, 128, 0, st);
        case B_RT_SOLVE: return batch_generic_launch<T, B_RT_SOLVE, NR>(wk, grid, 128, 0, st);
        case B_BACKSUB_W: return batch_generic_launch<T, B_BACKSUB_W, NR>(wk, grid, 128, 0, st);
        case B_ADD: return batch_generic_launch<T, B_ADD, NR>(wk, grid, 256, 0, st);
        default: break;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_generic(int op, int n, int mmax, const BatchWork* wk, bool fp32,
                                 unsigned grid, cudaStream_t st, int family) {
    if (use_large(n, fp32) && (op == B_WHITEN || op == B_LEVEL || op == B_SELINV))
        return launch_batch_large(op, n, wk, fp32, grid, st);
    if (op == B_WHITEN)
        if (const MedOps* m = med_whiten_ops(n, mmax, fp32)) return m->batch_whiten(wk, fp32, grid, st);
    if (op == B_WHITEN && !generic_whiten_fits(n, mmax))
        return launch_batch_large(op, n, wk, fp32, grid, st);
    if (op == B_LEVEL && family == 0)
        if (const MedOps* m = med_ops(n, fp32)) return m->batch_level(wk, fp32, grid, st);
    if (n <= 64)
        return fp32 ? batch_generic_t<float, 2>(op, n, mmax, wk, grid, st)
                    : batch_generic_t<double, 2>(op, n, mmax, wk, grid, st);
    return fp32 ? batch_generic_t<float, 4>(op, n, mmax, wk, grid, st)
                : batch_generic_t<double, 4>(op, n, mmax, wk, grid, st);
}

}  // namespace ks

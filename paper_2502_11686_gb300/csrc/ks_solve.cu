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

namespace ks {

constexpr int KS_NMAX = 64;

__device__ __forceinline__ int ctz64(int64_t x) { return __ffsll((long long)x) - 1; }

template <typename TR>
__device__ void backsub_row_generic(int n, int64_t k, int level, int64_t q, const TR* __restrict__ R,
                                    const double* __restrict__ w, double* __restrict__ u) {
    const int64_t c = ((2 * q + 1) << level) - 1;
    if (c >= k) return;
    const int nn = n * n;
    const TR* Rc = R + c * rstore_rs(n);
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    double r[KS_NMAX];
    for (int i = 0; i < n; ++i) r[i] = w ? w[c * n + i] : (double)Rc[3 * nn + i];
    if (a >= 0) {
        const double* ua = u + a * n;
        for (int i = 0; i < n; ++i) {
            double s = r[i];
            for (int p = 0; p < n; ++p) s = fma(-(double)Rc[nn + i * n + p], ua[p], s);
            r[i] = s;
        }
    }
    if (b < k) {
        const double* ub = u + b * n;
        for (int i = 0; i < n; ++i) {
            double s = r[i];
            for (int p = 0; p < n; ++p) s = fma(-(double)Rc[2 * nn + i * n + p], ub[p], s);
            r[i] = s;
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = r[i];
        for (int p = i + 1; p < n; ++p) s = fma(-(double)Rc[i * n + p], r[p], s);
        r[i] = s / (double)Rc[i * n + i];
    }
    for (int i = 0; i < n; ++i) u[c * n + i] = r[i];
}

template <typename TR>
__global__ void backsub_kernel(int n, int64_t k, int level, const TR* __restrict__ R,
                               const double* __restrict__ w, double* __restrict__ u) {
    backsub_row_generic<TR>(n, k, level, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, R, w, u);
}

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

// q_i = K_i^{-1} (F_i u_i + c_i - H_i u_{i+1}) with K_i = L_K L_K^T (one thread per step).
__device__ void refine_q_generic(const RefineArgs& a, int64_t i) {
    if (i + 1 >= a.k) return;
    const int n = a.n, nn = n * n;
    const double* F = a.F + ti_step(a.ti, TI_F, i) * nn;
    const double* H = a.H + ti_step(a.ti, TI_H, i) * nn;
    const double* Lk = a.LK + i * nn;
    const double* u0 = a.u + i * n;
    const double* u1 = a.u + (i + 1) * n;
    double e[KS_NMAX];
    for (int r = 0; r < n; ++r) {
        double s = a.c ? a.c[i * n + r] : 0.0;
        for (int p = 0; p < n; ++p) s = fma(F[r * n + p], u0[p], s);
        for (int p = 0; p < n; ++p) s = fma(-H[r * n + p], u1[p], s);
        e[r] = s;
    }
    for (int r = 0; r < n; ++r) {  // L y = e
        double s = e[r];
        for (int p = 0; p < r; ++p) s = fma(-Lk[r * n + p], e[p], s);
        e[r] = s / Lk[r * n + r];
    }
    for (int r = n - 1; r >= 0; --r) {  // L^T q = y
        double s = e[r];
        for (int p = r + 1; p < n; ++p) s = fma(-Lk[p * n + r], e[p], s);
        e[r] = s / Lk[r * n + r];
    }
    for (int r = 0; r < n; ++r) a.q[i * n + r] = e[r];
}

__global__ void refine_q_kernel(RefineArgs a) {
    refine_q_generic(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// g_c = H_{c-1}^T q_{c-1} - F_c^T q_c + G_c^T C_c^{-1} (o_c - G_c u_c).
__device__ void refine_g_generic(const RefineArgs& a, int64_t c) {
    if (c >= a.k) return;
    const int n = a.n, nn = n * n;
    double g[KS_NMAX];
    for (int r = 0; r < n; ++r) g[r] = 0.0;
    if (c >= 1) {
        const double* H = a.H + ti_step(a.ti, TI_H, c - 1) * nn;
        const double* qv = a.q + (c - 1) * n;
        for (int r = 0; r < n; ++r)
            for (int p = 0; p < n; ++p) g[r] = fma(H[p * n + r], qv[p], g[r]);
    }
    if (c + 1 < a.k) {
        const double* F = a.F + ti_step(a.ti, TI_F, c) * nn;
        const double* qv = a.q + c * n;
        for (int r = 0; r < n; ++r)
            for (int p = 0; p < n; ++p) g[r] = fma(-F[p * n + r], qv[p], g[r]);
    }
    int mi;
    int64_t go, co;
    if (a.m_uniform >= 0) {
        mi = a.m_uniform;
        go = c * mi;
        co = c * (int64_t)mi * mi;
    } else {
        mi = a.m[c];
        go = a.goff[c];
        co = a.coff[c];
    }
    if (mi > 0) {
        const double* G = a.G + ((a.ti & TI_G) ? 0 : go) * n;
        const double* Lc = a.LC + co;
        const double* uc = a.u + c * n;
        double v[KS_NMAX];
        for (int r = 0; r < mi; ++r) {
            double s = a.o[go + r];
            for (int p = 0; p < n; ++p) s = fma(-G[r * n + p], uc[p], s);
            v[r] = s;
        }
        for (int r = 0; r < mi; ++r) {
            double s = v[r];
            for (int p = 0; p < r; ++p) s = fma(-Lc[r * mi + p], v[p], s);
            v[r] = s / Lc[r * mi + r];
        }
        for (int r = mi - 1; r >= 0; --r) {
            double s = v[r];
            for (int p = r + 1; p < mi; ++p) s = fma(-Lc[p * mi + r], v[p], s);
            v[r] = s / Lc[r * mi + r];
        }
        for (int r = 0; r < n; ++r)
            for (int p = 0; p < mi; ++p) g[r] = fma(G[p * n + r], v[p], g[r]);
    }
    for (int r = 0; r < n; ++r) a.g[c * n + r] = g[r];
}

__global__ void refine_g_kernel(RefineArgs a) {
    refine_g_generic(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// R^T w = g at one level: every column alive at `level` first pulls the blocks of the rows
// eliminated at level-1 that touch it (rows c -+ 2^{level-1}), then, if it is eliminated at
// `level`, solves Rd_c^T w_c = g_c.
template <typename TR>
__device__ void rt_solve_generic(int n, int64_t k, int level, int64_t j, const TR* __restrict__ R,
                                 double* __restrict__ g, double* __restrict__ w) {
    if (j >= (k >> level)) return;
    const int64_t c = ((j + 1) << level) - 1;
    const int nn = n * n;
    const int64_t RS = rstore_rs(n);
    double r[KS_NMAX];
    for (int i = 0; i < n; ++i) r[i] = g[c * n + i];
    if (level >= 1) {
        const int64_t h = 1LL << (level - 1);
        if (c - h >= 0) {  // row c-h has its right block Rr at column c
            const TR* Rr = R + (c - h) * RS + 2 * nn;
            const double* wr = w + (c - h) * n;
            for (int i = 0; i < n; ++i) {
                double s = r[i];
                for (int p = 0; p < n; ++p) s = fma(-(double)Rr[p * n + i], wr[p], s);
                r[i] = s;
            }
        }
        if (c + h < k) {  // row c+h has its left block Rl at column c
            const TR* Rl = R + (c + h) * RS + nn;
            const double* wr = w + (c + h) * n;
            for (int i = 0; i < n; ++i) {
                double s = r[i];
                for (int p = 0; p < n; ++p) s = fma(-(double)Rl[p * n + i], wr[p], s);
                r[i] = s;
            }
        }
    }
    if (ctz64(c + 1) == level) {
        const TR* Rd = R + c * RS;
        for (int i = 0; i < n; ++i) {
            double s = r[i];
            for (int p = 0; p < i; ++p) s = fma(-(double)Rd[p * n + i], r[p], s);
            r[i] = s / (double)Rd[i * n + i];
        }
        for (int i = 0; i < n; ++i) w[c * n + i] = r[i];
    } else {
        for (int i = 0; i < n; ++i) g[c * n + i] = r[i];
    }
}

template <typename TR>
__global__ void rt_solve_kernel(int n, int64_t k, int level, const TR* __restrict__ R,
                                double* __restrict__ g, double* __restrict__ w) {
    rt_solve_generic<TR>(n, k, level, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, R, g, w);
}

__global__ void axpy_kernel(double* __restrict__ u, const double* __restrict__ d, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        u[i] += d[i];
}

static unsigned grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1LL << 30)) b = 1LL << 30;
    return (unsigned)b;
}

cudaError_t launch_backsub(int n, int64_t k, int level, const void* R, const double* w,
                           double* u, bool fp32, cudaStream_t st) {
    const int64_t cols = ((k >> level) + 1) / 2;
    const int threads = 128;
    if (fp32)
        backsub_kernel<float><<<grid_for(cols, threads), threads, 0, st>>>(n, k, level, (const float*)R, w, u);
    else
        backsub_kernel<double><<<grid_for(cols, threads), threads, 0, st>>>(n, k, level, (const double*)R, w, u);
    ++t_launches;
    return cudaGetLastError();
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

cudaError_t launch_refine_gradient(const RefineArgs& a, cudaStream_t st) {
    if (a.k > 1) {
        refine_q_kernel<<<grid_for(a.k - 1, 128), 128, 0, st>>>(a);
        ++t_launches;
    }
    refine_g_kernel<<<grid_for(a.k, 128), 128, 0, st>>>(a);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_rt_solve(int n, int64_t k, int level, const void* R, double* g, double* w,
                            bool fp32, cudaStream_t st) {
    const int64_t cols = k >> level;
    if (fp32)
        rt_solve_kernel<float><<<grid_for(cols, 128), 128, 0, st>>>(n, k, level, (const float*)R, g, w);
    else
        rt_solve_kernel<double><<<grid_for(cols, 128), 128, 0, st>>>(n, k, level, (const double*)R, g, w);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_axpy(double* u, const double* d, int64_t count, cudaStream_t st) {
    axpy_kernel<<<grid_for(count, 256) > 4096 ? 4096 : grid_for(count, 256), 256, 0, st>>>(u, d, count);
    ++t_launches;
    return cudaGetLastError();
}

// ---- warp-per-unit kernels of the column-owner path -----------------------------------------
// One warp per block row / column / step; lane l owns rows l and l+32 (n <= 64).  Triangular
// substitutions proceed one unknown at a time: its owner lane divides and broadcasts it with a
// shuffle, and every lane updates its own rows.  In FP32 + refinement mode the vectors are FP32
// except the residuals of the refinement, which are formed in FP64.

// Back substitution of block row q at `level`: u_c = Rd^{-1}(rhs - Rl u_a - Rr u_b).
// rhs = y from the R store (w == nullptr) or w_c.  Vectors of type TV, output of type TO.
template <typename TR, typename TV, typename TO>
__device__ void backsub_warp(int n, int64_t k, int level, int64_t q, const TR* __restrict__ R,
                             const TV* __restrict__ w, TO* __restrict__ u) {
    const int lane = threadIdx.x & 31;
    const int64_t c = ((2 * q + 1) << level) - 1;
    if (c >= k) return;
    const int nn = n * n;
    const TR* Rc = R + c * rstore_rs(n);
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    TV r0 = TV(0), r1 = TV(0);
    const int i0 = lane, i1 = lane + 32;
    if (i0 < n) r0 = w ? w[c * n + i0] : (TV)Rc[3 * nn + i0];
    if (i1 < n) r1 = w ? w[c * n + i1] : (TV)Rc[3 * nn + i1];
    if (a >= 0) {
        for (int p = 0; p < n; ++p) {
            const TV up = (TV)u[a * n + p];
            if (i0 < n) r0 = fma(-(TV)Rc[nn + i0 * n + p], up, r0);
            if (i1 < n) r1 = fma(-(TV)Rc[nn + i1 * n + p], up, r1);
        }
    }
    if (b < k) {
        for (int p = 0; p < n; ++p) {
            const TV up = (TV)u[b * n + p];
            if (i0 < n) r0 = fma(-(TV)Rc[2 * nn + i0 * n + p], up, r0);
            if (i1 < n) r1 = fma(-(TV)Rc[2 * nn + i1 * n + p], up, r1);
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        TV x = TV(0);
        if ((i & 31) == lane) x = ((i < 32) ? r0 : r1) / (TV)Rc[i * n + i];
        x = __shfl_sync(0xffffffffu, x, i & 31);
        if (i0 < i) r0 = fma(-(TV)Rc[i0 * n + i], x, r0);
        if (i1 < i) r1 = fma(-(TV)Rc[i1 * n + i], x, r1);
        if (i0 == i) r0 = x;
        if (i1 == i) r1 = x;
    }
    if (i0 < n) u[c * n + i0] = (TO)r0;
    if (i1 < n) u[c * n + i1] = (TO)r1;
}

// R^T w = g at `level` for alive column j (pull the two rows eliminated at level-1 that touch
// it, then solve with Rd^T if it is eliminated here).
template <typename TR, typename TV>
__device__ void rt_solve_warp(int n, int64_t k, int level, int64_t j, const TR* __restrict__ R,
                              TV* __restrict__ g, TV* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    if (j >= (k >> level)) return;
    const int64_t c = ((j + 1) << level) - 1;
    const int nn = n * n;
    const int64_t RS = rstore_rs(n);
    const int i0 = lane, i1 = lane + 32;
    TV r0 = i0 < n ? g[c * n + i0] : TV(0), r1 = i1 < n ? g[c * n + i1] : TV(0);
    if (level >= 1) {
        const int64_t h = 1LL << (level - 1);
        if (c - h >= 0) {
            const TR* Rr = R + (c - h) * RS + 2 * nn;
            const TV* wr = w + (c - h) * n;
            for (int p = 0; p < n; ++p) {
                const TV wp = wr[p];
                if (i0 < n) r0 = fma(-(TV)Rr[p * n + i0], wp, r0);
                if (i1 < n) r1 = fma(-(TV)Rr[p * n + i1], wp, r1);
            }
        }
        if (c + h < k) {
            const TR* Rl = R + (c + h) * RS + nn;
            const TV* wr = w + (c + h) * n;
            for (int p = 0; p < n; ++p) {
                const TV wp = wr[p];
                if (i0 < n) r0 = fma(-(TV)Rl[p * n + i0], wp, r0);
                if (i1 < n) r1 = fma(-(TV)Rl[p * n + i1], wp, r1);
            }
        }
    }
    if (ctz64(c + 1) == level) {
        const TR* Rd = R + c * RS;
        for (int i = 0; i < n; ++i) {
            TV x = TV(0);
            if ((i & 31) == lane) x = ((i < 32) ? r0 : r1) / (TV)Rd[i * n + i];
            x = __shfl_sync(0xffffffffu, x, i & 31);
            if (i0 > i && i0 < n) r0 = fma(-(TV)Rd[i * n + i0], x, r0);
            if (i1 > i && i1 < n) r1 = fma(-(TV)Rd[i * n + i1], x, r1);
            if (i0 == i) r0 = x;
            if (i1 == i) r1 = x;
        }
        if (i0 < n) w[c * n + i0] = r0;
        if (i1 < n) w[c * n + i1] = r1;
    } else {
        if (i0 < n) g[c * n + i0] = r0;
        if (i1 < n) g[c * n + i1] = r1;
    }
}

// Warp-cooperative solves with an FP64 lower-triangular factor L (ld = dim), in type TV:
// forward (L y = x) then backward (L^T z = y); x given per lane in rows lane, lane+32.
template <typename TV>
__device__ void llt_solve_warp(int dim, const double* __restrict__ Lf, TV& r0, TV& r1) {
    const int lane = threadIdx.x & 31;
    const int i0 = lane, i1 = lane + 32;
    for (int i = 0; i < dim; ++i) {
        TV x = TV(0);
        if ((i & 31) == lane) x = ((i < 32) ? r0 : r1) / (TV)Lf[i * dim + i];
        x = __shfl_sync(0xffffffffu, x, i & 31);
        if (i0 > i && i0 < dim) r0 = fma(-(TV)Lf[i0 * dim + i], x, r0);
        if (i1 > i && i1 < dim) r1 = fma(-(TV)Lf[i1 * dim + i], x, r1);
        if (i0 == i) r0 = x;
        if (i1 == i) r1 = x;
    }
    for (int i = dim - 1; i >= 0; --i) {
        TV x = TV(0);
        if ((i & 31) == lane) x = ((i < 32) ? r0 : r1) / (TV)Lf[i * dim + i];
        x = __shfl_sync(0xffffffffu, x, i & 31);
        if (i0 < i) r0 = fma(-(TV)Lf[i * dim + i0], x, r0);
        if (i1 < i) r1 = fma(-(TV)Lf[i * dim + i1], x, r1);
        if (i0 == i) r0 = x;
        if (i1 == i) r1 = x;
    }
}

// q_i = K_i^{-1} (F_i u_i + c_i - H_i u_{i+1}): the residual in FP64, the solve in TV.
template <typename TV>
__device__ void refine_q_warp(const RefineArgs& a, int64_t i, TV* __restrict__ q) {
    if (i + 1 >= a.k) return;
    const int lane = threadIdx.x & 31, n = a.n, nn = n * n;
    const double* F = a.F + ti_step(a.ti, TI_F, i) * nn;
    const double* H = a.H + ti_step(a.ti, TI_H, i) * nn;
    double e0 = 0.0, e1 = 0.0;
    const int i0 = lane, i1 = lane + 32;
    if (i0 < n) e0 = a.c ? a.c[i * n + i0] : 0.0;
    if (i1 < n) e1 = a.c ? a.c[i * n + i1] : 0.0;
    for (int p = 0; p < n; ++p) {
        const double u0 = a.u[i * n + p], u1 = a.u[(i + 1) * n + p];
        if (i0 < n) e0 = fma(-H[i0 * n + p], u1, fma(F[i0 * n + p], u0, e0));
        if (i1 < n) e1 = fma(-H[i1 * n + p], u1, fma(F[i1 * n + p], u0, e1));
    }
    TV r0 = (TV)e0, r1 = (TV)e1;
    llt_solve_warp<TV>(n, a.LK + i * nn, r0, r1);
    if (i0 < n) q[i * n + i0] = r0;
    if (i1 < n) q[i * n + i1] = r1;
}

// g_c = H_{c-1}^T q_{c-1} - F_c^T q_c + G_c^T C_c^{-1} (o_c - G_c u_c), o - G u in FP64.
template <typename TV>
__device__ void refine_g_warp(const RefineArgs& a, int64_t c, const TV* __restrict__ q,
                              TV* __restrict__ g) {
    if (c >= a.k) return;
    const int lane = threadIdx.x & 31, n = a.n, nn = n * n;
    const int i0 = lane, i1 = lane + 32;
    TV g0 = TV(0), g1 = TV(0);
    if (c >= 1) {
        const double* H = a.H + ti_step(a.ti, TI_H, c - 1) * nn;
        for (int p = 0; p < n; ++p) {
            const TV qp = q[(c - 1) * n + p];
            if (i0 < n) g0 = fma((TV)H[p * n + i0], qp, g0);
            if (i1 < n) g1 = fma((TV)H[p * n + i1], qp, g1);
        }
    }
    if (c + 1 < a.k) {
        const double* F = a.F + ti_step(a.ti, TI_F, c) * nn;
        for (int p = 0; p < n; ++p) {
            const TV qp = q[c * n + p];
            if (i0 < n) g0 = fma(-(TV)F[p * n + i0], qp, g0);
            if (i1 < n) g1 = fma(-(TV)F[p * n + i1], qp, g1);
        }
    }
    int mi;
    int64_t go, co;
    if (a.m_uniform >= 0) {
        mi = a.m_uniform;
        go = c * mi;
        co = c * (int64_t)mi * mi;
    } else {
        mi = a.m[c];
        go = a.goff[c];
        co = a.coff[c];
    }
    if (mi > 0) {
        const double* G = a.G + ((a.ti & TI_G) ? 0 : go) * n;
        double v0 = 0.0, v1 = 0.0;
        if (i0 < mi) v0 = a.o[go + i0];
        if (i1 < mi) v1 = a.o[go + i1];
        for (int p = 0; p < n; ++p) {
            const double up = a.u[c * n + p];
            if (i0 < mi) v0 = fma(-G[i0 * n + p], up, v0);
            if (i1 < mi) v1 = fma(-G[i1 * n + p], up, v1);
        }
        TV r0 = (TV)v0, r1 = (TV)v1;
        llt_solve_warp<TV>(mi, a.LC + co, r0, r1);
        for (int p = 0; p < mi; ++p) {
            const TV vp = __shfl_sync(0xffffffffu, p < 32 ? r0 : r1, p & 31);
            if (i0 < n) g0 = fma((TV)G[p * n + i0], vp, g0);
            if (i1 < n) g1 = fma((TV)G[p * n + i1], vp, g1);
        }
    }
    if (i0 < n) g[c * n + i0] = g0;
    if (i1 < n) g[c * n + i1] = g1;
}

template <typename TR, typename TV, typename TO>
__global__ void __launch_bounds__(128) backsub_warp_kernel(int n, int64_t k, int level, const TR* R,
                                                           const TV* w, TO* u) {
    const int64_t q = blockIdx.x * 4LL + (threadIdx.x >> 5);
    if (q < (k >> level) - (k >> (level + 1))) backsub_warp<TR, TV, TO>(n, k, level, q, R, w, u);
}

template <typename TR, typename TV>
__global__ void __launch_bounds__(128) rt_solve_warp_kernel(int n, int64_t k, int level, const TR* R,
                                                            TV* g, TV* w) {
    rt_solve_warp<TR, TV>(n, k, level, blockIdx.x * 4LL + (threadIdx.x >> 5), R, g, w);
}

template <typename TV>
__global__ void __launch_bounds__(128) refine_qg_warp_kernel(RefineArgs a, int which, TV* q, TV* g) {
    const int64_t x = blockIdx.x * 4LL + (threadIdx.x >> 5);
    if (which == 0) refine_q_warp<TV>(a, x, q);
    else refine_g_warp<TV>(a, x, q, g);
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

cudaError_t launch_backsub_warp(int n, int64_t k, int level, const void* R, bool fp32,
                                double* u, cudaStream_t st) {
    const int64_t rows = (k >> level) - (k >> (level + 1));
    if (fp32)  // FP32 first solve; the refinement corrects it
        backsub_warp_kernel<float, float, double><<<warps_grid(rows), 128, 0, st>>>(
            n, k, level, (const float*)R, (const float*)nullptr, u);
    else
        backsub_warp_kernel<double, double, double><<<warps_grid(rows), 128, 0, st>>>(
            n, k, level, (const double*)R, (const double*)nullptr, u);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_refine_warp(const RefineArgs& a, float* q, float* g, float* w, float* d,
                               const void* R, int L, cudaStream_t st) {
    const int64_t k = a.k;
    const float* Rf = static_cast<const float*>(R);
    if (k > 1) {
        refine_qg_warp_kernel<float><<<warps_grid(k - 1), 128, 0, st>>>(a, 0, q, g);
        ++t_launches;
    }
    refine_qg_warp_kernel<float><<<warps_grid(k), 128, 0, st>>>(a, 1, q, g);
    ++t_launches;
    for (int l = 0; l <= L; ++l) {
        rt_solve_warp_kernel<float, float><<<warps_grid(k >> l), 128, 0, st>>>(a.n, k, l, Rf, g, w);
        ++t_launches;
    }
    for (int l = L; l >= 0; --l) {
        backsub_warp_kernel<float, float, float><<<warps_grid((k >> l) - (k >> (l + 1))), 128, 0, st>>>(
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

// ---- batched column-owner launches ----------------------------------------------------------
template <typename T, int OP>
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
            backsub_warp<T, T, double>(n, P.k, l, x, reinterpret_cast<const T*>(P.R), (const T*)nullptr, P.u);
        } else if constexpr (OP == B_SELINV) {
            selinv_cta_row<T, SelAos<T>>(n, P.k, l, x, reinterpret_cast<const T*>(P.R),
                                         reinterpret_cast<T*>(P.Sx), P.cov, P.bad,
                                         reinterpret_cast<T*>(smem_raw));
        } else if constexpr (OP == B_REFINE_Q) {
            refine_q_warp<float>(refine_args_of(P), x, reinterpret_cast<float*>(P.q));
        } else if constexpr (OP == B_REFINE_G) {
            refine_g_warp<float>(refine_args_of(P), x, reinterpret_cast<const float*>(P.q),
                                 reinterpret_cast<float*>(P.g));
        } else if constexpr (OP == B_RT_SOLVE) {
            rt_solve_warp<float, float>(n, P.k, l, x, reinterpret_cast<const float*>(P.R),
                                        reinterpret_cast<float*>(P.g), reinterpret_cast<float*>(P.w));
        } else if constexpr (OP == B_BACKSUB_W) {
            backsub_warp<float, float, float>(n, P.k, l, x, reinterpret_cast<const float*>(P.R),
                                              reinterpret_cast<const float*>(P.w),
                                              reinterpret_cast<float*>(P.d));
        } else if constexpr (OP == B_ADD) {
            P.u[x] += (double)reinterpret_cast<const float*>(P.d)[x];
        }
    }
}

template <typename T, int OP>
static cudaError_t batch_generic_launch(const BatchWork* wk, unsigned grid, int threads, size_t smem,
                                        cudaStream_t st) {
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(batch_generic_k<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_generic_k<T, OP><<<grid, threads, smem, st>>>(wk);
    ++t_launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t batch_generic_t(int op, int n, int mmax, const BatchWork* wk, unsigned grid,
                                   cudaStream_t st) {
    const int wthreads = ((std::max(3 * n + 2, n + mmax) + 31) / 32) * 32;
    const int lthreads = ((3 * n + 1 + 31) / 32) * 32;
    switch (op) {
        case B_WHITEN:
            return batch_generic_launch<T, B_WHITEN>(wk, grid, wthreads,
                                                     sizeof(double) * (size_t)whiten_layout(n, mmax).total, st);
        case B_LEVEL:
            return batch_generic_launch<T, B_LEVEL>(wk, grid, lthreads, sizeof(T) * (size_t)tile_layout(n).total, st);
        case B_BASE: return batch_generic_launch<T, B_BASE>(wk, grid, 128, 0, st);
        case B_BACKSUB: return batch_generic_launch<T, B_BACKSUB>(wk, grid, 128, 0, st);
        case B_SELINV:
            return batch_generic_launch<T, B_SELINV>(wk, grid, 128, sizeof(T) * (size_t)selinv_layout(n).total, st);
        case B_REFINE_Q: return batch_generic_launch<T, B_REFINE_Q>(wk, grid, 128, 0, st);
        case B_REFINE_G: return batch_generic_launch<T, B_REFINE_G>(wk, grid, 128, 0, st);
        case B_RT_SOLVE: return batch_generic_launch<T, B_RT_SOLVE>(wk, grid, 128, 0, st);
        case B_BACKSUB_W: return batch_generic_launch<T, B_BACKSUB_W>(wk, grid, 128, 0, st);
        case B_ADD: return batch_generic_launch<T, B_ADD>(wk, grid, 256, 0, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_generic(int op, int n, int mmax, const BatchWork* wk, bool fp32,
                                 unsigned grid, cudaStream_t st) {
    return fp32 ? batch_generic_t<float>(op, n, mmax, wk, grid, st)
                : batch_generic_t<double>(op, n, mmax, wk, grid, st);
}

}  // namespace ks

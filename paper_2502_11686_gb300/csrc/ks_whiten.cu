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
#include "ks_householder.cuh"
#include "ks_internal.cuh"

namespace ks {

template <typename T>
__global__ void __launch_bounds__(256) whiten_kernel(WhitenArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sm = reinterpret_cast<double*>(smem_raw);
    const int n = a.n;
    const WhitenLayout L = whiten_layout(n, a.mmax);
    double* KC = sm + L.kc;
    double* W = sm + L.w;
    double* OC = sm + L.oc;
    double* Gm = sm + L.g;
    double* Tt = sm + L.t;
    double* scal = sm + L.scal;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t CS = level_cs(n);
    T* out = reinterpret_cast<T*>(a.level0);

    for (int64_t i = blockIdx.x; i < a.k; i += gridDim.x) {
        int mi;
        int64_t go, co;
        if (a.m_uniform >= 0) {
            mi = a.m_uniform;
            go = i * mi;
            co = i * (int64_t)mi * mi;
        } else {
            mi = a.m[i];
            go = a.goff[i];
            co = a.coff[i];
        }
        const bool hasE = (i + 1 < a.k);
        // ---- loads (coalesced over the row-major source blocks) ----
        if (hasE) {
            const double* Ki = a.K + i * (int64_t)n * n;
            const double* Fi = a.F + i * (int64_t)n * n;
            const double* Hi = a.H + i * (int64_t)n * n;
            for (int e = tid; e < n * n; e += nth) {
                int r = e / n, c = e - r * n;
                KC[r * L.ldk + c] = Ki[e];
                W[r * L.ldw + c] = -Fi[e];
                W[r * L.ldw + n + c] = Hi[e];
            }
            for (int r = tid; r < n; r += nth) W[r * L.ldw + 2 * n] = a.c ? a.c[i * n + r] : 0.0;
        }
        for (int e = tid; e < mi * mi; e += nth) {
            int r = e / mi, c = e - r * mi;
            OC[r * L.ldo + c] = a.C[co + e];
        }
        for (int e = tid; e < mi * n; e += nth) {
            int r = e / n, c = e - r * n;
            Gm[r * L.ldg + c] = a.G[go * n + e];
        }
        for (int r = tid; r < mi; r += nth) Gm[r * L.ldg + n] = a.o[go + r];
        for (int e = tid; e < n * L.ldt; e += nth) Tt[e] = 0.0;
        __syncthreads();

        // ---- Cholesky of K_i (threads [0,n)) and C_i (threads [n, n+mi)), right-looking,
        //      thread = column owner ----
        const int nK = hasE ? n : 0;
        const int steps = nK > mi ? nK : mi;
        double* A = nullptr;
        int lda = 0, col = -1, dim = 0;
        if (tid < nK) {
            A = KC; lda = L.ldk; col = tid; dim = nK;
        } else if (tid >= n && tid < n + mi) {
            A = OC; lda = L.ldo; col = tid - n; dim = mi;
        }
        for (int j = 0; j < steps; ++j) {
            if (A != nullptr && col == j && j < dim) {
                double d = A[j * lda + j];
                if (!(d > 0.0) || !isfinite(d)) {
                    flag_error(a.bad, ST_NOT_SPD, i);
                    d = 1.0;
                }
                d = sqrt(d);
                A[j * lda + j] = d;
                const double inv = 1.0 / d;
                for (int r = j + 1; r < dim; ++r) A[r * lda + j] *= inv;
            }
            __syncthreads();
            if (A != nullptr && col > j && col < dim) {
                const double lcj = A[col * lda + j];
                for (int r = col; r < dim; ++r) A[r * lda + col] = fma(-A[r * lda + j], lcj, A[r * lda + col]);
            }
            __syncthreads();
        }

        // ---- forward substitution: W <- L_K^{-1} W (2n+1 columns), Gm <- L_C^{-1} Gm ----
        {
            double* B = nullptr;
            const double* Lf = nullptr;
            int ldb = 0, ldl = 0, dim2 = 0;
            if (tid < 2 * n + 1) {
                if (hasE) { B = W + tid; ldb = L.ldw; Lf = KC; ldl = L.ldk; dim2 = n; }
            } else if (tid < 3 * n + 2) {
                if (mi > 0) { B = Gm + (tid - 2 * n - 1); ldb = L.ldg; Lf = OC; ldl = L.ldo; dim2 = mi; }
            }
            if (B != nullptr) {
                for (int r = 0; r < dim2; ++r) {
                    double s = B[r * ldb];
                    for (int q = 0; q < r; ++q) s = fma(-Lf[r * ldl + q], B[q * ldb], s);
                    B[r * ldb] = s / Lf[r * ldl + r];
                }
            }
        }
        __syncthreads();

        // ---- reduce the observation block: QR of [0 (n x n) ; Chat (mi x n)] with its rhs ----
        {
            const int fcol = (tid < n) ? tid : -1;
            double* ctop = (tid == n) ? (Tt + n) : nullptr;
            double* cbot = (tid == n) ? (Gm + n) : nullptr;
            tpqrt_columns<double>(n, mi, Tt, L.ldt, Gm, L.ldg, fcol, ctop, L.ldt, cbot, L.ldg, scal);
        }

        // ---- stores ----
        T* rec = out + i * CS;
        for (int e = tid; e < n * n; e += nth) {
            int r = e / n, c = e - r * n;
            rec[e] = (T)(c >= r ? Tt[r * L.ldt + c] : 0.0);
        }
        for (int r = tid; r < n; r += nth) rec[n * n + r] = (T)Tt[r * L.ldt + n];
        if (hasE) {
            T* nxt = out + (i + 1) * CS + (int64_t)n * n + n;
            for (int e = tid; e < 2 * n * n; e += nth) {
                int r = e / (2 * n), c = e - r * 2 * n;
                nxt[e] = (T)W[r * L.ldw + c];
            }
            for (int r = tid; r < n; r += nth) nxt[2 * n * n + r] = (T)W[r * L.ldw + 2 * n];
            if (a.LK != nullptr) {
                double* lk = a.LK + i * (int64_t)n * n;
                for (int e = tid; e < n * n; e += nth) {
                    int r = e / n, c = e - r * n;
                    lk[e] = c <= r ? KC[r * L.ldk + c] : 0.0;
                }
            }
        }
        if (a.LC != nullptr) {
            for (int e = tid; e < mi * mi; e += nth) {
                int r = e / mi, c = e - r * mi;
                a.LC[co + e] = c <= r ? OC[r * L.ldo + c] : 0.0;
            }
        }
        if (tid == 0) {
            double s = 0.0;
            for (int r = 0; r < mi; ++r) s = fma(Gm[r * L.ldg + n], Gm[r * L.ldg + n], s);
            a.resid[i] = s;
        }
        // Column norms^2 of U A for state i (Chat_i and B_i) and state i+1 (D_i).
        for (int col = tid; col < n; col += nth) {
            double sc = 0.0, sb = 0.0, sd = 0.0;
            for (int r = 0; r <= col; ++r) sc = fma(Tt[r * L.ldt + col], Tt[r * L.ldt + col], sc);
            if (hasE) {
                for (int r = 0; r < n; ++r) {
                    sb = fma(W[r * L.ldw + col], W[r * L.ldw + col], sb);
                    sd = fma(W[r * L.ldw + n + col], W[r * L.ldw + n + col], sd);
                }
                a.cd2[(i + 1) * n + col] = sd;
            }
            a.cn2[i * n + col] = sc + sb;
            if (i == 0) a.cd2[col] = 0.0;
        }
        __syncthreads();
    }
}

cudaError_t launch_whiten(const WhitenArgs& a, bool fp32, cudaStream_t st) {
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

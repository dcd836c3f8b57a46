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
#include "ks_householder.cuh"
#include "ks_internal.cuh"

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
    const TileLayout L = tile_layout(n);
    T* TOP2 = sm + L.top2;
    T* BOT2 = sm + L.bot2;
    T* BF = sm + L.bf;
    T* TOP3 = sm + L.top3;
    T* BOT3 = sm + L.bot3;
    T* scal = sm + L.scal;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nn = n * n;
    const int64_t nt = nc / 2;
    const IO io(n, nc, level, k, in, out, R);

    for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const int64_t j = 2 * t, s = j + 1;
        const bool triple = (nc & 1) && (t == nt - 1);
        const int64_t oj = ((j + 1) << level) - 1;  // original index of column j

        // ---- loads ----
        for (int e = tid; e < n * L.ld2; e += nth) {
            int r = e / L.ld2, c = e - r * L.ld2;
            T v = T(0);
            if (c < n) v = io.C(j, r, c);
            else if (c == 3 * n) v = io.RC(j, r);
            TOP2[e] = v;
        }
        if (j >= 1) {
            for (int e = tid; e < n * L.ld2; e += nth) {
                int r = e / L.ld2, c = e - r * L.ld2;
                T v = T(0);
                if (c < n) v = io.E(j, r, n + c);                  // D_j (factor bottom)
                else if (c < 2 * n) v = io.E(j, r, c - n);         // -B_j (left companion)
                else if (c == 3 * n) v = io.RE(j, r);              // rE_j
                BOT2[e] = v;
            }
        }
        {
            for (int e = tid; e < nn; e += nth) {
                int r = e / n, c = e - r * n;
                BF[r * L.ldf + c] = io.E(s, r, c);                  // -B_s
                BOT3[r * L.ld3 + c] = io.E(s, r, n + c);            // D_s
            }
            for (int r = tid; r < n; r += nth) BOT3[r * L.ld3 + n] = io.RE(s, r);    // rE_s
            for (int e = tid; e < nn; e += nth) {
                int r = e / n, c = e - r * n;
                TOP3[r * L.ld3 + c] = io.C(s, r, c);                // Chat_s
            }
            for (int r = tid; r < n; r += nth) TOP3[r * L.ld3 + n] = io.RC(s, r);    // rC_s
        }
        __syncthreads();

        // ---- step 1: [Chat_j ; -B_s] ----
        {
            const int fcol = tid < n ? tid : -1;
            T* ctop = nullptr;
            T* cbot = nullptr;
            if (tid >= n && tid < 2 * n) {
                ctop = TOP2 + 2 * n + (tid - n);
                cbot = BOT3 + (tid - n);
            } else if (tid == 2 * n) {
                ctop = TOP2 + 3 * n;
                cbot = BOT3 + n;
            }
            tpqrt_columns<T>(n, n, TOP2, L.ld2, BF, L.ldf, fcol, ctop, L.ld2, cbot, L.ld3, scal);
        }
        // ---- step 2: [Rtilde_j ; D_j] with companions [0 ; -B_j], [X_j ; 0], rhs ----
        if (j >= 1) {
            const int fcol = tid < n ? tid : -1;
            T* ctop = nullptr;
            T* cbot = nullptr;
            if (tid >= n && tid <= 3 * n) {
                ctop = TOP2 + tid;
                cbot = BOT2 + tid;
            }
            tpqrt_columns<T>(n, n, TOP2, L.ld2, BOT2, L.ld2, fcol, ctop, L.ld2, cbot, L.ld2, scal);
        }
        // ---- block row j of R, and the reduced coupling row of new column t ----
        {
            for (int e = tid; e < nn; e += nth) {
                int r = e / n, c = e - r * n;
                io.setR(t, oj, 0, r, c, c >= r ? TOP2[r * L.ld2 + c] : T(0));
                io.setR(t, oj, 1, r, c, (j >= 1) ? TOP2[r * L.ld2 + n + c] : T(0));
                io.setR(t, oj, 2, r, c, TOP2[r * L.ld2 + 2 * n + c]);
            }
            for (int r = tid; r < n; r += nth) {
                io.setY(t, oj, r, TOP2[r * L.ld2 + 3 * n]);
                if (diag_is_singular<T>(TOP2[r * L.ld2 + r], cn2[oj * n + r] + cd2[oj * n + r], n))
                    flag_error(bad, ST_SINGULAR, oj);
            }
            if (j >= 1) {
                for (int e = tid; e < 2 * nn; e += nth) {
                    int r = e / (2 * n), c = e - r * 2 * n;
                    io.setE(t, r, c, BOT2[r * L.ld2 + n + c]);
                }
                for (int r = tid; r < n; r += nth) io.setRE(t, r, BOT2[r * L.ld2 + 3 * n]);
            }
        }
        __syncthreads();

        // ---- tail: step 2 of column e (no right neighbour), reusing TOP2 / BF ----
        if (triple) {
            const int64_t e_ = j + 2;
            const int64_t oe = ((e_ + 1) << level) - 1;
            for (int e = tid; e < n * L.ld2; e += nth) {
                int r = e / L.ld2, c = e - r * L.ld2;
                T v = T(0);
                if (c < n) v = io.C(e_, r, c);
                else if (c == 2 * n) v = io.RC(e_, r);
                TOP2[e] = v;
            }
            for (int e = tid; e < nn; e += nth) {
                int r = e / n, c = e - r * n;
                BF[r * L.ldf + c] = io.E(e_, r, n + c);                 // D_e
                BOT3[(n + r) * L.ld3 + c] = io.E(e_, r, c);             // -B_e -> Z_e
            }
            for (int r = tid; r < n; r += nth) BOT3[(n + r) * L.ld3 + n] = io.RE(e_, r);
            __syncthreads();
            {
                const int fcol = tid < n ? tid : -1;
                T* ctop = nullptr;
                T* cbot = nullptr;
                if (tid >= n && tid < 2 * n) {
                    ctop = TOP2 + tid;
                    cbot = BOT3 + n * L.ld3 + (tid - n);
                } else if (tid == 2 * n) {
                    ctop = TOP2 + 2 * n;
                    cbot = BOT3 + n * L.ld3 + n;
                }
                tpqrt_columns<T>(n, n, TOP2, L.ld2, BF, L.ldf, fcol, ctop, L.ld2, cbot, L.ld3, scal);
            }
            for (int e = tid; e < nn; e += nth) {
                int r = e / n, c = e - r * n;
                io.setR(t + 1, oe, 0, r, c, c >= r ? TOP2[r * L.ld2 + c] : T(0));
                io.setR(t + 1, oe, 1, r, c, TOP2[r * L.ld2 + n + c]);
                io.setR(t + 1, oe, 2, r, c, T(0));
            }
            for (int r = tid; r < n; r += nth) {
                io.setY(t + 1, oe, r, TOP2[r * L.ld2 + 2 * n]);
                if (diag_is_singular<T>(TOP2[r * L.ld2 + r], cn2[oe * n + r] + cd2[oe * n + r], n))
                    flag_error(bad, ST_SINGULAR, oe);
            }
            __syncthreads();
        }

        // ---- step 3: [Chat_s ; Dtilde_s (; Z_e)] -> reduced diagonal block of column t ----
        {
            const int p3 = triple ? 2 * n : n;
            const int fcol = tid < n ? tid : -1;
            T* ctop = (tid == n) ? TOP3 + n : nullptr;
            T* cbot = (tid == n) ? BOT3 + n : nullptr;
            tpqrt_columns<T>(n, p3, TOP3, L.ld3, BOT3, L.ld3, fcol, ctop, L.ld3, cbot, L.ld3, scal);
            for (int e = tid; e < nn; e += nth) {
                int r = e / n, c = e - r * n;
                io.setC(t, r, c, TOP3[r * L.ld3 + c]);
            }
            for (int r = tid; r < n; r += nth) io.setRC(t, r, TOP3[r * L.ld3 + n]);
            if (tid == 0) {
                double acc = 0.0;
                for (int r = 0; r < p3; ++r) {
                    double v = (double)BOT3[r * L.ld3 + n];
                    acc = fma(v, v, acc);
                }
                resid[oj] = acc;
            }
        }
        __syncthreads();
    }
}

// The last alive column becomes the base block row: Rd = Chat (already triangular), y = rC.
template <typename T>
__global__ void base_kernel(int n, int64_t k, int L, const T* __restrict__ in, T* __restrict__ R,
                            const double* __restrict__ cn2, const double* __restrict__ cd2,
                            unsigned long long* bad) {
    const int64_t c = (1LL << L) - 1;
    const int nn = n * n;
    T* Rc = R + c * rstore_rs(n);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        Rc[e] = in[e];
        Rc[nn + e] = T(0);
        Rc[2 * nn + e] = T(0);
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        Rc[3 * nn + r] = in[nn + r];
        if (diag_is_singular<T>(in[r * n + r], cn2[c * n + r] + cd2[c * n + r], n))
            flag_error(bad, ST_SINGULAR, c);
    }
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

// ks_householder.cuh -- column-owner Householder QR of a triangular-over-full block pair.
//
// Every orthogonal step of the odd-even factorization (Section 3) is a QR factorization of two
// stacked blocks in which one block is already upper triangular:
//   step 1:  [Chat_j ; -B_{j+1}]       step 2:  [Rtilde_j ; D_j]       step 3: [Dtilde ; Chat]
// (the paper stacks steps 2 and 3 with the triangular block at the bottom; row order inside one
// QR does not change R^T R, and putting the triangle on top lets all three share one routine).
// With T (n x n, upper triangular) on top of a full p x n block M, the reflector that clears
// column kk touches row kk of T and all p rows of M only, so its support is p + 1 entries and
// the zero pattern of T below its diagonal is preserved.
//
// Reflector (LAPACK convention): alpha = T[kk][kk], x = M[:, kk], beta = -sign(alpha) *
// sqrt(alpha^2 + |x|^2) with sign(0) = +1, tau = (beta - alpha) / beta, v = [1 ; x / (alpha -
// beta)]; a zero x gives H = I.  Applying H to a column [a ; b] with gamma = 1 / (alpha - beta):
//   s = tau * (a_kk + gamma * x . b);   a_kk -= s;   b -= (s * gamma) x.
//
// Thread roles: each thread owns one column of the working matrix -- a factor column fcol of
// [T ; M], or one companion column given by (ctop, cbot): n entries in the top row block and p
// in the bottom one.  The owner of factor column kk+1 accumulates |x|^2 of its column while it
// applies reflector kk, so the only serial work per reflector is one sqrt and one divide.
#pragma once
#include <cuda_runtime.h>

namespace ks {

template <typename T>
__device__ __forceinline__ T hh_sqrt(T x);
template <>
__device__ __forceinline__ double hh_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float hh_sqrt<float>(float x) { return sqrtf(x); }

// All threads of the block must call this (it contains __syncthreads).  scal: 2n scratch.
template <typename T>
__device__ void tpqrt_columns(int n, int p, T* Tm, int ldT, T* Mm, int ldM, int fcol, T* ctop,
                              int ldct, T* cbot, int ldcb, T* scal) {
    // |x|^2 of factor column 0 (the only norm not produced by a previous update).
    if (fcol == 0) {
        T sg = T(0);
        for (int i = 0; i < p; ++i) {
            T x = Mm[i * ldM];
            sg = fma(x, x, sg);
        }
        scal[0] = sg;
    }
    __syncthreads();
    for (int kk = 0; kk < n; ++kk) {
        if (fcol == kk) {
            T alpha = Tm[kk * ldT + kk];
            T sigma = scal[2 * kk];
            T tau = T(0), gamma = T(0);
            if (sigma != T(0)) {
                T nrm = hh_sqrt<T>(fma(alpha, alpha, sigma));
                T beta = alpha >= T(0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                gamma = T(1) / (alpha - beta);
                Tm[kk * ldT + kk] = beta;
            }
            scal[2 * kk] = tau;
            scal[2 * kk + 1] = gamma;
        }
        __syncthreads();
        const T tau = scal[2 * kk], gamma = scal[2 * kk + 1];
        T* top = nullptr;
        T* bot = nullptr;
        int ldb = 0;
        if (fcol > kk) {
            top = Tm + kk * ldT + fcol;
            bot = Mm + fcol;
            ldb = ldM;
        } else if (fcol < 0 && ctop != nullptr) {
            top = ctop + kk * ldct;
            bot = cbot;
            ldb = ldcb;
        }
        const T* x = Mm + kk;
        if (top != nullptr) {
            const bool next = (fcol == kk + 1);
            if (tau != T(0)) {
                T s = T(0);
                for (int i = 0; i < p; ++i) s = fma(x[i * ldM], bot[i * ldb], s);
                s = tau * fma(gamma, s, *top);
                *top -= s;
                const T sg = -s * gamma;
                T nrm2 = T(0);
                for (int i = 0; i < p; ++i) {
                    T b = fma(sg, x[i * ldM], bot[i * ldb]);
                    bot[i * ldb] = b;
                    nrm2 = fma(b, b, nrm2);
                }
                if (next) scal[2 * kk + 2] = nrm2;
            } else if (next) {
                T nrm2 = T(0);
                for (int i = 0; i < p; ++i) nrm2 = fma(bot[i * ldb], bot[i * ldb], nrm2);
                scal[2 * kk + 2] = nrm2;
            }
        }
        __syncthreads();
    }
}

}  // namespace ks

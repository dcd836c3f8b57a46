// ks_med.cuh -- one level tile for medium state dimensions (compile-time N, 12 <= N <= 64),
// columns held in registers.
//
// Same steps as the column-owner kernel (Section 3: step 1 [Chat_j ; -B_s], step 2
// [Rtilde_j ; D_j], step 3 [Chat_s ; Dtilde_s], the tail of an odd level), same record layout
// (AosIO), but every thread keeps ITS column of the working matrix -- N entries of the triangle
// block row and N of the full block row -- in registers for the whole tile:
//   * the owner of factor column kk forms reflector kk from its own registers (its |x|^2 was
//     accumulated while it applied reflector kk-1) and publishes v = x / (alpha - beta) and tau
//     in shared memory;
//   * every thread with a later column reads v with 16-byte broadcast loads and updates its
//     registers: dot with four partial sums, then the axpy.
// Columns stay with their threads from step 1 to step 2 (factor columns keep Rtilde_j, step-1
// companions keep X_j as the tops of the right companions, the rhs keeps t_j); only Dtilde_s and
// s_s go through shared memory to step 3.  The three-block QR of the tail is done as two
// two-block passes, [Chat_s ; Dtilde_s] then [Chat'_s ; Z_e], which gives the same R factor and
// the same discarded residual.
#pragma once
#include "ks_internal.cuh"

namespace ks {
namespace med {

template <typename T>
__device__ __forceinline__ T msqrt(T x);
template <>
__device__ __forceinline__ double msqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float msqrt<float>(float x) { return sqrtf(x); }

// Shared memory of one tile (elements of T).
template <typename T, int N>
struct MedSmem {
    static constexpr int V = 0;                 // reflector tail, N entries (16-byte aligned)
    static constexpr int TAU = V + N;           // tau of the current reflector (+ pad)
    static constexpr int DT = TAU + 4;          // Dtilde_s, N x N, column c at DT + c*N
    static constexpr int SS = DT + N * N;       // s_s (N)
    static constexpr int ZE = SS + N;           // Z_e column block of the tail (N x N)
    static constexpr int ZR = ZE + N * N;       // z_e (N)
    static constexpr int TOTAL = ZR + N;
};

template <typename T, int N>
__device__ __forceinline__ T sumsq_(const T (&x)[N]) {
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i & 1) s1 = fma(x[i], x[i], s1); else s0 = fma(x[i], x[i], s0);
    }
    return s0 + s1;
}

// x[i] for a run-time i without indexing the register array (which would move it to memory).
template <typename T, int N>
__device__ __forceinline__ T pick_(const T (&x)[N], int i) {
    T v = x[0];
#pragma unroll
    for (int r = 1; r < N; ++r) v = (r == i) ? x[r] : v;
    return v;
}

// One Householder QR of [T ; M] over the threads of the block; thread roles:
//   fcol >= 0: owner of factor column fcol (top[] = its column of the triangle, bot[] = of M);
//   fcol <  0 and active: a companion column (top[], bot[]).
// norm2 (owner of factor column 0 only) must hold |bot|^2 on entry.
template <typename T, int N>
__device__ __forceinline__ void med_tpqrt(T (&top)[N], T (&bot)[N], int fcol, bool active, T* sm,
                                          T& norm2) {
    using S = MedSmem<T, N>;
    T* V = sm + S::V;
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
        if (fcol == kk) {
            const T alpha = top[kk];
            const T sigma = norm2;
            const T nrm = msqrt<T>(fma(alpha, alpha, sigma));
            const T beta = alpha >= T(0) ? -nrm : nrm;
            const T d = alpha - beta;
            const bool ok = sigma != T(0);
            const T r = T(1) / (beta * d);
            const T g = ok ? beta * r : T(0);
            sm[S::TAU] = ok ? -(d * d) * r : T(0);
            if (ok) top[kk] = beta;
#pragma unroll
            for (int i = 0; i < N; ++i) V[i] = bot[i] * g;
        }
        __syncthreads();
        if (active && (fcol < 0 || fcol > kk)) {
            const T tau = sm[S::TAU];
            T d0 = top[kk], d1 = T(0), d2 = T(0), d3 = T(0);
            if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
                for (int i = 0; i < N; i += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(V + i);
                    d0 = fma(q.x, bot[i], d0);
                    d1 = fma(q.y, bot[i + 1], d1);
                    d2 = fma(q.z, bot[i + 2], d2);
                    d3 = fma(q.w, bot[i + 3], d3);
                }
            } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
                for (int i = 0; i < N; i += 2) {
                    const double2 q = *reinterpret_cast<const double2*>(V + i);
                    if ((i & 2) == 0) {
                        d0 = fma(q.x, bot[i], d0);
                        d1 = fma(q.y, bot[i + 1], d1);
                    } else {
                        d2 = fma(q.x, bot[i], d2);
                        d3 = fma(q.y, bot[i + 1], d3);
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; ++i) d0 = fma(V[i], bot[i], d0);
            }
            const T sc = tau * ((d0 + d1) + (d2 + d3));
            top[kk] -= sc;
            if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
                for (int i = 0; i < N; i += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(V + i);
                    bot[i] = fma(-sc, q.x, bot[i]);
                    bot[i + 1] = fma(-sc, q.y, bot[i + 1]);
                    bot[i + 2] = fma(-sc, q.z, bot[i + 2]);
                    bot[i + 3] = fma(-sc, q.w, bot[i + 3]);
                }
            } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
                for (int i = 0; i < N; i += 2) {
                    const double2 q = *reinterpret_cast<const double2*>(V + i);
                    bot[i] = fma(-sc, q.x, bot[i]);
                    bot[i + 1] = fma(-sc, q.y, bot[i + 1]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; ++i) bot[i] = fma(-sc, V[i], bot[i]);
            }
            if (fcol == kk + 1) norm2 = sumsq_<T, N>(bot);
        }
        __syncthreads();
    }
}

// Tile t of a level (AosIO layout).  blockDim.x >= 3N+1.
template <typename T, int N>
__device__ void level_med_tile(const AosIO<T>& io, int64_t nc, int level, int64_t t,
                               double* __restrict__ resid, const double* __restrict__ cn2,
                               const double* __restrict__ cd2, unsigned long long* bad, T* sm) {
    using S = MedSmem<T, N>;
    const int tid = threadIdx.x;
    const int64_t nt = nc / 2;
    const int64_t j = 2 * t, s = j + 1;
    const bool triple = (nc & 1) && (t == nt - 1);
    const int64_t oj = ((j + 1) << level) - 1;
    // thread roles: [0, N) factor columns, [N, 2N) step-1 companions = step-2 right companions,
    // 2N the rhs, (2N, 3N] step-2 left companions.
    const bool is_fac = tid < N;
    const bool is_cmp = tid >= N && tid < 2 * N;
    const bool is_rhs = tid == 2 * N;
    const bool is_left = tid > 2 * N && tid <= 3 * N;
    const int c = is_fac ? tid : (is_cmp ? tid - N : (is_left ? tid - 2 * N - 1 : 0));
    T top[N], bot[N];
    T nrm2 = T(0);

    // ---- step 1: [Chat_j ; -B_s] with companions [0 ; D_s] and rhs [rC_j ; rE_s]
#pragma unroll
    for (int r = 0; r < N; ++r) {
        if (is_fac) { top[r] = io.C(j, r, c); bot[r] = io.E(s, r, c); }
        else if (is_cmp) { top[r] = T(0); bot[r] = io.E(s, r, N + c); }
        else if (is_rhs) { top[r] = io.RC(j, r); bot[r] = io.RE(s, r); }
        else { top[r] = T(0); bot[r] = T(0); }
    }
    if (tid == 0) nrm2 = sumsq_<T, N>(bot);
    med_tpqrt<T, N>(top, bot, is_fac ? c : -1, is_fac || is_cmp || is_rhs, sm, nrm2);
    // Dtilde_s (companion bottoms) and s_s (rhs bottom) -> shared memory for step 3
    if (is_cmp) {
#pragma unroll
        for (int r = 0; r < N; ++r) sm[S::DT + c * N + r] = bot[r];
    }
    if (is_rhs) {
#pragma unroll
        for (int r = 0; r < N; ++r) sm[S::SS + r] = bot[r];
    }
    // ---- step 2 (j >= 1): [Rtilde_j ; D_j], companions [0 ; -B_j] (left), [X_j ; 0] (right),
    //      rhs [t_j ; rE_j]
    if (j >= 1) {
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (is_fac) bot[r] = io.E(j, r, N + c);
            else if (is_cmp) bot[r] = T(0);
            else if (is_rhs) bot[r] = io.RE(j, r);
            else if (is_left) { top[r] = T(0); bot[r] = io.E(j, r, c); }
        }
        nrm2 = T(0);
        if (tid == 0) nrm2 = sumsq_<T, N>(bot);
        __syncthreads();   // step 1's stash writes vs the reuse of the reflector buffer
        med_tpqrt<T, N>(top, bot, is_fac ? c : -1, is_fac || is_cmp || is_rhs || is_left, sm, nrm2);
        // block row j of R and the reduced coupling row of new column t
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (is_fac) io.setR(t, oj, 0, r, c, r <= c ? top[r] : T(0));
            else if (is_left) { io.setR(t, oj, 1, r, c, top[r]); io.setE(t, r, c, bot[r]); }
            else if (is_cmp) { io.setR(t, oj, 2, r, c, top[r]); io.setE(t, r, N + c, bot[r]); }
            else if (is_rhs) { io.setY(t, oj, r, top[r]); io.setRE(t, r, bot[r]); }
        }
        if (is_fac && diag_is_singular<T>(pick_<T, N>(top, c), cn2[oj * N + c] + cd2[oj * N + c], N))
            flag_error(bad, ST_SINGULAR, oj);
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (is_fac) io.setR(t, oj, 0, r, c, r <= c ? top[r] : T(0));
            else if (is_cmp) { io.setR(t, oj, 2, r, c, top[r]); io.setR(t, oj, 1, r, c, T(0)); }
            else if (is_rhs) io.setY(t, oj, r, top[r]);
        }
        if (is_fac && diag_is_singular<T>(pick_<T, N>(top, c), cn2[oj * N + c] + cd2[oj * N + c], N))
            flag_error(bad, ST_SINGULAR, oj);
    }
    __syncthreads();
    // ---- tail (nc odd, last tile): step 2 of column e = nc-1 ([Chat_e ; D_e], companion
    //      [0 ; -B_e], rhs [rC_e ; rE_e]); its bottom rows Z_e, z_e join step 3.
    if (triple) {
        const int64_t e_ = j + 2;
        const int64_t oe = ((e_ + 1) << level) - 1;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (is_fac) { top[r] = io.C(e_, r, c); bot[r] = io.E(e_, r, N + c); }
            else if (is_cmp) { top[r] = T(0); bot[r] = io.E(e_, r, c); }
            else if (is_rhs) { top[r] = io.RC(e_, r); bot[r] = io.RE(e_, r); }
        }
        nrm2 = T(0);
        if (tid == 0) nrm2 = sumsq_<T, N>(bot);
        med_tpqrt<T, N>(top, bot, is_fac ? c : -1, is_fac || is_cmp || is_rhs, sm, nrm2);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (is_fac) io.setR(t + 1, oe, 0, r, c, r <= c ? top[r] : T(0));
            else if (is_cmp) {
                io.setR(t + 1, oe, 1, r, c, top[r]);
                io.setR(t + 1, oe, 2, r, c, T(0));
                sm[S::ZE + c * N + r] = bot[r];
            } else if (is_rhs) {
                io.setY(t + 1, oe, r, top[r]);
                sm[S::ZR + r] = bot[r];
            }
        }
        if (is_fac && diag_is_singular<T>(pick_<T, N>(top, c), cn2[oe * N + c] + cd2[oe * N + c], N))
            flag_error(bad, ST_SINGULAR, oe);
        __syncthreads();
    }
    // ---- step 3: [Chat_s ; Dtilde_s] (then [Chat'_s ; Z_e] for the tail) -> new column t
#pragma unroll
    for (int r = 0; r < N; ++r) {
        if (is_fac) { top[r] = io.C(s, r, c); bot[r] = sm[S::DT + c * N + r]; }
        else if (is_rhs) { top[r] = io.RC(s, r); bot[r] = sm[S::SS + r]; }
    }
    nrm2 = T(0);
    if (tid == 0) nrm2 = sumsq_<T, N>(bot);
    __syncthreads();
    med_tpqrt<T, N>(top, bot, is_fac ? c : -1, is_fac || is_rhs, sm, nrm2);
    double acc = 0.0;
    if (is_rhs) {
#pragma unroll
        for (int r = 0; r < N; ++r) acc = fma((double)bot[r], (double)bot[r], acc);
    }
    if (triple) {
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (is_fac) bot[r] = sm[S::ZE + c * N + r];
            else if (is_rhs) bot[r] = sm[S::ZR + r];
        }
        nrm2 = T(0);
        if (tid == 0) nrm2 = sumsq_<T, N>(bot);
        __syncthreads();
        med_tpqrt<T, N>(top, bot, is_fac ? c : -1, is_fac || is_rhs, sm, nrm2);
        if (is_rhs) {
#pragma unroll
            for (int r = 0; r < N; ++r) acc = fma((double)bot[r], (double)bot[r], acc);
        }
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        if (is_fac) io.setC(t, r, c, r <= c ? top[r] : T(0));
        else if (is_rhs) io.setRC(t, r, top[r]);
    }
    if (is_rhs) resid[oj] = acc;
    __syncthreads();
}

}  // namespace med
}  // namespace ks

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
            const T s2 = fma(alpha, alpha, sigma);
            const T nrm = msqrt<T>(s2);
            const T beta = alpha >= T(0) ? -nrm : nrm;
            const T d = alpha - beta;
            const bool ok = sigma != T(0) && s2 >= tiny_normal<T>();
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


// ------------------------------------------------------------------------------------------
// Whitening of one step (Section 2) for compile-time N, every m_i <= N.
//
//   1. Cholesky factors of K_i and C_i (FP64) in shared memory, right-looking with the column
//      scaling deferred: at pivot j the entries of both trailing triangles are spread evenly
//      over the block, one FMA each (A_rc -= A_rj A_cj / A_jj, the scaled column formed first;
//      two barriers per pivot), and at the end L_rc = A_rc / sqrt(A_cc) for all entries at once.
//      The FP64 pipe issues a warp instruction for the same time whatever its active lanes, so
//      packing the lanes is what sets this phase's cost.  C_i is padded to diag(C_i, I) when
//      m_i < N.
//   2. Forward substitution L^{-1} X, one right-hand column per thread held in registers
//      (right-looking, so the updates of a column are independent FMAs; the factor column is
//      read with 16-byte broadcast loads): threads [0, N] solve [G_i | o_i] with L_C, threads
//      [N+1, 3N+1] solve [-F_i | H_i | c_i] with L_K.
//   3. The whitened observation block [Chat_i | rC_i] (m_i x N, m_i <= N) is reduced to upper
//      triangular form by a Householder QR of its m_i rows (med_geqr), the N x N block padded
//      with zero rows.  With m_i <= N no row is discarded, so the residual part of step i is 0.
// Outputs are those of the column-owner whitening: level-0 record i ([Chat_i | rC_i]) and the
// coupling row of record i+1 ([-B_i | D_i | rE_i]), the column norms^2 of U A, the residual and,
// in refinement mode, the FP64 Cholesky factors.
template <typename T, int N>
struct MedWhitenSmem {
    static constexpr int LDA = N + 1;                           // odd leading dimension
    // FP64 part (elements of double)
    static constexpr int AK = 0;                                // K_i, then L_K (row-major)
    static constexpr int AC = AK + N * LDA;                     // diag(C_i, I), then L_C
    static constexpr int SC = AC + N * LDA;                     // 1 / sqrt(pivot), 2N
    static constexpr int NB = SC + 2 * N;                       // |B_i col|^2
    static constexpr int WB = NB + N;                           // scaled pivot columns, 2N
    static constexpr int IV = WB + 2 * N;                       // 1 / pivot (K, C) + pad
    static constexpr int DEND = IV + 2;
    static constexpr int TOFF = ((DEND * 8) + 15) & ~15;        // byte offset of the T part
    // working-precision part (elements of T)
    static constexpr int LK = 0;                                // L_K, column-major
    static constexpr int LC = LK + N * N;                       // L_C, column-major
    static constexpr int RK = LC + N * N;                       // 1 / diag(L_K)
    static constexpr int RC = RK + N;                           // 1 / diag(L_C)
    static constexpr int QR = RC + N;                           // reflector tail (N) + tau
    static constexpr int TAU = QR + N;
    static constexpr int TEND = TAU + 4;
    static constexpr int BYTES = TOFF + TEND * (int)sizeof(T);
};

// x[r] -= col[r] * xq for q < r < N (col 16-byte aligned; q a compile-time constant after
// unrolling), with 16-byte broadcast loads.
template <typename T, int N>
__device__ __forceinline__ void axpy_below_(T (&x)[N], const T* col, int q, T xq) {
    if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
        for (int r0 = 0; r0 < N; r0 += 4) {
            if (r0 + 3 > q) {
                const float4 v = *reinterpret_cast<const float4*>(col + r0);
                if (r0 > q) x[r0] = fma(-v.x, xq, x[r0]);
                if (r0 + 1 > q) x[r0 + 1] = fma(-v.y, xq, x[r0 + 1]);
                if (r0 + 2 > q) x[r0 + 2] = fma(-v.z, xq, x[r0 + 2]);
                x[r0 + 3] = fma(-v.w, xq, x[r0 + 3]);
            }
        }
    } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
        for (int r0 = 0; r0 < N; r0 += 2) {
            if (r0 + 1 > q) {
                const double2 v = *reinterpret_cast<const double2*>(col + r0);
                if (r0 > q) x[r0] = fma(-v.x, xq, x[r0]);
                x[r0 + 1] = fma(-v.y, xq, x[r0 + 1]);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r)
            if (r > q) x[r] = fma(-col[r], xq, x[r]);
    }
}

// sum_{r > q} V[r] x[r] with 16-byte broadcast loads (V 16-byte aligned), four partial sums.
template <typename T, int N>
__device__ __forceinline__ T dot_below_(const T (&x)[N], const T* V, int q) {
    T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
    if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
        for (int r0 = 0; r0 < N; r0 += 4) {
            if (r0 + 3 > q) {
                const float4 v = *reinterpret_cast<const float4*>(V + r0);
                if (r0 > q) d0 = fma(v.x, x[r0], d0);
                if (r0 + 1 > q) d1 = fma(v.y, x[r0 + 1], d1);
                if (r0 + 2 > q) d2 = fma(v.z, x[r0 + 2], d2);
                d3 = fma(v.w, x[r0 + 3], d3);
            }
        }
    } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
        for (int r0 = 0; r0 < N; r0 += 2) {
            if (r0 + 1 > q) {
                const double2 v = *reinterpret_cast<const double2*>(V + r0);
                if ((r0 & 2) == 0) {
                    if (r0 > q) d0 = fma(v.x, x[r0], d0);
                    d1 = fma(v.y, x[r0 + 1], d1);
                } else {
                    if (r0 > q) d2 = fma(v.x, x[r0], d2);
                    d3 = fma(v.y, x[r0 + 1], d3);
                }
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r)
            if (r > q) d0 = fma(V[r], x[r], d0);
    }
    return (d0 + d1) + (d2 + d3);
}

// In-place Householder QR of an m x N block (m <= N) held by columns: thread fcol >= 0 owns
// factor column fcol (rows in x[], rows >= m zero); active threads with fcol < 0 are companion
// columns the reflectors are applied to.  Reflector kk acts on rows kk..m-1; the owner of
// column kk+1 accumulates its next |tail|^2 while applying reflector kk (sig; the owner of
// column 0 passes it in).  On return rows r <= fcol of a factor column hold R (rows below the
// diagonal hold reflector tails) and companions hold Q^T applied to them.
template <typename T, int N>
__device__ __forceinline__ void med_geqr(T (&x)[N], int fcol, bool active, int m, T* V, T* tau_s,
                                         T& sig) {
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
        const bool live = kk < m;   // reflectors past m are identities; barriers stay uniform
        if (live && fcol == kk) {
            const T alpha = x[kk];
            const T s2 = fma(alpha, alpha, sig);
            const T nrm = msqrt<T>(s2);
            const T beta = alpha >= T(0) ? -nrm : nrm;
            const T d = alpha - beta;
            const bool ok = sig != T(0) && s2 >= tiny_normal<T>();
            const T r = T(1) / (beta * d);
            const T g = ok ? beta * r : T(0);
            *tau_s = ok ? -(d * d) * r : T(0);
            if (ok) x[kk] = beta;
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (i > kk) V[i] = x[i] * g;
        }
        __syncthreads();
        if (live && active && (fcol < 0 || fcol > kk)) {
            const T tau = *tau_s;
            const T sc = tau * (x[kk] + dot_below_<T, N>(x, V, kk));
            x[kk] -= sc;
            if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
                for (int r0 = 0; r0 < N; r0 += 4) {
                    if (r0 + 3 > kk) {
                        const float4 v = *reinterpret_cast<const float4*>(V + r0);
                        if (r0 > kk) x[r0] = fma(-sc, v.x, x[r0]);
                        if (r0 + 1 > kk) x[r0 + 1] = fma(-sc, v.y, x[r0 + 1]);
                        if (r0 + 2 > kk) x[r0 + 2] = fma(-sc, v.z, x[r0 + 2]);
                        x[r0 + 3] = fma(-sc, v.w, x[r0 + 3]);
                    }
                }
            } else {
                axpy_below_<T, N>(x, V, kk, sc);
            }
            if (fcol == kk + 1) {
                T s0 = T(0), s1 = T(0);
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    if (r > kk + 1) {
                        if (r & 1) s1 = fma(x[r], x[r], s1); else s0 = fma(x[r], x[r], s0);
                    }
                }
                sig = s0 + s1;
            }
        }
        __syncthreads();
    }
}

template <typename T, int N>
__device__ void whiten_med_step(const WhitenArgs& a, int64_t i, unsigned char* smem) {
    using S = MedWhitenSmem<T, N>;
    constexpr int LDA = S::LDA;
    double* dm = reinterpret_cast<double*>(smem);
    double* AK = dm + S::AK;
    double* AC = dm + S::AC;
    double* SC = dm + S::SC;
    double* nb = dm + S::NB;
    double* WB = dm + S::WB;
    double* IV = dm + S::IV;
    T* sm = reinterpret_cast<T*>(smem + S::TOFF);
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int nwarps = nth >> 5;
    constexpr int64_t NN2 = (int64_t)N * N;
    const int64_t CS = level_cs(N);
    T* out = reinterpret_cast<T*>(a.level0);
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
    const bool hasE = i + 1 < a.k;
    const double* Ci = a.C + ((a.ti & TI_C) ? 0 : co);
    const double* Gi = a.G + ((a.ti & TI_G) ? 0 : go) * N;

    // ---- phase 1: Cholesky factors of K_i and diag(C_i, I) in FP64 ----
    {
        const double* Ki = a.K + ti_step(a.ti, TI_K, i) * NN2;
        for (int e = tid; e < N * N; e += nth) {
            const int r = e / N, c = e - r * N;
            if (c <= r) {
                AK[r * LDA + c] = hasE ? Ki[e] : (r == c ? 1.0 : 0.0);
                AC[r * LDA + c] = (r < mi && c < mi) ? Ci[r * mi + c] : (r == c ? 1.0 : 0.0);
            }
        }
        if (tid == 0) {   // thread 0 wrote both leading entries above
            const double pk = AK[0], pc = AC[0];
            IV[0] = (pk > 0.0 && isfinite(pk)) ? 1.0 / pk : 1.0;
            IV[1] = (pc > 0.0 && isfinite(pc)) ? 1.0 / pc : 1.0;
        }
        __syncthreads();
        // Pivot j: W[c] = A_cj / A_jj (one multiply per entry), then every entry of the two
        // trailing triangles, spread evenly over the block, takes one FMA:
        // A_rc -= A_rj W[c].  The thread that updates A_{j+1,j+1} stores its reciprocal for the
        // next pivot.  (A non-positive pivot is replaced by 1 and flagged at the end.)
        for (int j = 0; j < N - 1; ++j) {
            const int t = N - 1 - j;
            if (tid < 2 * t) {
                const bool onC = tid >= t;
                const int r = j + 1 + (onC ? tid - t : tid);
                const double* A = onC ? AC : AK;
                WB[(onC ? N : 0) + r] = A[r * LDA + j] * IV[onC ? 1 : 0];
            }
            __syncthreads();
            const int tt = t * (t + 1) / 2;
            for (int e = tid; e < 2 * tt; e += nth) {
                const bool onC = e >= tt;
                const int e2 = onC ? e - tt : e;
                int rr = (int)((sqrtf(8.0f * (float)e2 + 1.0f) - 1.0f) * 0.5f);
                if ((rr + 1) * (rr + 2) / 2 <= e2) ++rr;
                if (rr * (rr + 1) / 2 > e2) --rr;
                const int r = j + 1 + rr, c = j + 1 + (e2 - rr * (rr + 1) / 2);
                double* A = onC ? AC : AK;
                const double v = fma(-A[r * LDA + j], WB[(onC ? N : 0) + c], A[r * LDA + c]);
                A[r * LDA + c] = v;
                if (r == j + 1 && c == j + 1) IV[onC ? 1 : 0] = (v > 0.0 && isfinite(v)) ? 1.0 / v : 1.0;
            }
            __syncthreads();
        }
        if (tid < 2 * N) {
            const bool onC = tid >= N;
            const int c = onC ? tid - N : tid;
            double* A = onC ? AC : AK;
            double d = A[c * LDA + c];
            if (!(d > 0.0) || !isfinite(d)) {
                flag_error(a.bad, ST_NOT_SPD, i);
                d = 1.0;
            }
            d = sqrt(d);
            const double inv = 1.0 / d;
            A[c * LDA + c] = d;
            SC[tid] = inv;
            sm[(onC ? S::RC : S::RK) + c] = (T)inv;
        }
        __syncthreads();
        for (int e = tid; e < 2 * N * N; e += nth) {
            const bool onC = e >= N * N;
            const int e2 = onC ? e - N * N : e;
            const int r = e2 / N, c = e2 - r * N;
            if (r > c) {
                double* A = onC ? AC : AK;
                const double v = A[r * LDA + c] * SC[(onC ? N : 0) + c];
                A[r * LDA + c] = v;
                sm[(onC ? S::LC : S::LK) + c * N + r] = (T)v;
            }
        }
        __syncthreads();
        if (hasE && a.LK != nullptr) {
            double* lk = a.LK + i * NN2;
            for (int e = tid; e < N * N; e += nth) {
                const int r = e / N, c = e - r * N;
                lk[e] = c <= r ? AK[r * LDA + c] : 0.0;
            }
        }
        if (a.LC != nullptr) {
            for (int e = tid; e < mi * mi; e += nth) {
                const int r = e / mi, c = e - r * mi;
                a.LC[co + e] = c <= r ? AC[r * LDA + c] : 0.0;
            }
        }
    }

    // ---- phase 2: forward substitution, one right-hand column per thread ----
    // roles: [0, N) column c of G_i; N: o_i; [N+1, 2N+1) column c of -F_i; [2N+1, 3N+1)
    //        column c of H_i; 3N+1: c_i.  Phase 3 then runs on threads [0, N] only.
    const bool onG = tid <= N;
    const bool onK = tid > N && tid <= 3 * N + 1;
    T x[N];
    {
        const double* Fi = a.F + ti_step(a.ti, TI_F, i) * NN2;
        const double* Hi = a.H + ti_step(a.ti, TI_H, i) * NN2;
        if (tid < N) {
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = r < mi ? (T)Gi[r * N + tid] : T(0);
        } else if (tid == N) {
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = r < mi ? (T)a.o[go + r] : T(0);
        } else if (tid < 2 * N + 1) {
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = hasE ? (T)(-Fi[r * N + tid - N - 1]) : T(0);
        } else if (tid < 3 * N + 1) {
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = hasE ? (T)Hi[r * N + tid - 2 * N - 1] : T(0);
        } else if (tid == 3 * N + 1) {
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = (hasE && a.c) ? (T)a.c[i * N + r] : T(0);
        } else {
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = T(0);
        }
        const bool solve = onG ? (mi > 0) : (onK && hasE);
        if (solve) {
            const T* Lt = sm + (onG ? S::LC : S::LK);
            const T* rdg = sm + (onG ? S::RC : S::RK);
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const T xq = x[q] * rdg[q];
                x[q] = xq;
                axpy_below_<T, N>(x, Lt + q * N, q, xq);
            }
        }
    }
    if (hasE && onK) {
        T* rec = out + (i + 1) * CS;
        if (tid < 3 * N + 1) {
            const int c2 = tid - N - 1;
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < N; ++r) {
                rec[NN2 + N + r * 2 * N + c2] = x[r];
                s = fma((double)x[r], (double)x[r], s);
            }
            if (c2 < N) nb[c2] = s;
            else a.cd2[(i + 1) * N + (c2 - N)] = s;
        } else {
#pragma unroll
            for (int r = 0; r < N; ++r) rec[3 * NN2 + N + r] = x[r];
        }
    }
    if (!hasE && tid > N && tid < 2 * N + 1) nb[tid - N - 1] = 0.0;
    if (i == 0 && tid < N) a.cd2[tid] = 0.0;

    // ---- phase 3: QR of the whitened observation block [Chat_i | rC_i] ----
    T sig = T(0);
    if (tid == 0) {
#pragma unroll
        for (int r = 1; r < N; ++r) sig = fma(x[r], x[r], sig);
    }
    __syncthreads();   // nb visible; the factors are no longer read
    med_geqr<T, N>(x, tid < N ? tid : -1, tid <= N, mi, sm + S::QR, sm + S::TAU, sig);
    T* rec = out + i * CS;
    if (tid < N) {
        double s = nb[tid];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const T v = (r <= tid && r < mi) ? x[r] : T(0);
            rec[r * N + tid] = v;
            s = fma((double)v, (double)v, s);
        }
        a.cn2[i * N + tid] = s;
    } else if (tid == N) {
#pragma unroll
        for (int r = 0; r < N; ++r) rec[NN2 + r] = r < mi ? x[r] : T(0);
        a.resid[i] = 0.0;
    }
    __syncthreads();
}

}  // namespace med
}  // namespace ks

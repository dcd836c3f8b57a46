// ks_small.cuh -- the whole smoother for small state dimensions (N <= 8, m_i <= N), one thread per
// independent unit of work (a step, a column pair, a block row), blocks held in registers.
//
// Why: on this GPU a warp instruction costs the FP64 pipe the same whether 1 or 32 lanes are
// active, and four warps per SM already hide its latency.  For small n the column-owner kernels
// leave most lanes idle, so here every lane owns a whole tile of a level instead and all 32
// lanes issue useful FMAs.  N is a compile-time constant so the blocks stay in registers.
//
// Layouts (element-major, "SoA", so that lane t touching record t makes coalesced accesses):
//  * level buffer with nc columns: two planes, even columns then odd columns; element e of
//    column j is at  plane[j&1][e * count(j&1) + j/2].  Record (CS elements):
//        [ Chat upper triangle (NT = N(N+1)/2) | rC (N) | E = [left | right] (N x 2N) | rE (N) ]
//  * R store, per level l: rows q = 0 .. rows_l-1 (the columns eliminated at l, original index
//    c = (2q+1) 2^l - 1), element e of row q at R[(k - (k>>l)) * RS + e * rows_l + q], with
//        [ Rd upper triangle (NT) | Rl (N x N) | Rr (N x N) | y (N) ],
//    rows_l = (k>>l) - (k>>(l+1)) and k - (k>>l) rows eliminated below level l.
//  * SelInv store: same per-level layout with [ Sl (N x N) | Sr (N x N) ] per row.
#pragma once
#include "ks_internal.cuh"

namespace ks {
namespace small {

template <int N>
struct Dims {
    static constexpr int NT = N * (N + 1) / 2;
    // level record
    static constexpr int OC = 0, ORC = NT, OE = NT + N, ORE = NT + N + 2 * N * N;
    static constexpr int CS = NT + 2 * N + 2 * N * N;
    // R record
    static constexpr int ORD = 0, ORL = NT, ORR = NT + N * N, OY = NT + 2 * N * N;
    static constexpr int RS = NT + 2 * N * N + N;
    static constexpr int SS = 2 * N * N;
};

__host__ __device__ constexpr int tri(int N, int r, int c) { return r * N - r * (r - 1) / 2 + (c - r); }


// Level buffer view (two planes).
template <typename T, int N>
struct LevelView {
    T* base;
    int64_t nE, nO;
    __device__ LevelView(T* b, int64_t nc) : base(b), nE((nc + 1) >> 1), nO(nc >> 1) {}
    __device__ __forceinline__ T* at(int64_t j, int e) const {
        return (j & 1) ? base + (int64_t)Dims<N>::CS * nE + (int64_t)e * nO + (j >> 1)
                       : base + (int64_t)e * nE + (j >> 1);
    }
};

// Per-level row store view (R or S).
template <typename T>
struct RowView {
    T* base;
    int64_t rows;
    __device__ RowView(T* store, int64_t k, int level, int rec)
        : base(store + (k - (k >> level)) * (int64_t)rec),
          rows((k >> level) - (k >> (level + 1))) {}
    __device__ __forceinline__ T* at(int64_t q, int e) const { return base + (int64_t)e * rows + q; }
};

// ---- Householder QR of [T ; M] in registers (T: N x N upper triangular, M: P x N) ----------
// Same reflector convention as the column-owner kernels: beta = -sign(alpha) |[alpha; x]|,
// tau = (beta - alpha) / beta, v = [1 ; x / (alpha - beta)], zero x (or alpha^2 + |x|^2 below
// the smallest normal number) -> no reflection.  The
// scaled tail x / (alpha - beta) is stored in place of x, so applying H to [a ; b] is
//   s = tau (a_kk + v . b),  a_kk -= s,  b -= s v.
template <typename T, int N, int P>
__device__ __forceinline__ void reg_factor(T (&Tm)[N][N], T (&M)[P][N], T (&tau)[N]) {
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
        const T alpha = Tm[kk][kk];
        T sigma = T(0);
#pragma unroll
        for (int i = 0; i < P; ++i) sigma = fma(M[i][kk], M[i][kk], sigma);
        const T s2 = fma(alpha, alpha, sigma);
        const T nrm = sqrt(s2);
        const T beta = alpha >= T(0) ? -nrm : nrm;
        const T d = alpha - beta;
        const bool ok = sigma != T(0) && s2 >= tiny_normal<T>();
        const T r = T(1) / (beta * d);   // one reciprocal gives both tau and 1 / (alpha - beta)
        const T g = ok ? beta * r : T(0);
        const T ta = ok ? -(d * d) * r : T(0);
        Tm[kk][kk] = ok ? beta : alpha;
        tau[kk] = ta;
#pragma unroll
        for (int i = 0; i < P; ++i) M[i][kk] *= g;
#pragma unroll
        for (int c = kk + 1; c < N; ++c) {
            T dot = Tm[kk][c];
#pragma unroll
            for (int i = 0; i < P; ++i) dot = fma(M[i][kk], M[i][c], dot);
            const T sc = ta * dot;
            Tm[kk][c] -= sc;
#pragma unroll
            for (int i = 0; i < P; ++i) M[i][c] = fma(-sc, M[i][kk], M[i][c]);
        }
    }
}

template <typename T, int N, int P>
__device__ __forceinline__ void reg_apply(const T (&M)[P][N], const T (&tau)[N], T (&top)[N],
                                          T (&bot)[P]) {
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
        T dot = top[kk];
#pragma unroll
        for (int i = 0; i < P; ++i) dot = fma(M[i][kk], bot[i], dot);
        const T sc = tau[kk] * dot;
        top[kk] -= sc;
#pragma unroll
        for (int i = 0; i < P; ++i) bot[i] = fma(-sc, M[i][kk], bot[i]);
    }
}

// Per-thread scratch in shared memory, element-major across the block (conflict-free).
template <typename T>
struct Stash {
    T* base;
    int nth, tid;
    __device__ __forceinline__ T& operator()(int e) const { return base[e * nth + tid]; }
};

template <typename T, int N>
__device__ __forceinline__ void load_upper(const LevelView<const T, N>& V, int64_t j, T (&A)[N][N]) {
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) A[r][c] = c >= r ? *V.at(j, Dims<N>::OC + tri(N, r, c)) : T(0);
}

// ---- whitening of one step, one thread --------------------------------------------------
template <typename T, int N>
__device__ void whiten_step(const WhitenArgs& a, int64_t i, T* out0) {
    using D = Dims<N>;
    const int64_t k = a.k;
    LevelView<T, N> O(out0, k);
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
    double cb2[N];
#pragma unroll
    for (int c = 0; c < N; ++c) cb2[c] = 0.0;
    if (i + 1 < k) {
        // K_i = L L^T in FP64.
        const double* Ki = a.K + ti_step(a.ti, TI_K, i) * N * N;
        double L[N][N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c) L[r][c] = Ki[r * N + c];
        bool bad = false;
        double linv[N];   // 1 / diag(L), reused by the solves (an FP64 divide is costly)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double dj = L[j][j];
#pragma unroll
            for (int p = 0; p < j; ++p) dj = fma(-L[j][p], L[j][p], dj);
            bad |= !(dj > 0.0) || !isfinite(dj);
            dj = (dj > 0.0 && isfinite(dj)) ? sqrt(dj) : 1.0;
            L[j][j] = dj;
            const double inv = 1.0 / dj;
            linv[j] = inv;
#pragma unroll
            for (int r = j + 1; r < N; ++r) {
                double s = L[r][j];
#pragma unroll
                for (int p = 0; p < j; ++p) s = fma(-L[r][p], L[j][p], s);
                L[r][j] = s * inv;
            }
        }
        if (bad) flag_error(a.bad, ST_NOT_SPD, i);
        if (a.LK) {
            double* lk = a.LK + i * N * N;
#pragma unroll
            for (int r = 0; r < N; ++r)
#pragma unroll
                for (int c = 0; c < N; ++c) lk[r * N + c] = c <= r ? L[r][c] : 0.0;
        }
        T Lt[N][N], dinv[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            dinv[r] = (T)linv[r];
#pragma unroll
            for (int c = 0; c < r; ++c) Lt[r][c] = (T)L[r][c];
        }
        // [-B | D | rE] = L^{-1} [-F | H | c], column by column (FP64 mode in double, refine
        // mode in FP32 from the FP64 factor).
        const double* Fi = a.F + ti_step(a.ti, TI_F, i) * N * N;
        const double* Hi = a.H + ti_step(a.ti, TI_H, i) * N * N;
        double cd2[N];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
#pragma unroll
            for (int c = 0; c < N; ++c) {
                T x[N];
#pragma unroll
                for (int r = 0; r < N; ++r) x[r] = half == 0 ? (T)(-Fi[r * N + c]) : (T)Hi[r * N + c];
                double s2 = 0.0;
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    T s = x[r];
#pragma unroll
                    for (int p = 0; p < r; ++p) s = fma(-Lt[r][p], x[p], s);
                    x[r] = s * dinv[r];
                    s2 = fma((double)x[r], (double)x[r], s2);
                    *O.at(i + 1, D::OE + r * 2 * N + half * N + c) = x[r];
                }
                if (half == 0) cb2[c] = s2; else cd2[c] = s2;
            }
        }
        {
            T x[N];
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = a.c ? (T)a.c[i * N + r] : T(0);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                T s = x[r];
#pragma unroll
                for (int p = 0; p < r; ++p) s = fma(-Lt[r][p], x[p], s);
                x[r] = s * dinv[r];
                *O.at(i + 1, D::ORE + r) = x[r];
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c) a.cd2[(i + 1) * N + c] = cd2[c];
    }
    if (i == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) a.cd2[c] = 0.0;
    }
    // Observation: C_i = Lo Lo^T (padded with the identity beyond m_i), [Chat | rC] = Lo^{-1}[G | o],
    // then QR of [0 ; Chat] -> N x N upper triangle.
    T Tm[N][N], top[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        top[r] = T(0);
#pragma unroll
        for (int c = 0; c < N; ++c) Tm[r][c] = T(0);
    }
    double res = 0.0;
    if (mi > 0) {
        const double* Ci = a.C + ((a.ti & TI_C) ? 0 : co);
        double Lo[N][N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c)
                Lo[r][c] = (r < mi) ? Ci[r * mi + c] : (r == c ? 1.0 : 0.0);
        bool bad = false;
        double oinv[N];   // 1 / diag(Lo), reused by the solve
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double dj = Lo[j][j];
#pragma unroll
            for (int p = 0; p < j; ++p) dj = fma(-Lo[j][p], Lo[j][p], dj);
            bad |= !(dj > 0.0) || !isfinite(dj);
            dj = (dj > 0.0 && isfinite(dj)) ? sqrt(dj) : 1.0;
            Lo[j][j] = dj;
            const double inv = 1.0 / dj;
            oinv[j] = inv;
#pragma unroll
            for (int r = j + 1; r < N; ++r) {
                double s = Lo[r][j];
#pragma unroll
                for (int p = 0; p < j; ++p) s = fma(-Lo[r][p], Lo[j][p], s);
                Lo[r][j] = s * inv;
            }
        }
        if (bad) flag_error(a.bad, ST_NOT_SPD, i);
        if (a.LC) {
#pragma unroll
            for (int r = 0; r < N; ++r)
#pragma unroll
                for (int c = 0; c < N; ++c)
                    if (r < mi && c < mi) a.LC[co + r * mi + c] = c <= r ? Lo[r][c] : 0.0;
        }
        T M[N][N], ob[N];
        const double* Gi = a.G + ((a.ti & TI_G) ? 0 : go) * N;
        const double* oi = a.o + go;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            ob[r] = r < mi ? (T)oi[r] : T(0);
#pragma unroll
            for (int c = 0; c < N; ++c) M[r][c] = r < mi ? (T)Gi[r * N + c] : T(0);
        }
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const T dv = (T)oinv[r];
#pragma unroll
            for (int p = 0; p < r; ++p) {
                const T l = (T)Lo[r][p];
#pragma unroll
                for (int c = 0; c < N; ++c) M[r][c] = fma(-l, M[p][c], M[r][c]);
                ob[r] = fma(-l, ob[p], ob[r]);
            }
#pragma unroll
            for (int c = 0; c < N; ++c) M[r][c] *= dv;
            ob[r] *= dv;
        }
        T tau[N];
        reg_factor<T, N, N>(Tm, M, tau);
        reg_apply<T, N, N>(M, tau, top, ob);
#pragma unroll
        for (int r = 0; r < N; ++r) res = fma((double)ob[r], (double)ob[r], res);
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
#pragma unroll
        for (int c = r; c < N; ++c) *O.at(i, D::OC + tri(N, r, c)) = Tm[r][c];
        *O.at(i, D::ORC + r) = top[r];
    }
#pragma unroll
    for (int c = 0; c < N; ++c) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r <= c; ++r) s = fma((double)Tm[r][c], (double)Tm[r][c], s);
        a.cn2[i * N + c] = s + cb2[c];
    }
    a.resid[i] = res;
}

// ---- one tile of a level, one thread ----------------------------------------------------
template <typename T, int N>
__device__ __forceinline__ void check_diag(const T (&Tm)[N][N], const double* cn2, const double* cd2,
                                           int64_t c, unsigned long long* bad) {
#pragma unroll
    for (int r = 0; r < N; ++r)
        if (diag_is_singular<T>(Tm[r][r], cn2[c * N + r] + cd2[c * N + r], N)) {
            flag_error(bad, ST_SINGULAR, c);
            break;
        }
}

// Stash slots of one level tile (per thread, element-major in shared memory).
template <int N>
struct TileSlots {
    static constexpr int X = 0, DT = N * N, TJ = 2 * N * N, SS = 2 * N * N + N,
                         RT = 2 * N * N + 2 * N, COUNT = 2 * N * N + 2 * N + N * (N + 1) / 2;
};

// Tail of a level with an odd number of columns: step 2 of the last column e (no right
// neighbour) and step 3 of its left neighbour s with the extra block row Z_e.  Only the last
// tile of such a level runs it; kept out of line so it does not raise the register budget of
// the common path.
template <typename T, int N>
__device__ __noinline__ void level_tail(const LevelView<const T, N> I, LevelView<T, N> O,
                                        const RowView<T> RV, int level, int64_t t, int64_t oj,
                                        double* resid, const double* cn2, const double* cd2,
                                        unsigned long long* bad, const Stash<T> st) {
    using D = Dims<N>;
    using S = TileSlots<N>;
    const int64_t s = 2 * t + 1, e_ = 2 * t + 2;
    const int64_t oe = ((e_ + 1) << level) - 1;
    {
        T Te[N][N], Me[N][N], tau[N];
        load_upper<T, N>(I, e_, Te);
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) Me[r][c] = *I.at(e_, D::OE + r * 2 * N + N + c);
        reg_factor<T, N, N>(Te, Me, tau);
        check_diag<T, N>(Te, cn2, cd2, oe, bad);
        for (int r = 0; r < N; ++r)
            for (int c = r; c < N; ++c) *RV.at(t + 1, D::ORD + tri(N, r, c)) = Te[r][c];
        for (int c = 0; c < N; ++c) {
            T top[N], bot[N];
            for (int r = 0; r < N; ++r) {
                top[r] = T(0);
                bot[r] = *I.at(e_, D::OE + r * 2 * N + c);
            }
            reg_apply<T, N, N>(Me, tau, top, bot);
            for (int r = 0; r < N; ++r) {
                *RV.at(t + 1, D::ORL + r * N + c) = top[r];
                *RV.at(t + 1, D::ORR + r * N + c) = T(0);
                st(S::X + r * N + c) = bot[r];   // Z_e
            }
        }
        T top[N], bot[N];
        for (int r = 0; r < N; ++r) {
            top[r] = *I.at(e_, D::ORC + r);
            bot[r] = *I.at(e_, D::ORE + r);
        }
        reg_apply<T, N, N>(Me, tau, top, bot);
        for (int r = 0; r < N; ++r) {
            *RV.at(t + 1, D::OY + r) = top[r];
            st(S::TJ + r) = bot[r];   // z_e
        }
    }
    T T3[N][N], M3[2 * N][N], tau3[N];
    load_upper<T, N>(I, s, T3);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            M3[r][c] = st(S::DT + r * N + c);
            M3[N + r][c] = st(S::X + r * N + c);
        }
    reg_factor<T, N, 2 * N>(T3, M3, tau3);
    T top3[N], bot3[2 * N];
    for (int r = 0; r < N; ++r) {
        top3[r] = *I.at(s, D::ORC + r);
        bot3[r] = st(S::SS + r);
        bot3[N + r] = st(S::TJ + r);
    }
    reg_apply<T, N, 2 * N>(M3, tau3, top3, bot3);
    double acc = 0.0;
    for (int r = 0; r < 2 * N; ++r) acc = fma((double)bot3[r], (double)bot3[r], acc);
    resid[oj] = acc;
    for (int r = 0; r < N; ++r) {
        for (int c = r; c < N; ++c) *O.at(t, D::OC + tri(N, r, c)) = T3[r][c];
        *O.at(t, D::ORC + r) = top3[r];
    }
}

template <typename T, int N>
__device__ void level_tile(int64_t nc, int level, int64_t k, int64_t t, const T* in, T* out,
                           T* R, double* resid, const double* cn2, const double* cd2,
                           unsigned long long* bad, const Stash<T>& st) {
    using D = Dims<N>;
    using S = TileSlots<N>;
    const LevelView<const T, N> I(in, nc);
    LevelView<T, N> O(out, nc >> 1);
    const RowView<T> RV(R, k, level, D::RS);
    const int64_t nt = nc >> 1;
    const int64_t j = 2 * t, s = j + 1;
    const bool triple = (nc & 1) && (t == nt - 1);
    const int64_t oj = ((j + 1) << level) - 1;

    // ---- step 1: [Chat_j ; -B_s], companions [0 ; D_s] and rhs [rC_j ; rE_s]
    {
        T T1[N][N], M1[N][N], tau[N];
        load_upper<T, N>(I, j, T1);
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) M1[r][c] = *I.at(s, D::OE + r * 2 * N + c);
        reg_factor<T, N, N>(T1, M1, tau);
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = r; c < N; ++c) st(S::RT + tri(N, r, c)) = T1[r][c];   // Rtilde_j
#pragma unroll 1
        for (int c = 0; c < N; ++c) {
            T top[N], bot[N];
#pragma unroll
            for (int r = 0; r < N; ++r) {
                top[r] = T(0);
                bot[r] = *I.at(s, D::OE + r * 2 * N + N + c);
            }
            reg_apply<T, N, N>(M1, tau, top, bot);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                st(S::X + r * N + c) = top[r];    // X_j
                st(S::DT + r * N + c) = bot[r];   // Dtilde_s
            }
        }
        T top[N], bot[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            top[r] = *I.at(j, D::ORC + r);
            bot[r] = *I.at(s, D::ORE + r);
        }
        reg_apply<T, N, N>(M1, tau, top, bot);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            st(S::TJ + r) = top[r];   // t_j
            st(S::SS + r) = bot[r];   // s_s
        }
    }
    // ---- step 2 (j >= 1): [Rtilde_j ; D_j], companions [0 ; -B_j], [X_j ; 0], rhs [t_j ; rE_j]
    if (j >= 1) {
        T T2[N][N], M2[N][N], tau[N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                T2[r][c] = c >= r ? st(S::RT + tri(N, r, c)) : T(0);
                M2[r][c] = *I.at(j, D::OE + r * 2 * N + N + c);
            }
        reg_factor<T, N, N>(T2, M2, tau);
        check_diag<T, N>(T2, cn2, cd2, oj, bad);
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = r; c < N; ++c) *RV.at(t, D::ORD + tri(N, r, c)) = T2[r][c];
#pragma unroll 1
        for (int c = 0; c < N; ++c) {  // left companion -> Rl (top), Z (bottom)
            T top[N], bot[N];
#pragma unroll
            for (int r = 0; r < N; ++r) {
                top[r] = T(0);
                bot[r] = *I.at(j, D::OE + r * 2 * N + c);
            }
            reg_apply<T, N, N>(M2, tau, top, bot);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                *RV.at(t, D::ORL + r * N + c) = top[r];
                *O.at(t, D::OE + r * 2 * N + c) = bot[r];
            }
        }
#pragma unroll 1
        for (int c = 0; c < N; ++c) {  // right companion -> Rr (top), Xtilde (bottom)
            T top[N], bot[N];
#pragma unroll
            for (int r = 0; r < N; ++r) {
                top[r] = st(S::X + r * N + c);
                bot[r] = T(0);
            }
            reg_apply<T, N, N>(M2, tau, top, bot);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                *RV.at(t, D::ORR + r * N + c) = top[r];
                *O.at(t, D::OE + r * 2 * N + N + c) = bot[r];
            }
        }
        T top[N], bot[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            top[r] = st(S::TJ + r);
            bot[r] = *I.at(j, D::ORE + r);
        }
        reg_apply<T, N, N>(M2, tau, top, bot);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            *RV.at(t, D::OY + r) = top[r];
            *O.at(t, D::ORE + r) = bot[r];
        }
    } else {
        T T2[N][N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) T2[r][c] = c >= r ? st(S::RT + tri(N, r, c)) : T(0);
        check_diag<T, N>(T2, cn2, cd2, oj, bad);
#pragma unroll
        for (int r = 0; r < N; ++r) {
#pragma unroll
            for (int c = r; c < N; ++c) *RV.at(t, D::ORD + tri(N, r, c)) = T2[r][c];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                *RV.at(t, D::ORL + r * N + c) = T(0);
                *RV.at(t, D::ORR + r * N + c) = st(S::X + r * N + c);
            }
            *RV.at(t, D::OY + r) = st(S::TJ + r);
        }
    }
    if (triple) {
        level_tail<T, N>(I, O, RV, level, t, oj, resid, cn2, cd2, bad, st);
        return;
    }
    // ---- step 3: [Chat_s ; Dtilde_s] -> reduced diagonal block of new column t
    {
        T T3[N][N], M3[N][N], tau3[N];
        load_upper<T, N>(I, s, T3);
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) M3[r][c] = st(S::DT + r * N + c);
        reg_factor<T, N, N>(T3, M3, tau3);
        T top3[N], bot3[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            top3[r] = *I.at(s, D::ORC + r);
            bot3[r] = st(S::SS + r);
        }
        reg_apply<T, N, N>(M3, tau3, top3, bot3);
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < N; ++r) acc = fma((double)bot3[r], (double)bot3[r], acc);
        resid[oj] = acc;
#pragma unroll
        for (int r = 0; r < N; ++r) {
#pragma unroll
            for (int c = r; c < N; ++c) *O.at(t, D::OC + tri(N, r, c)) = T3[r][c];
            *O.at(t, D::ORC + r) = top3[r];
        }
    }
}

// ---- back substitution for one row --------------------------------------------------------
// u_c = Rd^{-1} (rhs - Rl u_a - Rr u_b), rhs = y (w == nullptr) or w_c.
template <typename TR, int N>
__device__ void backsub_row(int64_t k, int level, int64_t q, const TR* R, const double* w,
                            double* u) {
    using D = Dims<N>;
    const RowView<const TR> RV(R, k, level, D::RS);
    const int64_t c = ((2 * q + 1) << level) - 1;
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    double r[N];
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = w ? w[c * N + i] : (double)*RV.at(q, D::OY + i);
    if (a >= 0) {
        double ua[N];
#pragma unroll
        for (int p = 0; p < N; ++p) ua[p] = u[a * N + p];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int p = 0; p < N; ++p) r[i] = fma(-(double)*RV.at(q, D::ORL + i * N + p), ua[p], r[i]);
    }
    if (b < k) {
        double ub[N];
#pragma unroll
        for (int p = 0; p < N; ++p) ub[p] = u[b * N + p];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int p = 0; p < N; ++p) r[i] = fma(-(double)*RV.at(q, D::ORR + i * N + p), ub[p], r[i]);
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        double s = r[i];
#pragma unroll
        for (int p = i + 1; p < N; ++p) s = fma(-(double)*RV.at(q, D::ORD + tri(N, i, p)), r[p], s);
        r[i] = s / (double)*RV.at(q, D::ORD + tri(N, i, i));
    }
#pragma unroll
    for (int i = 0; i < N; ++i) u[c * N + i] = r[i];
}

// ---- odd-even SelInv for one row (Algorithm 2 body) ---------------------------------------
// With Ri = Rd^{-1}, Ta = Ri Rl, Tb = Ri Rr:
//   Sl = S_{c,a} = -(Ta S_aa + Tb S_ba),  Sr = S_{c,b} = -(Ta S_ab + Tb S_bb),
//   S_cc = Ri Ri^T - Sl Ta^T - Sr Tb^T     (upper triangle computed, mirrored on output).
// Ta, Tb live in the shared-memory stash (the FP64 pipe, not operand bandwidth, is the limit).
template <int N>
struct SelinvSlots {
    static constexpr int TA = 0, TB = N * N, RI = 2 * N * N, COUNT = 3 * N * N;
};

template <typename T, int N>
__device__ void selinv_row(int64_t k, int level, int64_t q, const T* R, T* Sx, double* Sd,
                           unsigned long long* bad, const Stash<T>& st) {
    using D = Dims<N>;
    using SL = SelinvSlots<N>;
    const RowView<const T> RV(R, k, level, D::RS);
    const RowView<T> SV(Sx, k, level, D::SS);
    const int64_t c = ((2 * q + 1) << level) - 1;
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    const bool ha = a >= 0, hb = b < k;
    // Ri = Rd^{-1} (upper triangular), one column at a time, into the stash.
    {
        T Rd[N][N];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j2 = 0; j2 < N; ++j2) Rd[i][j2] = j2 >= i ? *RV.at(q, D::ORD + tri(N, i, j2)) : T(0);
#pragma unroll
        for (int col = 0; col < N; ++col) {
            T x[N];
#pragma unroll
            for (int i = N - 1; i >= 0; --i) {
                if (i > col) {
                    x[i] = T(0);
                    continue;
                }
                T s = (i == col) ? T(1) : T(0);
#pragma unroll
                for (int p = i + 1; p <= col; ++p) s = fma(-Rd[i][p], x[p], s);
                x[i] = s / Rd[i][i];
            }
#pragma unroll
            for (int i = 0; i < N; ++i) st(SL::RI + i * N + col) = x[i];
        }
    }
    // Ta = Ri Rl, Tb = Ri Rr -> stash (zero blocks for absent neighbours).
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        const bool has = blk == 0 ? ha : hb;
        const int off = blk == 0 ? D::ORL : D::ORR;
        const int so = blk == 0 ? SL::TA : SL::TB;
#pragma unroll 1
        for (int col = 0; col < N; ++col) {
            T x[N];
#pragma unroll
            for (int p = 0; p < N; ++p) x[p] = has ? *RV.at(q, off + p * N + col) : T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T s = T(0);
#pragma unroll
                for (int p = i; p < N; ++p) s = fma(st(SL::RI + i * N + p), x[p], s);
                st(so + i * N + col) = s;
            }
        }
    }
    // S_cc = Ri Ri^T (upper triangle).
    T S[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j2 = i; j2 < N; ++j2) {
            T s = T(0);
#pragma unroll
            for (int p = j2; p < N; ++p) s = fma(st(SL::RI + i * N + p), st(SL::RI + j2 * N + p), s);
            S[i][j2] = s;
        }
    // Cross block S_ab of the two neighbours, held by whichever of them is eliminated at
    // level+1 (they are adjacent there).
    const T* sab = nullptr;
    bool sab_t = false;
    const RowView<const T> SV1(Sx, k, level + 1, D::SS);
    if (ha && hb) {
        if (ctz64(a + 1) == level + 1) {
            sab = SV1.at((a + 1) >> (level + 2), N * N);   // Sr_a = S_{a,b}
        } else {
            sab = SV1.at((b + 1) >> (level + 2), 0);       // Sl_b = S_{b,a}
            sab_t = true;
        }
    }
    // Columns of Sl = -(Ta S_aa + Tb S_ba) and Sr = -(Ta S_ab + Tb S_bb); S_cc -= Sl Ta^T + Sr Tb^T.
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        const bool has = blk == 0 ? ha : hb;
        if (has) {
#pragma unroll 1
            for (int col = 0; col < N; ++col) {
                T x1[N], x2[N];
#pragma unroll
                for (int p = 0; p < N; ++p) {
                    T vab = T(0);   // S_ab[p][col] for blk 1, S_ba[p][col] = S_ab[col][p] for blk 0
                    if (sab) {
                        const bool rowmajor = (blk == 1) != sab_t;
                        vab = rowmajor ? *(sab + (int64_t)(p * N + col) * SV1.rows)
                                       : *(sab + (int64_t)(col * N + p) * SV1.rows);
                    }
                    if (blk == 0) {
                        x1[p] = (T)Sd[a * N * N + p * N + col];
                        x2[p] = vab;
                    } else {
                        x1[p] = vab;
                        x2[p] = (T)Sd[b * N * N + p * N + col];
                    }
                }
                T y[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T s = T(0);
#pragma unroll
                    for (int p = 0; p < N; ++p) {
                        s = fma(st(SL::TA + i * N + p), x1[p], s);
                        s = fma(st(SL::TB + i * N + p), x2[p], s);
                    }
                    y[i] = -s;
                    *SV.at(q, blk * N * N + i * N + col) = y[i];
                }
                const int so = blk == 0 ? SL::TA : SL::TB;
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int j2 = i; j2 < N; ++j2) S[i][j2] = fma(-y[i], st(so + j2 * N + col), S[i][j2]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < N * N; ++e) *SV.at(q, blk * N * N + e) = T(0);
        }
    }
    bool neg = false;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        neg |= !(S[i][i] > T(0));
#pragma unroll
        for (int j2 = 0; j2 < N; ++j2) Sd[c * N * N + i * N + j2] = (double)(j2 >= i ? S[i][j2] : S[j2][i]);
    }
    if (neg) flag_error(bad, ST_SINGULAR, c);
}

// ---- refinement (KS_FP32_REFINE) -----------------------------------------------------------
// Mixed-precision iterative refinement: only the residuals -- differences of nearly equal
// quantities -- are formed in FP64; the correction solve R^T R d = g runs in FP32 with the
// FP32 R, like the factorization itself.

// q_i = K_i^{-1} e_i with e_i = F_i u_i + c_i - H_i u_{i+1} (e in FP64, the solve in FP32).
template <int N>
__device__ void refine_q_step(const RefineArgs& a, int64_t i, float* q) {
    const double* F = a.F + ti_step(a.ti, TI_F, i) * N * N;
    const double* H = a.H + ti_step(a.ti, TI_H, i) * N * N;
    const double* Lk = a.LK + i * N * N;
    double u0[N], u1[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        u0[p] = a.u[i * N + p];
        u1[p] = a.u[(i + 1) * N + p];
    }
    float e[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        double s = a.c ? a.c[i * N + r] : 0.0;
#pragma unroll
        for (int p = 0; p < N; ++p) s = fma(F[r * N + p], u0[p], s);
#pragma unroll
        for (int p = 0; p < N; ++p) s = fma(-H[r * N + p], u1[p], s);
        e[r] = (float)s;
    }
    float L[N][N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) L[r][c] = (float)Lk[r * N + c];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        float s = e[r];
#pragma unroll
        for (int p = 0; p < r; ++p) s = fmaf(-L[r][p], e[p], s);
        e[r] = s / L[r][r];
    }
#pragma unroll
    for (int r = N - 1; r >= 0; --r) {
        float s = e[r];
#pragma unroll
        for (int p = r + 1; p < N; ++p) s = fmaf(-L[p][r], e[p], s);
        e[r] = s / L[r][r];
    }
#pragma unroll
    for (int r = 0; r < N; ++r) q[i * N + r] = e[r];
}

// g_c = H_{c-1}^T q_{c-1} - F_c^T q_c + G_c^T C_c^{-1} (o_c - G_c u_c); o - G u in FP64.
template <int N>
__device__ void refine_g_col(const RefineArgs& a, int64_t c, const float* q, float* g) {
    float acc[N];
#pragma unroll
    for (int r = 0; r < N; ++r) acc[r] = 0.f;
    if (c >= 1) {
        const double* H = a.H + ti_step(a.ti, TI_H, c - 1) * N * N;
        float qv[N];
#pragma unroll
        for (int p = 0; p < N; ++p) qv[p] = q[(c - 1) * N + p];
#pragma unroll
        for (int p = 0; p < N; ++p)
#pragma unroll
            for (int r = 0; r < N; ++r) acc[r] = fmaf((float)H[p * N + r], qv[p], acc[r]);
    }
    if (c + 1 < a.k) {
        const double* F = a.F + ti_step(a.ti, TI_F, c) * N * N;
        float qv[N];
#pragma unroll
        for (int p = 0; p < N; ++p) qv[p] = q[c * N + p];
#pragma unroll
        for (int p = 0; p < N; ++p)
#pragma unroll
            for (int r = 0; r < N; ++r) acc[r] = fmaf(-(float)F[p * N + r], qv[p], acc[r]);
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
        const double* G = a.G + ((a.ti & TI_G) ? 0 : go) * N;
        const double* Lc = a.LC + co;
        double uc[N];
#pragma unroll
        for (int p = 0; p < N; ++p) uc[p] = a.u[c * N + p];
        float v[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r < mi) {
                double s = a.o[go + r];
#pragma unroll
                for (int p = 0; p < N; ++p) s = fma(-G[r * N + p], uc[p], s);
                v[r] = (float)s;
            } else {
                v[r] = 0.f;
            }
        }
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r < mi) {
                float s = v[r];
#pragma unroll
                for (int p = 0; p < r; ++p) s = fmaf(-(float)Lc[r * mi + p], v[p], s);
                v[r] = s / (float)Lc[r * mi + r];
            }
        }
#pragma unroll
        for (int r = N - 1; r >= 0; --r) {
            if (r < mi) {
                float s = v[r];
#pragma unroll
                for (int p = r + 1; p < N; ++p)
                    if (p < mi) s = fmaf(-(float)Lc[p * mi + r], v[p], s);
                v[r] = s / (float)Lc[r * mi + r];
            }
        }
#pragma unroll
        for (int p = 0; p < N; ++p)
            if (p < mi)
#pragma unroll
                for (int r = 0; r < N; ++r) acc[r] = fmaf((float)G[p * N + r], v[p], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < N; ++r) g[c * N + r] = acc[r];
}

// R^T w = g at one level for one alive column: pull the blocks of the rows eliminated at
// level-1 that touch column c, then, if c is eliminated at this level, solve Rd^T w_c = g_c.
template <typename TR, typename TV, int N>
__device__ void rt_solve_col(int64_t k, int level, int64_t jj, const TR* R, TV* g, TV* w) {
    using D = Dims<N>;
    const int64_t c = ((jj + 1) << level) - 1;
    TV r[N];
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = g[c * N + i];
    if (level >= 1) {
        const RowView<const TR> RP(R, k, level - 1, D::RS);
        const int64_t h = 1LL << (level - 1);
        if (c - h >= 0) {  // row c-h: its right block Rr sits in column c
            const int64_t qq = (c - h + 1) >> level;
            TV wr[N];
#pragma unroll
            for (int p = 0; p < N; ++p) wr[p] = w[(c - h) * N + p];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int p = 0; p < N; ++p) r[i] = fma(-(TV)*RP.at(qq, D::ORR + p * N + i), wr[p], r[i]);
        }
        if (c + h < k) {  // row c+h: its left block Rl sits in column c
            const int64_t qq = (c + h + 1) >> level;
            TV wr[N];
#pragma unroll
            for (int p = 0; p < N; ++p) wr[p] = w[(c + h) * N + p];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int p = 0; p < N; ++p) r[i] = fma(-(TV)*RP.at(qq, D::ORL + p * N + i), wr[p], r[i]);
        }
    }
    if (ctz64(c + 1) == level) {
        const RowView<const TR> RV(R, k, level, D::RS);
        const int64_t q = (c + 1) >> (level + 1);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            TV s = r[i];
#pragma unroll
            for (int p = 0; p < i; ++p) s = fma(-(TV)*RV.at(q, D::ORD + tri(N, p, i)), r[p], s);
            r[i] = s / (TV)*RV.at(q, D::ORD + tri(N, i, i));
        }
#pragma unroll
        for (int i = 0; i < N; ++i) w[c * N + i] = r[i];
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) g[c * N + i] = r[i];
    }
}

// R d = w for one row, all in FP32 (the correction of the refinement).
template <int N>
__device__ void backsub_row_f(int64_t k, int level, int64_t q, const float* R, const float* w,
                              float* d) {
    using D = Dims<N>;
    const RowView<const float> RV(R, k, level, D::RS);
    const int64_t c = ((2 * q + 1) << level) - 1;
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    float r[N];
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = w[c * N + i];
    if (a >= 0) {
        float ua[N];
#pragma unroll
        for (int p = 0; p < N; ++p) ua[p] = d[a * N + p];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int p = 0; p < N; ++p) r[i] = fmaf(-*RV.at(q, D::ORL + i * N + p), ua[p], r[i]);
    }
    if (b < k) {
        float ub[N];
#pragma unroll
        for (int p = 0; p < N; ++p) ub[p] = d[b * N + p];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int p = 0; p < N; ++p) r[i] = fmaf(-*RV.at(q, D::ORR + i * N + p), ub[p], r[i]);
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        float s = r[i];
#pragma unroll
        for (int p = i + 1; p < N; ++p) s = fmaf(-*RV.at(q, D::ORD + tri(N, i, p)), r[p], s);
        r[i] = s / *RV.at(q, D::ORD + tri(N, i, i));
    }
#pragma unroll
    for (int i = 0; i < N; ++i) d[c * N + i] = r[i];
}

}  // namespace small
}  // namespace ks

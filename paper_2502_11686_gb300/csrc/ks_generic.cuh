// ks_generic.cuh -- the column-owner (one thread block per unit) kernels' per-unit bodies, shared
// by the single-problem launches and the batched launches.
#pragma once
#include "ks_householder.cuh"
#include "ks_internal.cuh"

namespace ks {

// One step of the column-owner whitening: every thread of the block must call it.  The two
// Cholesky factorizations run in FP64; the triangular solves and the QR of the observation block
// run in the working precision T (the smem slots are sized for doubles either way).
template <typename T>
__device__ void whiten_cta_step(const WhitenArgs& a, int64_t i, double* sm) {
    const int n = a.n;
    const WhitenLayout L = whiten_layout(n, a.mmax);
    double* KC = sm + L.kc;
    T* W = reinterpret_cast<T*>(sm + L.w);
    double* OC = sm + L.oc;
    T* Gm = reinterpret_cast<T*>(sm + L.g);
    T* Tt = reinterpret_cast<T*>(sm + L.t);
    T* scal = reinterpret_cast<T*>(sm + L.scal);
    T* KT = reinterpret_cast<T*>(sm + L.kt);
    T* OT = reinterpret_cast<T*>(sm + L.ot);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t CS = level_cs(n);
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
    const bool hasE = (i + 1 < a.k);
    // ---- loads (coalesced over the row-major source blocks) ----
    if (hasE) {
        const double* Ki = a.K + ti_step(a.ti, TI_K, i) * (int64_t)n * n;
        const double* Fi = a.F + ti_step(a.ti, TI_F, i) * (int64_t)n * n;
        const double* Hi = a.H + ti_step(a.ti, TI_H, i) * (int64_t)n * n;
        for (int e = tid; e < n * n; e += nth) {
            int r = e / n, c = e - r * n;
            KC[r * L.ldk + c] = Ki[e];
            W[r * L.ldw + c] = (T)(-Fi[e]);
            W[r * L.ldw + n + c] = (T)Hi[e];
        }
        for (int r = tid; r < n; r += nth) W[r * L.ldw + 2 * n] = a.c ? (T)a.c[i * n + r] : T(0);
    }
    for (int e = tid; e < mi * mi; e += nth) {
        int r = e / mi, c = e - r * mi;
        OC[r * L.ldo + c] = a.C[((a.ti & TI_C) ? 0 : co) + e];
    }
    for (int e = tid; e < mi * n; e += nth) {
        int r = e / n, c = e - r * n;
        Gm[r * L.ldg + c] = (T)a.G[((a.ti & TI_G) ? 0 : go) * n + e];
    }
    for (int r = tid; r < mi; r += nth) Gm[r * L.ldg + n] = (T)a.o[go + r];
    for (int e = tid; e < n * L.ldt; e += nth) Tt[e] = T(0);
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

    // ---- working-precision copies of the factors ----
    for (int e = tid; e < nK * nK; e += nth) {
        int r = e / nK, c = e - r * nK;
        KT[r * L.ldk + c] = (T)KC[r * L.ldk + c];
    }
    for (int e = tid; e < mi * mi; e += nth) {
        int r = e / mi, c = e - r * mi;
        OT[r * L.ldo + c] = (T)OC[r * L.ldo + c];
    }
    __syncthreads();

    // ---- forward substitution: W <- L_K^{-1} W (2n+1 columns), Gm <- L_C^{-1} Gm ----
    {
        T* B = nullptr;
        const T* Lf = nullptr;
        int ldb = 0, ldl = 0, dim2 = 0;
        if (tid < 2 * n + 1) {
            if (hasE) { B = W + tid; ldb = L.ldw; Lf = KT; ldl = L.ldk; dim2 = n; }
        } else if (tid < 3 * n + 2) {
            if (mi > 0) { B = Gm + (tid - 2 * n - 1); ldb = L.ldg; Lf = OT; ldl = L.ldo; dim2 = mi; }
        }
        if (B != nullptr) {
            for (int r = 0; r < dim2; ++r) {
                T s = B[r * ldb];
                for (int q = 0; q < r; ++q) s = fma(-Lf[r * ldl + q], B[q * ldb], s);
                B[r * ldb] = s / Lf[r * ldl + r];
            }
        }
    }
    __syncthreads();

    // ---- reduce the observation block: QR of [0 (n x n) ; Chat (mi x n)] with its rhs ----
    {
        const int fcol = (tid < n) ? tid : -1;
        T* ctop = (tid == n) ? (Tt + n) : nullptr;
        T* cbot = (tid == n) ? (Gm + n) : nullptr;
        tpqrt_columns<T>(n, mi, Tt, L.ldt, Gm, L.ldg, fcol, ctop, L.ldt, cbot, L.ldg, scal);
    }

    // ---- stores ----
    T* rec = out + i * CS;
    for (int e = tid; e < n * n; e += nth) {
        int r = e / n, c = e - r * n;
        rec[e] = c >= r ? Tt[r * L.ldt + c] : T(0);
    }
    for (int r = tid; r < n; r += nth) rec[n * n + r] = Tt[r * L.ldt + n];
    if (hasE) {
        T* nxt = out + (i + 1) * CS + (int64_t)n * n + n;
        for (int e = tid; e < 2 * n * n; e += nth) {
            int r = e / (2 * n), c = e - r * 2 * n;
            nxt[e] = W[r * L.ldw + c];
        }
        for (int r = tid; r < n; r += nth) nxt[2 * n * n + r] = W[r * L.ldw + 2 * n];
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
        for (int r = 0; r < mi; ++r) s = fma((double)Gm[r * L.ldg + n], (double)Gm[r * L.ldg + n], s);
        a.resid[i] = s;
    }
    // Column norms^2 of U A for state i (Chat_i and B_i) and state i+1 (D_i).
    for (int col = tid; col < n; col += nth) {
        double sc = 0.0, sb = 0.0, sd = 0.0;
        for (int r = 0; r <= col; ++r) sc = fma((double)Tt[r * L.ldt + col], (double)Tt[r * L.ldt + col], sc);
        if (hasE) {
            for (int r = 0; r < n; ++r) {
                sb = fma((double)W[r * L.ldw + col], (double)W[r * L.ldw + col], sb);
                sd = fma((double)W[r * L.ldw + n + col], (double)W[r * L.ldw + n + col], sd);
            }
            a.cd2[(i + 1) * n + col] = sd;
        }
        a.cn2[i * n + col] = sc + sb;
        if (i == 0) a.cd2[col] = 0.0;
    }
    __syncthreads();
}

// Tile t of one level, column-owner scheme: every thread of the block must call it.
template <typename T, typename IO>
__device__ void level_cta_tile(const IO& io, int n, int64_t nc, int level, int64_t t,
                               double* __restrict__ resid, const double* __restrict__ cn2,
                               const double* __restrict__ cd2, unsigned long long* bad, T* sm) {
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

// The last alive column becomes the base block row: Rd = Chat (already triangular), y = rC.
template <typename T>
__device__ void base_block(int n, int64_t k, int L, const T* __restrict__ in, T* __restrict__ R,
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

}  // namespace ks

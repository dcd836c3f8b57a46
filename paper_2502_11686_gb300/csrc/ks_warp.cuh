// ks_warp.cuh -- warp-per-unit vector solves of the column-owner and large-state paths: back
// substitution (Section 3.1), the R^T solve and the residual/gradient steps of the refinement.
// Lane l holds rows l, l+32, ..., l+32(NR-1) of the unit's vector, so NR = ceil(n/32) rows per
// lane (NR = 2 for n <= 64, 4 for n <= 128).
#pragma once
#include "ks_internal.cuh"

namespace ks {

// The register of rows[] that holds row i (i >> 5), selected without a run-time index.
template <int NR, typename TV>
__device__ __forceinline__ TV row_of(const TV (&r)[NR], int i) {
    TV v = r[0];
#pragma unroll
    for (int s = 1; s < NR; ++s) v = ((i >> 5) == s) ? r[s] : v;
    return v;
}

// Back substitution of block row q at `level`: u_c = Rd^{-1}(rhs - Rl u_a - Rr u_b).
// rhs = y from the R store (w == nullptr) or w_c.  Vectors of type TV, output of type TO.
template <int NR, typename TR, typename TV, typename TO>
__device__ void backsub_warp(int n, int64_t k, int level, int64_t q, const TR* __restrict__ R,
                             const TV* __restrict__ w, TO* __restrict__ u) {
    const int lane = threadIdx.x & 31;
    const int64_t c = ((2 * q + 1) << level) - 1;
    if (c >= k) return;
    const int nn = n * n;
    const TR* Rc = R + c * rstore_rs(n);
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    TV r[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const int i = lane + 32 * s;
        r[s] = TV(0);
        if (i < n) r[s] = w ? w[c * n + i] : (TV)Rc[3 * nn + i];
    }
    if (a >= 0) {
        for (int p = 0; p < n; ++p) {
            const TV up = (TV)u[a * n + p];
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int i = lane + 32 * s;
                if (i < n) r[s] = fma(-(TV)Rc[nn + i * n + p], up, r[s]);
            }
        }
    }
    if (b < k) {
        for (int p = 0; p < n; ++p) {
            const TV up = (TV)u[b * n + p];
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int i = lane + 32 * s;
                if (i < n) r[s] = fma(-(TV)Rc[2 * nn + i * n + p], up, r[s]);
            }
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        TV x = TV(0);
        if ((i & 31) == lane) x = row_of<NR, TV>(r, i) / (TV)Rc[i * n + i];
        x = __shfl_sync(0xffffffffu, x, i & 31);
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int ii = lane + 32 * s;
            if (ii < i) r[s] = fma(-(TV)Rc[ii * n + i], x, r[s]);
            if (ii == i) r[s] = x;
        }
    }
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const int i = lane + 32 * s;
        if (i < n) u[c * n + i] = (TO)r[s];
    }
}

// R^T w = g at `level` for alive column j (pull the two rows eliminated at level-1 that touch
// it, then solve with Rd^T if it is eliminated here).
template <int NR, typename TR, typename TV>
__device__ void rt_solve_warp(int n, int64_t k, int level, int64_t j, const TR* __restrict__ R,
                              TV* __restrict__ g, TV* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    if (j >= (k >> level)) return;
    const int64_t c = ((j + 1) << level) - 1;
    const int nn = n * n;
    const int64_t RS = rstore_rs(n);
    TV r[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const int i = lane + 32 * s;
        r[s] = i < n ? g[c * n + i] : TV(0);
    }
    if (level >= 1) {
        const int64_t h = 1LL << (level - 1);
        if (c - h >= 0) {
            const TR* Rr = R + (c - h) * RS + 2 * nn;
            const TV* wr = w + (c - h) * n;
            for (int p = 0; p < n; ++p) {
                const TV wp = wr[p];
#pragma unroll
                for (int s = 0; s < NR; ++s) {
                    const int i = lane + 32 * s;
                    if (i < n) r[s] = fma(-(TV)Rr[p * n + i], wp, r[s]);
                }
            }
        }
        if (c + h < k) {
            const TR* Rl = R + (c + h) * RS + nn;
            const TV* wr = w + (c + h) * n;
            for (int p = 0; p < n; ++p) {
                const TV wp = wr[p];
#pragma unroll
                for (int s = 0; s < NR; ++s) {
                    const int i = lane + 32 * s;
                    if (i < n) r[s] = fma(-(TV)Rl[p * n + i], wp, r[s]);
                }
            }
        }
    }
    if (ctz64(c + 1) == level) {
        const TR* Rd = R + c * RS;
        for (int i = 0; i < n; ++i) {
            TV x = TV(0);
            if ((i & 31) == lane) x = row_of<NR, TV>(r, i) / (TV)Rd[i * n + i];
            x = __shfl_sync(0xffffffffu, x, i & 31);
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int ii = lane + 32 * s;
                if (ii > i && ii < n) r[s] = fma(-(TV)Rd[i * n + ii], x, r[s]);
                if (ii == i) r[s] = x;
            }
        }
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int i = lane + 32 * s;
            if (i < n) w[c * n + i] = r[s];
        }
    } else {
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int i = lane + 32 * s;
            if (i < n) g[c * n + i] = r[s];
        }
    }
}

// Warp-cooperative solves with an FP64 lower-triangular factor L (ld = dim), in type TV:
// forward (L y = x) then backward (L^T z = y); x given per lane in rows lane + 32 s.
template <int NR, typename TV>
__device__ void llt_solve_warp(int dim, const double* __restrict__ Lf, TV (&r)[NR]) {
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < dim; ++i) {
        TV x = TV(0);
        if ((i & 31) == lane) x = row_of<NR, TV>(r, i) / (TV)Lf[i * dim + i];
        x = __shfl_sync(0xffffffffu, x, i & 31);
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int ii = lane + 32 * s;
            if (ii > i && ii < dim) r[s] = fma(-(TV)Lf[ii * dim + i], x, r[s]);
            if (ii == i) r[s] = x;
        }
    }
    for (int i = dim - 1; i >= 0; --i) {
        TV x = TV(0);
        if ((i & 31) == lane) x = row_of<NR, TV>(r, i) / (TV)Lf[i * dim + i];
        x = __shfl_sync(0xffffffffu, x, i & 31);
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int ii = lane + 32 * s;
            if (ii < i) r[s] = fma(-(TV)Lf[i * dim + ii], x, r[s]);
            if (ii == i) r[s] = x;
        }
    }
}

// q_i = K_i^{-1} (F_i u_i + c_i - H_i u_{i+1}): the residual in FP64, the solve in TV.
template <int NR, typename TV>
__device__ void refine_q_warp(const RefineArgs& a, int64_t i, TV* __restrict__ q) {
    if (i + 1 >= a.k) return;
    const int lane = threadIdx.x & 31, n = a.n, nn = n * n;
    const double* F = a.F + ti_step(a.ti, TI_F, i) * nn;
    const double* H = a.H + ti_step(a.ti, TI_H, i) * nn;
    double e[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const int ii = lane + 32 * s;
        e[s] = (ii < n && a.c) ? a.c[i * n + ii] : 0.0;
    }
    for (int p = 0; p < n; ++p) {
        const double u0 = a.u[i * n + p], u1 = a.u[(i + 1) * n + p];
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int ii = lane + 32 * s;
            if (ii < n) e[s] = fma(-H[ii * n + p], u1, fma(F[ii * n + p], u0, e[s]));
        }
    }
    TV r[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) r[s] = (TV)e[s];
    llt_solve_warp<NR, TV>(n, a.LK + i * nn, r);
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const int ii = lane + 32 * s;
        if (ii < n) q[i * n + ii] = r[s];
    }
}

// g_c = H_{c-1}^T q_{c-1} - F_c^T q_c + G_c^T C_c^{-1} (o_c - G_c u_c), o - G u in FP64.
template <int NR, typename TV>
__device__ void refine_g_warp(const RefineArgs& a, int64_t c, const TV* __restrict__ q,
                              TV* __restrict__ g) {
    if (c >= a.k) return;
    const int lane = threadIdx.x & 31, n = a.n, nn = n * n;
    TV gv[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) gv[s] = TV(0);
    if (c >= 1) {
        const double* H = a.H + ti_step(a.ti, TI_H, c - 1) * nn;
        for (int p = 0; p < n; ++p) {
            const TV qp = q[(c - 1) * n + p];
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int ii = lane + 32 * s;
                if (ii < n) gv[s] = fma((TV)H[p * n + ii], qp, gv[s]);
            }
        }
    }
    if (c + 1 < a.k) {
        const double* F = a.F + ti_step(a.ti, TI_F, c) * nn;
        for (int p = 0; p < n; ++p) {
            const TV qp = q[c * n + p];
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int ii = lane + 32 * s;
                if (ii < n) gv[s] = fma(-(TV)F[p * n + ii], qp, gv[s]);
            }
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
        double v[NR];
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            const int ii = lane + 32 * s;
            v[s] = ii < mi ? a.o[go + ii] : 0.0;
        }
        for (int p = 0; p < n; ++p) {
            const double up = a.u[c * n + p];
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int ii = lane + 32 * s;
                if (ii < mi) v[s] = fma(-G[ii * n + p], up, v[s]);
            }
        }
        TV r[NR];
#pragma unroll
        for (int s = 0; s < NR; ++s) r[s] = (TV)v[s];
        llt_solve_warp<NR, TV>(mi, a.LC + co, r);
        for (int p = 0; p < mi; ++p) {
            const TV vp = __shfl_sync(0xffffffffu, row_of<NR, TV>(r, p), p & 31);
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const int ii = lane + 32 * s;
                if (ii < n) gv[s] = fma((TV)G[p * n + ii], vp, gv[s]);
            }
        }
    }
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const int ii = lane + 32 * s;
        if (ii < n) g[c * n + ii] = gv[s];
    }
}

}  // namespace ks

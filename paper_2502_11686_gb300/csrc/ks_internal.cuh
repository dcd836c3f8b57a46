// ks_internal.cuh -- layouts, status words and launch wrappers shared by the libks.so sources.
//
// Data layout in HBM (all row-major, T = double in KS_FP64 mode, float in KS_FP32_REFINE):
//
//  * Level buffer: one record of CS = 3n^2 + 2n elements per alive block column j of the
//    current level (Section 3: every alive column carries one "C" block and one coupling row to
//    its left neighbour, so the level problem has the structure of the original one):
//        [ Chat_j (n x n, upper triangular) | rC_j (n) | E_j (n x 2n) | rE_j (n) ]
//    E_j = [ left | right ] is the whitened coupling block row between columns j-1 and j with
//    the coefficients of u_{j-1} (the paper's -B_j) and of u_j (the paper's D_j); E_0 is unused.
//  * R store: one record of RS = 3n^2 + n elements per ORIGINAL state index c (each block column
//    is eliminated exactly once, at level l(c) = ctz(c+1)):
//        [ Rd_c (n x n upper) | Rl_c (n x n, at column c - 2^l) | Rr_c (n x n, at c + 2^l) | y_c (n) ]
//    Rl exists iff c >= 2^l, Rr iff c + 2^l < k; absent blocks are stored as zeros.
//  * SelInv store: Sl_c, Sr_c (n x n each, record 2n^2) = S_{c, c-2^l}, S_{c, c+2^l}; the
//    diagonal blocks S_cc go straight to the covariance output [k][n][n].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ks {

enum { ST_ARG = 1, ST_NOT_SPD = 2, ST_SINGULAR = 3, ST_TIMEOUT = 6, ST_NONFINITE = 8, ST_NCODES = 9 };

// Order in which a call reports its device error words (the first one set wins), and the
// message of each.  A non-finite input, or a timed-out wait (which leaves the rest of that
// launch's results undefined), makes R look singular as well, so both are reported first.
constexpr int status_order[] = {ST_NOT_SPD, ST_NONFINITE, ST_TIMEOUT, ST_SINGULAR, ST_ARG};
inline const char* status_message(int code) {
    switch (code) {
        case ST_NOT_SPD: return "a covariance matrix is not SPD at step";
        case ST_NONFINITE: return "a non-finite input value (NaN or Inf) in the equations of state";
        case ST_SINGULAR: return "singular diagonal block of R at state";
        case ST_TIMEOUT: return "a bounded device wait gave up (tensor-core completion) at";
        case ST_ARG: return "bad argument detected on device at";
        default: return "device error at";
    }
}

// Device error words: bad[code] = smallest failing index seen (ULLONG_MAX = none).
__device__ __forceinline__ void flag_error(unsigned long long* bad, int code, long long idx) {
    atomicMin(bad + code, (unsigned long long)idx);
}

__host__ __device__ __forceinline__ int odd_ld(int x) { return x | 1; }
// Trailing zero bits of x > 0: the level at which column x - 1 is eliminated.
__device__ __forceinline__ int ctz64(int64_t x) { return __ffsll((long long)x) - 1; }
__host__ __device__ __forceinline__ int64_t level_cs(int n) { return 3LL * n * n + 2LL * n; }
__host__ __device__ __forceinline__ int64_t rstore_rs(int n) { return 3LL * n * n + n; }

// Shared-memory layout of one level tile (elements of T).  Leading dimensions are odd so that
// a warp reading a column (stride ld) hits distinct banks.
struct TileLayout {
    int n, ld2, ldf, ld3;
    int top2, bot2, bf, top3, bot3, scal, total;
};

__host__ __device__ inline TileLayout tile_layout(int n) {
    TileLayout L;
    L.n = n;
    L.ld2 = odd_ld(3 * n + 1);
    L.ldf = odd_ld(n);
    L.ld3 = odd_ld(n + 1);
    L.top2 = 0;
    L.bot2 = L.top2 + n * L.ld2;
    L.bf = L.bot2 + n * L.ld2;
    L.top3 = L.bf + n * L.ldf;
    L.bot3 = L.top3 + n * L.ld3;
    L.scal = L.bot3 + 2 * n * L.ld3;
    L.total = L.scal + 2 * n;
    return L;
}

// Shared-memory layout of the whitening of one step (elements of double).
struct WhitenLayout {
    int n, m, ldk, ldw, ldo, ldg, ldt;
    int kc, w, oc, g, t, top, scal, kt, ot, total;
};

__host__ __device__ inline WhitenLayout whiten_layout(int n, int m) {
    WhitenLayout L;
    L.n = n;
    L.m = m;
    L.ldk = odd_ld(n);          // K_i, then its Cholesky factor
    L.ldw = odd_ld(2 * n + 1);  // [F_i | H_i | c_i], then L_K^{-1} of it
    L.ldo = odd_ld(m > 0 ? m : 1);
    L.ldg = odd_ld(n + 1);      // [G_i | o_i], then L_C^{-1} of it
    L.ldt = odd_ld(n + 1);      // [Chat_i | rC_i] (n rows)
    L.kc = 0;
    L.w = L.kc + n * L.ldk;
    L.oc = L.w + n * L.ldw;
    L.g = L.oc + m * L.ldo;
    L.t = L.g + m * L.ldg;
    L.top = L.t;  // alias: the rhs column of the top block is column n of t
    L.scal = L.t + n * L.ldt;
    L.kt = L.scal + 2 * n;       // working-precision copies of the two Cholesky factors
    L.ot = L.kt + n * L.ldk;
    L.total = L.ot + m * L.ldo;
    return L;
}

// Shared-memory layout of one SelInv column (elements of T).
struct SelinvLayout {
    int n, ldr, ldt, lds;
    int rd, tt, ri, sii, sl, total;
};

__host__ __device__ inline SelinvLayout selinv_layout(int n) {
    SelinvLayout L;
    L.n = n;
    L.ldr = odd_ld(n);
    L.ldt = odd_ld(2 * n);
    L.lds = odd_ld(2 * n);
    L.rd = 0;
    L.tt = L.rd + n * L.ldr;     // [Ta | Tb] = Rd^{-1} [Rl | Rr]
    L.ri = L.tt + n * L.ldt;     // Rd^{-1}
    L.sii = L.ri + n * L.ldr;    // S_II (2n x 2n)
    L.sl = L.sii + 2 * n * L.lds;  // [Sl | Sr]
    L.total = L.sl + n * L.ldt;
    return L;
}

// ---------------------------------------------------------------------------------------------
// Record access policies of the column-owner kernels.  AosIO: the generic layout (records per
// column, R / S rows by original state index).  SoaIO: the element-major layout of the
// small-state path (even / odd column planes, packed upper triangles, R / S rows per level), so
// that the column-owner kernels can also run the top levels of a small-state problem, where a
// level has too few tiles for one thread per tile.
template <typename T>
struct AosIO {
    int n;
    int64_t CS, RS;
    const T* in;
    T* out;
    T* R;
    __device__ AosIO(int n_, int64_t, int, int64_t, const T* i, T* o, T* r)
        : n(n_), CS(level_cs(n_)), RS(rstore_rs(n_)), in(i), out(o), R(r) {}
    __device__ T C(int64_t j, int r, int c) const { return in[j * CS + r * n + c]; }
    __device__ T RC(int64_t j, int r) const { return in[j * CS + n * n + r]; }
    __device__ T E(int64_t j, int r, int c2) const { return in[j * CS + n * n + n + r * 2 * n + c2]; }
    __device__ T RE(int64_t j, int r) const { return in[j * CS + 3 * n * n + n + r]; }
    __device__ void setC(int64_t t, int r, int c, T v) const { out[t * CS + r * n + c] = c >= r ? v : T(0); }
    __device__ void setRC(int64_t t, int r, T v) const { out[t * CS + n * n + r] = v; }
    __device__ void setE(int64_t t, int r, int c2, T v) const { out[t * CS + n * n + n + r * 2 * n + c2] = v; }
    __device__ void setRE(int64_t t, int r, T v) const { out[t * CS + 3 * n * n + n + r] = v; }
    // Block row of the column with level row q and original index oc; part 0/1/2 = Rd/Rl/Rr.
    __device__ void setR(int64_t, int64_t oc, int part, int r, int c, T v) const {
        R[oc * RS + part * n * n + r * n + c] = v;
    }
    __device__ void setY(int64_t, int64_t oc, int r, T v) const { R[oc * RS + 3 * n * n + r] = v; }
};

template <typename T>
struct SoaIO {
    int n, nt, CS, RS;
    int64_t nE, nO, nE2, nO2, rows, roff;
    const T* in;
    T* out;
    T* R;
    __device__ SoaIO(int n_, int64_t nc, int level, int64_t k, const T* i, T* o, T* r)
        : n(n_), nt(n_ * (n_ + 1) / 2), in(i), out(o), R(r) {
        CS = nt + 2 * n + 2 * n * n;
        RS = nt + 2 * n * n + n;
        nE = (nc + 1) >> 1;
        nO = nc >> 1;
        nE2 = ((nc >> 1) + 1) >> 1;
        nO2 = (nc >> 1) >> 1;
        rows = (k >> level) - (k >> (level + 1));
        roff = (k - (k >> level)) * (int64_t)RS;
    }
    __device__ int tri(int r, int c) const { return r * n - r * (r - 1) / 2 + (c - r); }
    __device__ T ie(int64_t j, int e) const {
        return (j & 1) ? in[(int64_t)CS * nE + (int64_t)e * nO + (j >> 1)] : in[(int64_t)e * nE + (j >> 1)];
    }
    __device__ T* oe(int64_t t, int e) const {
        return (t & 1) ? out + (int64_t)CS * nE2 + (int64_t)e * nO2 + (t >> 1) : out + (int64_t)e * nE2 + (t >> 1);
    }
    __device__ T C(int64_t j, int r, int c) const { return c >= r ? ie(j, tri(r, c)) : T(0); }
    __device__ T RC(int64_t j, int r) const { return ie(j, nt + r); }
    __device__ T E(int64_t j, int r, int c2) const { return ie(j, nt + n + r * 2 * n + c2); }
    __device__ T RE(int64_t j, int r) const { return ie(j, nt + n + 2 * n * n + r); }
    __device__ void setC(int64_t t, int r, int c, T v) const { if (c >= r) *oe(t, tri(r, c)) = v; }
    __device__ void setRC(int64_t t, int r, T v) const { *oe(t, nt + r) = v; }
    __device__ void setE(int64_t t, int r, int c2, T v) const { *oe(t, nt + n + r * 2 * n + c2) = v; }
    __device__ void setRE(int64_t t, int r, T v) const { *oe(t, nt + n + 2 * n * n + r) = v; }
    __device__ void setR(int64_t q, int64_t, int part, int r, int c, T v) const {
        if (part == 0) {
            if (c >= r) R[roff + (int64_t)tri(r, c) * rows + q] = v;
        } else {
            R[roff + (int64_t)(nt + (part - 1) * n * n + r * n + c) * rows + q] = v;
        }
    }
    __device__ void setY(int64_t q, int64_t, int r, T v) const {
        R[roff + (int64_t)(nt + 2 * n * n + r) * rows + q] = v;
    }
};

// ---------------------------------------------------------------------------------------------
// Launch wrappers (defined in the .cu files).  All return cudaGetLastError() of the launch and
// add the number of kernels they launched to t_launches (the calling thread's counter).
extern thread_local uint64_t t_launches;

// Time-invariant inputs: a set bit means the array holds ONE matrix used at every step (stride
// 0); the kernels still read it for every step.  G and C may be time invariant only when every
// step has the same observation count.
enum { TI_F = 1, TI_H = 2, TI_K = 4, TI_G = 8, TI_C = 16 };
__host__ __device__ __forceinline__ int64_t ti_step(unsigned ti, unsigned bit, int64_t i) {
    return (ti & bit) ? 0 : i;
}

struct WhitenArgs {
    unsigned ti;                  // TI_* bits
    int64_t k;
    int n, mmax, m_uniform;       // m_uniform >= 0: every m_i equals it; -1: use goff/coff
    const int32_t* m;             // device [k] (m_uniform < 0)
    const int64_t* goff;          // device [k+1] row offsets into G/o (m_uniform < 0)
    const int64_t* coff;          // device [k+1] value offsets into C (m_uniform < 0)
    const double *F, *H, *c, *K, *G, *o, *C;
    void* level0;                 // out: level buffer (T), k records
    double* resid;                // out: [k] rows discarded by the observation pre-reduction
    double* LK;                   // out (refine mode): [k-1][n][n] Cholesky factors of K_i
    double* LC;                   // out (refine mode): packed Cholesky factors of C_i
    double* cn2;                  // out [k][n]: |Chat_i col|^2 + |B_i col|^2 (state i)
    double* cd2;                  // out [k][n]: |D_{i-1} col|^2 (state i; row 0 = 0)
    unsigned long long* bad;
    void* scratch;                // large-state path: the second level buffer (free while whitening)
    void* cta_scratch;            // state dimensions above 128: per-block slices (packed factors)
    int64_t cta_scratch_stride;   //   bytes per block
};

// Smallest normal number of T.  The reflector kernels that form tau and 1 / (alpha - beta) from
// the single reciprocal 1 / (beta (alpha - beta)) treat a column with alpha^2 + |x|^2 below it as
// zero: that product would be subnormal and its reciprocal overflow.  (In a rank-deficient block
// the columns past its rank keep rounding-level tails that shrink by a factor of about eps per
// reflector, so they reach that range after a few columns.)
template <typename T>
__host__ __device__ __forceinline__ T tiny_normal();
template <>
__host__ __device__ __forceinline__ double tiny_normal<double>() { return 2.2250738585072014e-308; }
template <>
__host__ __device__ __forceinline__ float tiny_normal<float>() { return 1.17549435e-38f; }

// Numerical singularity test of a finished diagonal block of R: |R_ii| is compared with the
// 2-norm of column i of the whitened matrix U A for that state (orthogonal transformations
// keep column norms, so |R_ii| <= that norm, and a ratio at rounding level means the column is
// dependent on the columns eliminated before it).
template <typename T>
__host__ __device__ __forceinline__ double singular_tol(int n);
template <>
__host__ __device__ __forceinline__ double singular_tol<double>(int n) { return 4.0 * n * 2.220446049250313e-16; }
template <>
__host__ __device__ __forceinline__ double singular_tol<float>(int n) { return 1.0 * n * 1.1920928955078125e-7; }

template <typename T>
__device__ __forceinline__ bool diag_is_singular(T d, double colnorm2, int n) {
    const double dd = (double)d;
    const double tol = singular_tol<T>(n);
    return !(dd * dd > tol * tol * colnorm2) || !isfinite(dd);
}

cudaError_t launch_whiten(const WhitenArgs& a, bool fp32, cudaStream_t st);

// After the whitening: flags ST_NONFINITE at state i when a column norm of the whitened blocks
// of state i (cn2, cd2: F_i, H_{i-1}, G_i through the whitening) or an entry of o_i or c_i is
// NaN or infinite.  Grid-stride and coalesced over each array.
cudaError_t launch_check_finite(const WhitenArgs& a, cudaStream_t st);

// Large-state path (one thread block per unit, in place; see ks_large.cu): used for state
// dimensions the column-owner kernels cannot hold in shared memory, up to LARGE_NMAX, with
// every m_i <= n.
constexpr int LARGE_NMAX = 128;
// Above LARGE_NMAX (up to HUGE_NMAX) the same kernels run with the QR panel in shared memory and
// the Cholesky factors, Rd^{-1} and M of SelInv in per-block slices of a global scratch (ks_smooth and
// ks_covariances only; the batched and served forms stop at LARGE_NMAX).
constexpr int HUGE_NMAX = 512;
// Per-block scratch of the whitening (bytes) and the number of blocks it is sized for.
size_t huge_whiten_scratch_bytes(int n);
unsigned huge_grid(int64_t units);
cudaError_t launch_selinv_huge(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                               void* ri_scratch, unsigned long long* bad, bool fp32, cudaStream_t st);
__host__ __device__ __forceinline__ bool use_large(int n, bool fp32) { return fp32 ? n > 64 : n > 48; }
size_t large_smem_bytes(int n, bool fp32);
// Whether the column-owner whitening of (n, mmax) fits the opt-in shared memory of sm_103a;
// otherwise (mmax <= n) the large-state whitening runs.
constexpr int SMEM_OPTIN_SM103 = 232448;
inline bool generic_whiten_fits(int n, int mmax) {
    return (size_t)whiten_layout(n, mmax).total * sizeof(double) <= (size_t)SMEM_OPTIN_SM103;
}
cudaError_t launch_whiten_large(const WhitenArgs& a, bool fp32, cudaStream_t st);
cudaError_t launch_level_large(int n, int64_t nc, int level, void* in, void* out, void* R,
                               double* resid, const double* cn2, const double* cd2,
                               unsigned long long* bad, bool fp32, cudaStream_t st);
cudaError_t launch_selinv_large(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                                unsigned long long* bad, bool fp32, cudaStream_t st);
struct BatchWork;
cudaError_t launch_batch_large(int op, int n, const BatchWork* wk, bool fp32, unsigned grid,
                               cudaStream_t st);

cudaError_t launch_level(int n, int64_t nc, int level, int64_t k, const void* in, void* out,
                         void* R, double* resid, const double* cn2, const double* cd2,
                         unsigned long long* bad, bool fp32, cudaStream_t st);

// The column-owner level kernel on the small-state layout (top levels of a small problem).
cudaError_t launch_level_soa(int n, int64_t nc, int level, int64_t k, const void* in, void* out,
                             void* R, double* resid, const double* cn2, const double* cd2,
                             unsigned long long* bad, bool fp32, cudaStream_t st);
// The column-owner SelInv kernel on the small-state layout.
cudaError_t launch_selinv_soa(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                              unsigned long long* bad, bool fp32, cudaStream_t st);

cudaError_t launch_base(int n, int64_t k, int L, const void* in, void* R, const double* cn2,
                        const double* cd2, unsigned long long* bad, bool fp32, cudaStream_t st);

// Odd-even SelInv at one level (Algorithm 2 body for every column eliminated at `level`).
cudaError_t launch_selinv(int n, int64_t k, int level, const void* R, void* Sx, double* Sd,
                          unsigned long long* bad, bool fp32, cudaStream_t st);

// Lag-one blocks cov(u_i, u_{i+1}) gathered from the SelInv store.
cudaError_t launch_cross(int n, int64_t k, const void* Sx, double* cross, bool fp32,
                         cudaStream_t st);

// Sum of a [count] FP64 array into *out (single block, deterministic order).
cudaError_t launch_sum(const double* x, int64_t count, double* out, cudaStream_t st);

// Refinement (KS_FP32_REFINE).  g = (UA)^T U (b - A u) in FP64 (Section 2's normal equations
// of the whitened system), then R^T w = g level by level, then R d = w, u += d.
struct RefineArgs {
    unsigned ti;
    int64_t k;
    int n, m_uniform;
    const int32_t* m;
    const int64_t *goff, *coff;
    const double *F, *H, *c, *G, *o, *LK, *LC;
    const double* u;
    double* g;     // out [k][n]
    double* q;     // scratch [k-1][n]: K_i^{-1} (F_i u_i + c_i - H_i u_{i+1})
};

// Warp-per-unit back substitution and mixed-precision refinement of the column-owner path.
cudaError_t launch_backsub_warp(int n, int64_t k, int level, const void* R, bool fp32,
                                double* u, cudaStream_t st);
cudaError_t launch_refine_warp(const RefineArgs& a, float* q, float* g, float* w, float* d,
                               const void* R, int L, cudaStream_t st);

// ---------------------------------------------------------------------------------------------
// Batched problems.  Every problem of a batch has a descriptor in device memory; a launch
// covers the units (steps, tiles, rows ...) of all problems of one class (same n and path) at
// one level, and maps a global unit index to (problem, local unit) through a prefix sum.  The
// descriptors and work lists live at fixed device addresses, so a captured CUDA graph of the
// launch sequence can be replayed for any batch of the same shape.
struct ProbDesc {
    unsigned ti;
    int cur_level;                // serving: this problem's level in the current launch
    int64_t k;
    int n, m_uniform, mmax, L;
    const int32_t* m;
    const int64_t *goff, *coff;
    const double *F, *H, *c, *K, *G, *o, *C;
    void* lvl[2];                 // ping-pong level buffers
    void* R;                      // R store
    double* resid;                // [2k]
    double *cn2, *cd2;            // [k][n] each
    double* u;                    // smoothed states [k][n]
    double *LK, *LC;              // Cholesky factors (refine mode)
    void *q, *g, *w, *d;          // refinement vectors
    void* Sx;                     // SelInv store
    double* cov;                  // covariances [k][n][n] or nullptr
    unsigned long long* bad;      // this problem's error words [ST_NCODES]
};

struct BatchWork {
    const ProbDesc* desc;  // all problems of the batch
    const int* probs;      // the problems of this launch's class
    const int64_t* off;    // prefix sum of units per problem [np + 1]
    int np;
    int level;             // >= 0: the level of every problem; -1: each problem's cur_level
};

__device__ __forceinline__ int work_level(const BatchWork& w, const ProbDesc& P) {
    return w.level >= 0 ? w.level : P.cur_level;
}

// Index into probs of the problem owning global unit u (off[p] <= u < off[p+1]).
__device__ __forceinline__ int batch_find(const int64_t* off, int np, int64_t u) {
    int lo = 0, hi = np;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ WhitenArgs whiten_args_of(const ProbDesc& P) {
    WhitenArgs a;
    a.ti = P.ti;
    a.k = P.k; a.n = P.n; a.mmax = P.mmax; a.m_uniform = P.m_uniform;
    a.m = P.m; a.goff = P.goff; a.coff = P.coff;
    a.F = P.F; a.H = P.H; a.c = P.c; a.K = P.K; a.G = P.G; a.o = P.o; a.C = P.C;
    a.level0 = P.lvl[0]; a.resid = P.resid + P.k; a.LK = P.LK; a.LC = P.LC;
    a.cn2 = P.cn2; a.cd2 = P.cd2; a.bad = P.bad;
    a.scratch = P.lvl[1];
    return a;
}

__device__ __forceinline__ RefineArgs refine_args_of(const ProbDesc& P) {
    RefineArgs a;
    a.ti = P.ti;
    a.k = P.k; a.n = P.n; a.m_uniform = P.m_uniform; a.m = P.m; a.goff = P.goff; a.coff = P.coff;
    a.F = P.F; a.H = P.H; a.c = P.c; a.G = P.G; a.o = P.o; a.LK = P.LK; a.LC = P.LC;
    a.u = P.u; a.g = (double*)P.g; a.q = (double*)P.q;
    return a;
}

// Batched launches of one class: `grid` blocks, persistent over the work list.
enum BatchOp {
    B_WHITEN = 0, B_LEVEL, B_BASE, B_BACKSUB, B_SELINV, B_REFINE_Q, B_REFINE_G, B_RT_SOLVE,
    B_BACKSUB_W, B_ADD, B_NOPS
};

// Kernels of the small-state path (one thread per step / tile / row, element-major layouts),
// one table per compile-time N.  small_ops(n) is nullptr when n has no table.
struct SmallOps {
    int n;
    cudaError_t (*whiten)(const WhitenArgs&, bool fp32, cudaStream_t);
    cudaError_t (*level)(int64_t nc, int level, int64_t k, const void* in, void* out, void* R,
                         double* resid, const double* cn2, const double* cd2,
                         unsigned long long* bad, bool fp32, cudaStream_t);
    cudaError_t (*base)(int64_t k, int L, const void* in, void* R, const double* cn2,
                        const double* cd2, unsigned long long* bad, bool fp32, cudaStream_t);
    cudaError_t (*backsub)(int64_t k, int level, const void* R, const double* w, double* u,
                           bool fp32, cudaStream_t);
    cudaError_t (*selinv)(int64_t k, int level, const void* R, void* Sx, double* Sd,
                          unsigned long long* bad, bool fp32, cudaStream_t);
    cudaError_t (*cross)(int64_t k, const void* Sx, double* cross, bool fp32, cudaStream_t);
    // Refinement (FP32 mode only): q, g from FP64 residuals; R^T w = g; R d = w; u += d.
    cudaError_t (*refine)(const RefineArgs& a, float* q, float* g, float* w, float* d,
                          const void* R, int L, cudaStream_t);
    // Batched form: one launch of operation `op` over the work list at `wk` (device memory).
    cudaError_t (*batch)(int op, const BatchWork* wk, bool fp32, unsigned grid, cudaStream_t);
};

// Register-column level and whitening kernels of medium state dimensions (compiled for a few
// n); used in place of the column-owner kernels when med_ops(n, fp32) (levels) or
// med_whiten_ops(n, mmax, fp32) (whitening) is not null.
struct MedOps {
    int n;
    bool fp64;             // FP64 levels compiled
    cudaError_t (*level)(int64_t nc, int level, int64_t k, const void* in, void* out, void* R,
                         double* resid, const double* cn2, const double* cd2,
                         unsigned long long* bad, bool fp32, cudaStream_t);
    cudaError_t (*batch_level)(const BatchWork* wk, bool fp32, unsigned grid, cudaStream_t);
    bool wfp64;            // FP64 whitening compiled
    cudaError_t (*whiten)(const WhitenArgs& a, bool fp32, cudaStream_t);
    cudaError_t (*batch_whiten)(const BatchWork* wk, bool fp32, unsigned grid, cudaStream_t);
};
const MedOps* med_ops(int n, bool fp32);
const MedOps* med_whiten_ops(int n, int mmax, bool fp32);

// Batched column-owner launches (classes with n > 8 or some m_i > n).
// family (levels of n with a register-column kernel): 0 = register-column, 1 = column owner.
cudaError_t launch_batch_generic(int op, int n, int mmax, const BatchWork* wk, bool fp32,
                                 unsigned grid, cudaStream_t st, int family = 0);
const SmallOps* small_ops(int n);
constexpr int SMALL_NMAX = 8;

}  // namespace ks

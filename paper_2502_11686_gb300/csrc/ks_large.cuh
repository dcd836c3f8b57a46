// ks_large.cuh -- the large-state path (state dimension above the shared-memory limit of the
// column-owner kernels, up to LARGE_NMAX = 128): whitening, the levels of the odd-even
// factorization and SelInv with one thread block (256 threads) per unit, working IN PLACE on the
// records in device memory (the unit's records stay in L2 while it is processed).
//
// * Levels (Section 3, steps 1-3 and the tail triple).  Every step is one "triangle over full
//   block" Householder QR, done blocked: a panel of PB = 32 reflectors is factored in shared
//   memory, its compact-WY form I - V T V^T built (T upper triangular, Schreiber & Van Loan
//   1989), and the trailing columns -- the rest of the factor and the companion blocks -- are
//   updated 32 columns at a time, X <- X - V (T^T (V^T X)).  The operands are the records
//   themselves: the R store row of the eliminated column receives [Rd | Rl | Rr | y] directly,
//   the new column's record is built in the output buffer, and the input records of the tile
//   (each read by this tile only) serve as the full blocks.
// * Whitening (Section 2): the Cholesky factors of K_i and C_i in FP64 (packed, shared memory,
//   right-looking, all threads on the trailing triangle), the triangular solves in the working
//   precision with one thread per right-hand column and 32 rows in registers, and the QR of the
//   whitened observation block with the blocked routine above.  The free second level buffer
//   holds the whitened observation block of each step.
// * SelInv (Section 4, Algorithm 2) reorganised so that no buffer beyond the outputs is needed:
//   with A = [Rl | Rr] and Ri = Rd^{-1} (shared memory),
//     P = A S_II            -> the S store row of c          (S_II from the neighbours' S blocks)
//     [Sl | Sr] = -Ri P     in place, row blocks top-down (Ri is upper triangular)
//     M = Ri - [Sl | Sr] A^T -> the covariance slot of c
//     S_cc = M Ri^T         in place, one row block at a time, then symmetrised,
//   which is S_cc = Ri Ri^T - [Sl | Sr] T^T with T = Ri A, the form of Algorithm 2.
//
// FP32 trailing updates on the tensor cores (tcgen05, 3xTF32; ks_tc.cuh).  With the panel's
// compact-WY factor I - V T V^T, a chunk of up to 128 trailing columns X = [Xt ; Xb] is
// updated as
//     W1 = Xt + V^T Xb      tensor cores: D1 = Xb^T V, Xb^T staged in TMEM (lane = column),
//                           V^T in shared memory; M = 128, N = 32, K = p
//     W2 = T^T W1           CUDA cores, one thread per column (32 x 32 triangle)
//     Xt -= W2; Xb -= V W2  tensor cores: D2 = V W2, V and W2^T in shared memory; M = 128,
//                           N = chunk width, K = 32
// with FP32 accumulators in TMEM (512 columns per block: Xb^T hi | lo, D1, D2).  Each product
// is the sum of the hi.lo, lo.hi and hi.hi TF32 products, which keeps FP32 accuracy.  Chunks
// narrower than 16 columns (the right-hand side) stay on the CUDA-core update.  The MMAs are
// issued by one thread and complete through an mbarrier; every wait is bounded and a timeout
// sets ST_TIMEOUT, stops further tensor-core work and still frees the TMEM.
#pragma once
#include <cstdlib>

#include "ks_internal.cuh"
#include "ks_tc.cuh"

namespace ks {
namespace large {

constexpr int NTH = 256;   // threads per block
constexpr int PB = 32;     // reflectors per panel
constexpr int CW = 32;     // columns per trailing-update chunk
constexpr int PMAX = LARGE_NMAX;
constexpr int LDV = PB + 1;
static_assert(NTH == 8 * PB && PMAX % 8 == 0, "the register panel gives each column 8 threads");

// Shared memory of the blocked QR (elements of T).
struct QrSmem {
    static constexpr int VB = 0;                       // PMAX x LDV: the panel's full-block part
    static constexpr int TP = VB + PMAX * LDV;         // PB x LDV: the panel's triangle part
    static constexpr int TM = TP + PB * LDV;           // PB x LDV: the T factor of the panel
    static constexpr int YG = TM + PB * LDV;           // PB x LDV: V^T V
    static constexpr int TAU = YG + PB * LDV;          // PB
    static constexpr int XT = TAU + PB;                // PB x CW: chunk rows of the triangle part
    static constexpr int XB = XT + PB * CW;            // PMAX x CW: chunk of the full block
    static constexpr int W1 = XB + PMAX * CW;          // PB x CW
    static constexpr int W2 = W1 + PB * CW;            // PB x CW
    static constexpr int TOTAL = W2 + PB * CW;
    static constexpr bool COMPACT = false;
};

// A column block of the stacked matrix [top ; bot]: top has the n rows of the triangle, bot the
// p rows of the full block; element (r, c) at top[r * ldt + c] / bot[r * ldb + c].
template <typename T>
struct Blk {
    T* top;
    int64_t ldt;
    T* bot;
    int64_t ldb;
    int ncols;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Trailing update of columns [c0, c0 + w) of block B by the panel's reflectors (top rows
// kk0 .. kk0 + bw - 1): X <- X - V T^T V^T X.
template <typename T>
__device__ void apply_chunk(const Blk<T>& B, int c0, int w, int kk0, int bw, int p, T* sm) {
    const T* Vb = sm + QrSmem::VB;
    const T* Tm = sm + QrSmem::TM;
    T* Xt = sm + QrSmem::XT;
    T* Xb = sm + QrSmem::XB;
    T* W1 = sm + QrSmem::W1;
    T* W2 = sm + QrSmem::W2;
    const int tid = threadIdx.x;
    for (int e = tid; e < PB * CW; e += NTH) {
        const int i = e / CW, j = e - i * CW;
        Xt[e] = (i < bw && j < w) ? B.top[(int64_t)(kk0 + i) * B.ldt + c0 + j] : T(0);
    }
    for (int e = tid; e < p * CW; e += NTH) {
        const int r = e / CW, j = e - r * CW;
        Xb[e] = j < w ? B.bot[(int64_t)r * B.ldb + c0 + j] : T(0);
    }
    __syncthreads();
    const int q = tid >> 3, j0 = (tid & 7) * 4;   // 32 x 32 outputs, 4 per thread
    {
        T a0 = Xt[q * CW + j0], a1 = Xt[q * CW + j0 + 1], a2 = Xt[q * CW + j0 + 2], a3 = Xt[q * CW + j0 + 3];
        for (int r = 0; r < p; ++r) {
            const T v = Vb[r * LDV + q];
            const T* x = Xb + r * CW + j0;
            a0 = fma(v, x[0], a0);
            a1 = fma(v, x[1], a1);
            a2 = fma(v, x[2], a2);
            a3 = fma(v, x[3], a3);
        }
        W1[q * CW + j0] = a0; W1[q * CW + j0 + 1] = a1; W1[q * CW + j0 + 2] = a2; W1[q * CW + j0 + 3] = a3;
    }
    __syncthreads();
    {
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        for (int s = 0; s <= q; ++s) {
            const T tv = Tm[s * LDV + q];
            const T* x = W1 + s * CW + j0;
            a0 = fma(tv, x[0], a0);
            a1 = fma(tv, x[1], a1);
            a2 = fma(tv, x[2], a2);
            a3 = fma(tv, x[3], a3);
        }
        W2[q * CW + j0] = a0; W2[q * CW + j0 + 1] = a1; W2[q * CW + j0 + 2] = a2; W2[q * CW + j0 + 3] = a3;
    }
    __syncthreads();
    for (int e = tid; e < bw * CW; e += NTH) {
        const int i = e / CW, j = e - i * CW;
        if (j < w) B.top[(int64_t)(kk0 + i) * B.ldt + c0 + j] = Xt[e] - W2[e];
    }
    for (int r = q; r < p; r += 32) {
        T a0 = Xb[r * CW + j0], a1 = Xb[r * CW + j0 + 1], a2 = Xb[r * CW + j0 + 2], a3 = Xb[r * CW + j0 + 3];
        for (int s = 0; s < bw; ++s) {
            const T v = Vb[r * LDV + s];
            const T* x = W2 + s * CW + j0;
            a0 = fma(-v, x[0], a0);
            a1 = fma(-v, x[1], a1);
            a2 = fma(-v, x[2], a2);
            a3 = fma(-v, x[3], a3);
        }
        T* dst = B.bot + (int64_t)r * B.ldb + c0 + j0;
        if (j0 < w) dst[0] = a0;
        if (j0 + 1 < w) dst[1] = a1;
        if (j0 + 2 < w) dst[2] = a2;
        if (j0 + 3 < w) dst[3] = a3;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Tensor-core state of a block (FP32 kernels).
struct TcSmem {   // byte offsets inside the block's tensor-core region
    static constexpr int B1 = 0;           // [V^T hi ; V^T lo], 64 x 128 tile (rows q | 32 + q, depth r)
    static constexpr int A2H = 32768;      // V, 128 x 32 tile (rows r, depth q), hi
    static constexpr int A2L = 49152;      //   lo
    static constexpr int B2H = 65536;      // W2^T, 128 x 32 tile (rows c, depth q), hi
    static constexpr int B2L = 81920;      //   lo
    static constexpr int MBAR = 98304;     // MMA completion barrier
    static constexpr int SLOT = 98312;     // TMEM address written by the allocation
    static constexpr int ABORT = 98316;    // set after a timed-out wait
    static constexpr int BYTES = 98320;
};
// TMEM columns: Xb^T hi | lo (A of the first product), D1 = [Xb^T_hi V_hi + Xb^T_lo V_hi |
// Xb^T_hi V_lo] (64 columns), D2 (up to 128 columns).
constexpr uint32_t TM_A1H = 0, TM_A1L = 128, TM_D1 = 256, TM_D2 = 384, TM_COLS = 512;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 20;   // polls; about a second at most
// Test-only stall mode (KS_TEST_STALL_TC=1, level kernels): the first chunk of each block issues
// no MMA and no commit, so its completion wait can only run out.  That exercises the timeout
// path (ST_TIMEOUT, abort flag, TMEM still freed) with nothing in flight on the tensor cores;
// the shorter limit keeps the test quick.
constexpr uint32_t TC_STALL_TEST_LIMIT = 1u << 14;
constexpr int TC_CW = 128;                 // columns per tensor-core chunk

// Compact layout of the FP32 tensor-core level kernel, small enough for two blocks per SM
// (TMEM is then taken per trailing update, see TcState::transient).  Only T and tau persist
// through a panel's trailing update; the panel buffers (V, the triangle, V^T V, the reflector
// exchange) are dead by then and live in the W2^T tiles of the tensor-core region, which are
// written only by the trailing update.  Offsets in floats from the start of shared memory; the
// tensor-core region starts at byte TC_BYTES.
struct QrSmemTc {
    static constexpr int TM = 0;
    static constexpr int TAU = TM + PB * LDV;
    static constexpr int TC_BYTES = ((TAU + PB) * 4 + 127) & ~127;
    static constexpr int VB = (TC_BYTES + TcSmem::B2H) / 4;
    static constexpr int TP = VB + PMAX * LDV;
    static constexpr int YG = TP + PB * LDV;
    static constexpr int XT = YG + PB * LDV;           // [2][PMAX] reflector exchange of the panel
    static constexpr int END = XT + 2 * PMAX;
    static constexpr int BYTES = TC_BYTES + TcSmem::BYTES;
    static constexpr bool COMPACT = true;
    static_assert(END * 4 <= TC_BYTES + TcSmem::MBAR, "panel buffers overlap the W2^T tiles only");
};

struct TcState {
    unsigned char* smem;                   // the region (TcSmem)
    uint32_t tmem;                         // first of TM_COLS allocated columns
    uint32_t phase;                        // parity of the next completion to wait for
    unsigned long long* bad;               // error words for ST_TIMEOUT
    int stall;                             // test-only stall mode (see TC_STALL_TEST_LIMIT)
    int transient;                         // TMEM taken per trailing update (tc_acquire/release)
};

__host__ __device__ inline size_t tc_align(size_t b) { return (b + 127) & ~(size_t)127; }

// Whole block: allocate TMEM (warp 0) unless `transient`, initialise the completion barrier.
// With `transient` the block holds no TMEM between trailing updates: tc_acquire takes all 512
// columns before one and tc_release frees them after it, so two blocks on an SM take turns on
// the tensor memory while the other one factors its panel on the CUDA cores.  A block never
// waits for TMEM while holding some, and every acquire is followed by a release (also after a
// timed-out wait), so the allocation of the other block always completes.
__device__ inline void tc_setup(TcState& tc, unsigned char* region, unsigned long long* bad,
                         int stall = 0, int transient = 0) {
    tc.smem = region;
    tc.phase = 0;
    tc.bad = bad;
    tc.stall = stall;
    tc.transient = transient;
    tc.tmem = 0;
    uint32_t* slot = reinterpret_cast<uint32_t*>(region + TcSmem::SLOT);
    if (threadIdx.x < 32 && !transient) {
        tc::tmem_alloc(slot, TM_COLS);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(reinterpret_cast<uint64_t*>(region + TcSmem::MBAR), 1);
        *reinterpret_cast<int*>(region + TcSmem::ABORT) = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (!transient) tc.tmem = *slot;
}

// Whole block, after its last tensor-core operation.
__device__ inline void tc_teardown(TcState& tc) {
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        if (tc.transient) tc::tmem_relinquish();
        else tc::tmem_dealloc(tc.tmem, TM_COLS);
    }
}

// Whole block, transient mode: take / give back the TMEM of one trailing update.
__device__ inline void tc_acquire(TcState& tc) {
    if (!tc.transient) return;
    uint32_t* slot = reinterpret_cast<uint32_t*>(tc.smem + TcSmem::SLOT);
    if (threadIdx.x < 32) tc::tmem_alloc(slot, TM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    tc.tmem = *slot;
}
__device__ inline void tc_release(TcState& tc) {
    if (!tc.transient) return;
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tc.tmem, TM_COLS);
}

// Whole block: wait for the last commit (bounded), then a barrier.  A timeout anywhere sets the
// abort flag (no further MMAs or waits) and ST_TIMEOUT.
__device__ inline void tc_wait(TcState& tc) {
    int* abort = reinterpret_cast<int*>(tc.smem + TcSmem::ABORT);
    bool ok = true;
    if (!*abort)
        ok = tc::mbar_wait(reinterpret_cast<uint64_t*>(tc.smem + TcSmem::MBAR), tc.phase,
                           tc.stall ? TC_STALL_TEST_LIMIT : TC_WAIT_LIMIT);
    tc.phase ^= 1u;
    if (__syncthreads_or(!ok) && threadIdx.x == 0) {
        if (!*abort && tc.bad != nullptr) flag_error(tc.bad, ST_TIMEOUT, 0);
        *abort = 1;
    }
    tc::fence_after();
}

// The panel's V (p x bw in QrSmem::VB, zero-padded to 128 x 32) as the two shared-memory
// operands: B1 = [V^T hi ; V^T lo] (rows q and 32 + q, depth r) and A2 = V (rows r, depth q),
// the latter split hi | lo.
template <typename L>
__device__ void tc_panel_prep(int p, int bw, const float* sm, TcState& tc) {
    const float* Vb = sm + L::VB;
    float* b1 = reinterpret_cast<float*>(tc.smem + TcSmem::B1);
    float* a2h = reinterpret_cast<float*>(tc.smem + TcSmem::A2H);
    float* a2l = reinterpret_cast<float*>(tc.smem + TcSmem::A2L);
    for (int e = threadIdx.x; e < 128 * PB; e += NTH) {
        const int q = e >> 7, r = e & 127;
        const float x = (r < p && q < bw) ? Vb[r * LDV + q] : 0.f;
        const float h = tc::tf32_hi(x), l = x - h;
        const uint32_t ia = tc::tile_off(128, r, q) >> 2;
        a2h[ia] = h;
        a2l[ia] = l;
        b1[tc::tile_off(2 * PB, q, r) >> 2] = h;
        b1[tc::tile_off(2 * PB, PB + q, r) >> 2] = l;
    }
    tc::fence_proxy_async_smem();
}

// A chunk of up to TC_CW trailing columns gathered from up to TC_SEGS column ranges of the
// blocks a panel updates (the rest of the factor, the companions, the right-hand side).
constexpr int TC_SEGS = 4;
struct TcChunk {
    int nseg, w;
    Blk<float> b[TC_SEGS];
    int c0[TC_SEGS];            // first column of segment s inside its block
    int off[TC_SEGS + 1];       // first chunk column of segment s; off[nseg] = w
};

// Block and in-block column of chunk column c (c < w).
__device__ __forceinline__ int tc_seg(const TcChunk& ch, int c) {
    int s = 0;
#pragma unroll
    for (int q = 1; q < TC_SEGS; ++q)
        if (q < ch.nseg && c >= ch.off[q]) s = q;
    return s;
}

// Part [J0, J1) of the first epilogue for chunk column c (see tc_apply_chunk): W2^T[c][j] =
// sum_{q <= j} W1^T[c][q] T[q][j], Xt[j][c] -= W2^T[c][j], and W2^T[c][j] (hi | lo) into the B2
// tile.  J0 and J1 are multiples of 4.
template <int J0, int J1>
__device__ __forceinline__ void tc_epi1_part(const float (&v)[32], const float (&xt)[32], bool live,
                                             float* top, int64_t ldt, int kk0, int bw, int c,
                                             const float* Tm, float* b2h, float* b2l) {
    float w2[J1 - J0];
#pragma unroll
    for (int j = J0; j < J1; ++j) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int q = 0; q <= j; ++q) {
            if (q & 1) a1 = fma(v[q], Tm[q * LDV + j], a1);
            else a0 = fma(v[q], Tm[q * LDV + j], a0);
        }
        w2[j - J0] = a0 + a1;
    }
    if (live) {
#pragma unroll
        for (int j = J0; j < J1; ++j)
            if (j < bw) top[(int64_t)(kk0 + j) * ldt] = xt[j] - w2[j - J0];
    }
#pragma unroll
    for (int j = J0; j < J1; j += 4) {
        float4 h4, l4;
        h4.x = tc::tf32_hi(w2[j - J0]);     l4.x = w2[j - J0] - h4.x;
        h4.y = tc::tf32_hi(w2[j - J0 + 1]); l4.y = w2[j - J0 + 1] - h4.y;
        h4.z = tc::tf32_hi(w2[j - J0 + 2]); l4.z = w2[j - J0 + 2] - h4.z;
        h4.w = tc::tf32_hi(w2[j - J0 + 3]); l4.w = w2[j - J0 + 3] - h4.w;
        const uint32_t o = tc::tile_off(128, c, j) >> 2;
        *reinterpret_cast<float4*>(b2h + o) = h4;
        *reinterpret_cast<float4*>(b2l + o) = l4;
    }
}

// Trailing update of the chunk's columns by the panel whose reflectors are rows kk0 .. kk0 +
// bw - 1 of the triangle part (see the file comment).  Whole block.
__device__ inline void tc_apply_chunk(const TcChunk& ch, int kk0, int bw, int p, const float* Tm,
                                      TcState& tc) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, half = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * q4) << 16;
    const int w = ch.w;
    const int KP = (p + 7) & ~7;
    const int NR = (p + 15) & ~15;   // rows of the second product (its N)
    const int* abort = reinterpret_cast<const int*>(tc.smem + TcSmem::ABORT);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tc.smem + TcSmem::MBAR);
    // Thread-column c = 32 q4 + lane (the same column for both warp halves): its block column.
    const int c = 32 * q4 + lane;
    const bool live = c < w;
    const int sg = live ? tc_seg(ch, c) : 0;
    const int cc = live ? ch.c0[sg] + (c - ch.off[sg]) : 0;
    // 1. Xb^T into TMEM: lane c = chunk column c, columns r (hi at TM_A1H, lo at TM_A1L); the
    //    warp halves take alternate 32-row pieces, all loads of a warp issued before its stores.
    {
        const float* col = live ? ch.b[sg].bot + cc : nullptr;
        const int64_t ldb = live ? ch.b[sg].ldb : 0;
        float x0[32], x1[32];
        const int pa = half, pb = half + 2;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int ra = pa * 32 + j, rb = pb * 32 + j;
            x0[j] = (live && ra < p) ? col[(int64_t)ra * ldb] : 0.f;
            x1[j] = (live && rb < p) ? col[(int64_t)rb * ldb] : 0.f;
        }
        float h[32], l[32];
        if (pa * 32 < KP) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                h[j] = tc::tf32_hi(x0[j]);
                l[j] = x0[j] - h[j];
            }
            tc::tmem_st32(tc.tmem + lanes + TM_A1H + (uint32_t)(pa * 32), h);
            tc::tmem_st32(tc.tmem + lanes + TM_A1L + (uint32_t)(pa * 32), l);
        }
        if (pb * 32 < KP) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                h[j] = tc::tf32_hi(x1[j]);
                l[j] = x1[j] - h[j];
            }
            tc::tmem_st32(tc.tmem + lanes + TM_A1H + (uint32_t)(pb * 32), h);
            tc::tmem_st32(tc.tmem + lanes + TM_A1L + (uint32_t)(pb * 32), l);
        }
    }
    tc::fence_before();
    __syncthreads();
    // 2. D1 (M = 128 columns c, K = KP rows): one N = 64 product Xb^T_hi [V_hi | V_lo] and one
    //    N = 32 product Xb^T_lo V_hi into its first 32 columns, per K = 8 step.  (In the
    //    test-only stall mode nothing is issued, so the wait below runs out.)
    if (tid == 0 && !*abort && !tc.stall) {
        tc::fence_after();
        const uint32_t id64 = tc::idesc_tf32(128, 2 * PB), id32 = tc::idesc_tf32(128, PB);
        const uint64_t b0 = tc::tile_desc(tc::smem_u32(tc.smem + TcSmem::B1), 2 * PB, 0);
        const uint32_t d1 = tc.tmem + TM_D1;
        for (int s = 0; s < KP / 8; ++s) {
            const uint64_t bd = b0 + (uint64_t)((32 * 2 * PB * s) >> 4);
            tc::mma_ts(d1, tc.tmem + TM_A1H + 8 * s, bd, id64, s > 0 ? 1u : 0u);
            tc::mma_ts(d1, tc.tmem + TM_A1L + 8 * s, bd, id32, 1u);
        }
        tc::commit(mbar);
    }
    tc_wait(tc);
    // 3. W1 = Xt + D1^T (both halves of every warp group hold the column's 32 values), then
    //    W2^T = W1^T T split over the halves: j < 24 and j >= 24.
    {
        float* top = live ? ch.b[sg].top + cc : nullptr;
        const int64_t ldt = live ? ch.b[sg].ldt : 0;
        float v[32], v2[32];
        tc::tmem_ld32(tc.tmem + lanes + TM_D1, v);
        tc::tmem_ld32(tc.tmem + lanes + TM_D1 + PB, v2);
        float xt[32];
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            xt[q] = (live && q < bw) ? top[(int64_t)(kk0 + q) * ldt] : 0.f;
            v[q] += v2[q] + xt[q];
        }
        float* b2h = reinterpret_cast<float*>(tc.smem + TcSmem::B2H);
        float* b2l = reinterpret_cast<float*>(tc.smem + TcSmem::B2L);
        if (half == 0) tc_epi1_part<0, 24>(v, xt, live, top, ldt, kk0, bw, c, Tm, b2h, b2l);
        else tc_epi1_part<24, 32>(v, xt, live, top, ldt, kk0, bw, c, Tm, b2h, b2l);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before();
    __syncthreads();
    // 4. D2^T = W2^T V^T (M = 128 chunk columns c, N = NR rows r, K = 32): lane c, column r --
    //    the layout of Xb^T in TMEM, so step 5 updates a column from its own TMEM lane.
    if (tid == 0 && !*abort) {
        tc::fence_after();
        const uint32_t id = tc::idesc_tf32(128, NR);
        const uint64_t wh = tc::tile_desc(tc::smem_u32(tc.smem + TcSmem::B2H), 128, 0);
        const uint64_t wl = tc::tile_desc(tc::smem_u32(tc.smem + TcSmem::B2L), 128, 0);
        const uint64_t vh = tc::tile_desc(tc::smem_u32(tc.smem + TcSmem::A2H), 128, 0);
        const uint64_t vl = tc::tile_desc(tc::smem_u32(tc.smem + TcSmem::A2L), 128, 0);
        const uint32_t d2 = tc.tmem + TM_D2;
        for (int s = 0; s < PB / 8; ++s) {
            const uint64_t st = (uint64_t)((32 * 128 * s) >> 4);
            tc::mma_ss(d2, wh + st, vl + st, id, s > 0 ? 1u : 0u);
            tc::mma_ss(d2, wl + st, vh + st, id, 1u);
            tc::mma_ss(d2, wh + st, vh + st, id, 1u);
        }
        tc::commit(mbar);
    }
    tc_wait(tc);
    // 5. Xb = (Xb^T hi + lo) - D2^T, from this column's TMEM lane (rows 64 half .. + 63 in two
    //    32-row pieces); the stores of a warp run along a row, lane = column.
    {
        float* base = live ? ch.b[sg].bot + cc : nullptr;
        const int64_t ldb = live ? ch.b[sg].ldb : 0;
        for (int piece = 0; piece < 2; ++piece) {
            const int r0 = 64 * half + 32 * piece;
            if (r0 >= KP) break;   // uniform over the warp
            float x[32], t[32];
            tc::tmem_ld32(tc.tmem + lanes + TM_A1H + (uint32_t)r0, x);
            tc::tmem_ld32(tc.tmem + lanes + TM_A1L + (uint32_t)r0, t);
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) x[rr] += t[rr];
            tc::tmem_ld32(tc.tmem + lanes + TM_D2 + (uint32_t)r0, t);
#pragma unroll
            for (int rr = 0; rr < 32; ++rr)
                if (live && r0 + rr < p) base[(int64_t)(r0 + rr) * ldb] = x[rr] - t[rr];
        }
    }
    tc::fence_before();
    __syncthreads();
}

// Compact-WY factor T (PB x PB, upper triangular) of a panel of bw reflectors with taus tau and
// Gram matrix Y = V^T V (strict upper part used):  T[i][i] = tau_i and, for q < i,
// T[q][i] = -tau_i sum_{q <= s < i} T[q][s] Y[s][i]  (Schreiber & Van Loan 1989).  Rows are
// independent.  Lane q of one warp forms row q from left to right; each finished T[q][s] goes
// into the partial sums of all later columns at once, so a step is a row of independent FMAs
// rather than a dependent dot product.  Whole warp.
template <typename T>
__device__ __forceinline__ void wy_t_factor(T* Tm, const T* Y, const T* tau, int bw) {
    const int lane = threadIdx.x & 31;
    T acc[PB];
#pragma unroll
    for (int i = 0; i < PB; ++i) acc[i] = T(0);
    T* tq = Tm + lane * LDV;
#pragma unroll
    for (int s = 0; s < PB; ++s) {
        const T ts = s < bw ? tau[s] : T(0);
        const T t = lane < s ? -ts * acc[s] : (lane == s ? ts : T(0));
        tq[s] = t;
#pragma unroll
        for (int i = s + 1; i < PB; ++i) acc[i] = fma(t, Y[s * LDV + i], acc[i]);
    }
}

// Blocked "triangle over full block" QR: F.top (n x n, upper triangular) over F.bot (p x n),
// applied to the companion blocks C[0 .. nc).  On return F.top holds R; F.bot is consumed.
// With tc (FP32 only) the trailing updates run on the tensor cores.  L is the shared-memory
// layout (QrSmem, or QrSmemTc with tc, FP32 only).
template <typename T, typename L = QrSmem>
__device__ void tpqrt_wy(int n, int p, const Blk<T>& F, const Blk<T>* C, int nc, T* sm,
                         TcState* tc = nullptr) {
    T* Vb = sm + L::VB;
    T* Tp = sm + L::TP;
    T* Tm = sm + L::TM;
    T* Y = sm + L::YG;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (p == 0) return;
    for (int kk0 = 0; kk0 < n; kk0 += PB) {
        const int bw = n - kk0 < PB ? n - kk0 : PB;
        __syncthreads();
        for (int e = tid; e < p * PB; e += NTH) {
            const int r = e / PB, j = e - r * PB;
            Vb[r * LDV + j] = j < bw ? F.bot[(int64_t)r * F.ldb + kk0 + j] : T(0);
        }
        for (int e = tid; e < PB * PB; e += NTH) {
            const int i = e / PB, j = e - i * PB;
            Tp[i * LDV + j] = (i < bw && j < bw && i <= j) ? F.top[(int64_t)(kk0 + i) * F.ldt + kk0 + j] : T(0);
        }
        __syncthreads();
        // Panel, register form: thread t works on panel column j = t / 8 and holds the rows
        // r = t % 8 + 8 s (s < PMAX / 8) of the full block.  Reflector i: the eight threads of
        // column i form it and publish v (double-buffered, so one barrier per reflector); every
        // later column applies it at once (16-term partial dots, a three-step group reduction)
        // and recomputes its |x|^2 for when its own turn comes.
        {
            constexpr int RS = PMAX / 8;
            const int j = tid >> 3, sub = tid & 7;
            T* XV = sm + L::XT;   // [2][PMAX] (the chunk buffers are free during the panel)
            auto gsum = [](T v) {
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                return v;
            };
            T x[RS];
            T a0 = T(0);
#pragma unroll
            for (int s2 = 0; s2 < RS; ++s2) {
                const int r = sub + 8 * s2;
                x[s2] = (r < p && j < bw) ? Vb[r * LDV + j] : T(0);
                a0 = fma(x[s2], x[s2], a0);
            }
            T sig = gsum(a0);
            for (int i = 0; i < bw; ++i) {
                T* v = XV + (i & 1) * PMAX;
                if (j == i) {
                    const T alpha = Tp[i * LDV + i];
                    T g = T(0), tau = T(0), beta = alpha;
                    if (sig != T(0)) {
                        const T nrm = sqrt(fma(alpha, alpha, sig));
                        beta = alpha >= T(0) ? -nrm : nrm;
                        g = T(1) / (alpha - beta);
                        tau = (beta - alpha) / beta;
                    }
#pragma unroll
                    for (int s2 = 0; s2 < RS; ++s2) {
                        x[s2] *= g;
                        v[sub + 8 * s2] = x[s2];
                    }
                    if (sub == 0) {
                        Tp[i * LDV + i] = beta;
                        sm[L::TAU + i] = tau;
                    }
                }
                __syncthreads();
                const T tau = sm[L::TAU + i];
                T d = T(0);
#pragma unroll
                for (int s2 = 0; s2 < RS; ++s2) d = fma(v[sub + 8 * s2], x[s2], d);
                d = gsum(d);
                if (j > i && j < bw) {
                    const T sc = tau * (d + Tp[i * LDV + j]);
#pragma unroll
                    for (int s2 = 0; s2 < RS; ++s2) x[s2] = fma(-sc, v[sub + 8 * s2], x[s2]);
                    if (sub == 0) Tp[i * LDV + j] -= sc;
                }
                T a = T(0);
#pragma unroll
                for (int s2 = 0; s2 < RS; ++s2) a = fma(x[s2], x[s2], a);
                sig = gsum(a);
            }
#pragma unroll
            for (int s2 = 0; s2 < RS; ++s2) {
                const int r = sub + 8 * s2;
                if (r < p) Vb[r * LDV + j] = x[s2];
            }
        }
        __syncthreads();
        // R entries of the panel back to the triangle; Gram matrix V^T V of the panel.
        for (int e = tid; e < bw * bw; e += NTH) {
            const int i = e / bw, j = e - i * bw;
            if (i <= j) F.top[(int64_t)(kk0 + i) * F.ldt + kk0 + j] = Tp[i * LDV + j];
        }
        for (int e = tid; e < PB * PB; e += NTH) {
            const int a = e / PB, b = e - a * PB;
            T s = T(0);
            if (a < b && b < bw)
                for (int r = 0; r < p; ++r) s = fma(Vb[r * LDV + a], Vb[r * LDV + b], s);
            Y[a * LDV + b] = s;
        }
        __syncthreads();
        if (warp == 0) wy_t_factor<T>(Tm, Y, sm + L::TAU, bw);
        __syncthreads();
        // Trailing update: the rest of the factor, then every companion block.
        if constexpr (sizeof(T) == 4) {
            if (tc != nullptr) {
                tc_panel_prep<L>(p, bw, sm, *tc);
                tc_acquire(*tc);
                // Every trailing column (rest of the factor, then the companions) packed into
                // chunks of TC_CW columns.
                TcChunk ch;
                ch.nseg = 0;
                ch.w = 0;
                auto flush = [&]() {
                    if (ch.w > 0) {
                        ch.off[ch.nseg] = ch.w;
                        tc_apply_chunk(ch, kk0, bw, p, Tm, *tc);
                    }
                    ch.nseg = 0;
                    ch.w = 0;
                };
                auto add = [&](const Blk<T>& B, int first) {
                    for (int c = first; c < B.ncols;) {
                        if (ch.nseg == TC_SEGS || ch.w == TC_CW) flush();
                        const int take = (B.ncols - c) < (TC_CW - ch.w) ? (B.ncols - c) : (TC_CW - ch.w);
                        ch.b[ch.nseg] = B;
                        ch.c0[ch.nseg] = c;
                        ch.off[ch.nseg] = ch.w;
                        ++ch.nseg;
                        ch.w += take;
                        c += take;
                    }
                };
                add(F, kk0 + bw);
                for (int b = 0; b < nc; ++b) add(C[b], 0);
                flush();
                tc_release(*tc);
                continue;
            }
        }
        if constexpr (!L::COMPACT) {
            for (int c0 = kk0 + bw; c0 < n; c0 += CW)
                apply_chunk<T>(F, c0, (n - c0) < CW ? (n - c0) : CW, kk0, bw, p, sm);
            for (int b = 0; b < nc; ++b)
                for (int c0 = 0; c0 < C[b].ncols; c0 += CW)
                    apply_chunk<T>(C[b], c0, (C[b].ncols - c0) < CW ? (C[b].ncols - c0) : CW, kk0, bw, p, sm);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Blocked "triangle over full block" QR for full blocks of more than PMAX rows (state dimensions
// above 128, up to BIG_NMAX).  The panel's reflectors stay in shared memory (p x PB); reflector
// i is formed by one warp (norm by a shuffle reduction) and applied to the later panel columns
// by all warps, a column per warp at a time; then the compact-WY factor T and the trailing
// update of the remaining columns, BCW(T) columns at a time with the chunk of the full block
// staged in shared memory:  W1 = Xt + V^T Xb,  W2 = T^T W1,  Xt -= W2,  Xb -= V W2.
constexpr int BIG_NMAX = 512;
template <typename T> struct BigCw { static constexpr int v = 32; };
template <> struct BigCw<double> { static constexpr int v = 8; };

template <typename T>
struct BigSmem {
    static constexpr int CW_ = BigCw<T>::v;
    // offsets (elements of T) for full blocks of p rows
    __host__ __device__ static int vs(int) { return 0; }
    __host__ __device__ static int tp(int p) { return p * LDV; }
    __host__ __device__ static int tm(int p) { return tp(p) + PB * LDV; }
    __host__ __device__ static int yg(int p) { return tm(p) + PB * LDV; }
    __host__ __device__ static int tau(int p) { return yg(p) + PB * LDV; }
    __host__ __device__ static int xt(int p) { return tau(p) + PB; }
    __host__ __device__ static int xb(int p) { return xt(p) + PB * CW_; }
    __host__ __device__ static int w1(int p) { return xb(p) + p * CW_; }
    __host__ __device__ static int w2(int p) { return w1(p) + PB * CW_; }
    __host__ __device__ static int total(int p) { return w2(p) + PB * CW_; }
    __host__ __device__ static size_t bytes(int p) { return (size_t)total(p) * sizeof(T); }
};

// Columns [c0, c0 + w) of block B by the panel (top rows kk0 .. kk0 + bw - 1).
template <typename T>
__device__ void big_apply_chunk(const Blk<T>& B, int c0, int w, int kk0, int bw, int p, T* sm) {
    constexpr int CW_ = BigCw<T>::v;
    const T* Vs = sm + BigSmem<T>::vs(p);
    const T* Tm = sm + BigSmem<T>::tm(p);
    T* Xt = sm + BigSmem<T>::xt(p);
    T* Xb = sm + BigSmem<T>::xb(p);
    T* W1 = sm + BigSmem<T>::w1(p);
    T* W2 = sm + BigSmem<T>::w2(p);
    const int tid = threadIdx.x;
    for (int e = tid; e < PB * CW_; e += NTH) {
        const int i = e / CW_, j = e - i * CW_;
        Xt[e] = (i < bw && j < w) ? B.top[(int64_t)(kk0 + i) * B.ldt + c0 + j] : T(0);
    }
    for (int e = tid; e < p * CW_; e += NTH) {
        const int r = e / CW_, j = e - r * CW_;
        Xb[e] = j < w ? B.bot[(int64_t)r * B.ldb + c0 + j] : T(0);
    }
    __syncthreads();
    // W1: PB x CW outputs over NTH threads, OUT consecutive columns each
    constexpr int OUT = PB * CW_ / NTH;
    static_assert(OUT >= 1 && CW_ % OUT == 0, "chunk width");
    {
        const int q = tid / (CW_ / OUT), j0 = (tid % (CW_ / OUT)) * OUT;
        T acc[OUT];
#pragma unroll
        for (int o = 0; o < OUT; ++o) acc[o] = Xt[q * CW_ + j0 + o];
        for (int r = 0; r < p; ++r) {
            const T v = Vs[r * LDV + q];
#pragma unroll
            for (int o = 0; o < OUT; ++o) acc[o] = fma(v, Xb[r * CW_ + j0 + o], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < OUT; ++o) W1[q * CW_ + j0 + o] = acc[o];
    }
    __syncthreads();
    {
        const int q = tid / (CW_ / OUT), j0 = (tid % (CW_ / OUT)) * OUT;
        T acc[OUT];
#pragma unroll
        for (int o = 0; o < OUT; ++o) acc[o] = T(0);
        for (int s = 0; s <= q; ++s) {
            const T tv = Tm[s * LDV + q];
#pragma unroll
            for (int o = 0; o < OUT; ++o) acc[o] = fma(tv, W1[s * CW_ + j0 + o], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < OUT; ++o) W2[q * CW_ + j0 + o] = acc[o];
    }
    __syncthreads();
    for (int e = tid; e < bw * CW_; e += NTH) {
        const int i = e / CW_, j = e - i * CW_;
        if (j < w) B.top[(int64_t)(kk0 + i) * B.ldt + c0 + j] = Xt[e] - W2[e];
    }
    for (int e = tid; e < p * CW_; e += NTH) {
        const int r = e / CW_, j = e - r * CW_;
        if (j >= w) continue;
        T a = Xb[e];
        for (int s = 0; s < bw; ++s) a = fma(-Vs[r * LDV + s], W2[s * CW_ + j], a);
        B.bot[(int64_t)r * B.ldb + c0 + j] = a;
    }
    __syncthreads();
}

template <typename T>
__device__ void tpqrt_big(int n, int p, const Blk<T>& F, const Blk<T>* C, int nc, T* sm) {
    constexpr int CW_ = BigCw<T>::v;
    T* Vs = sm + BigSmem<T>::vs(p);
    T* Tp = sm + BigSmem<T>::tp(p);
    T* Tm = sm + BigSmem<T>::tm(p);
    T* Y = sm + BigSmem<T>::yg(p);
    T* tau_s = sm + BigSmem<T>::tau(p);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = NTH / 32;
    if (p == 0) return;
    for (int kk0 = 0; kk0 < n; kk0 += PB) {
        const int bw = n - kk0 < PB ? n - kk0 : PB;
        __syncthreads();
        for (int e = tid; e < p * PB; e += NTH) {
            const int r = e / PB, j = e - r * PB;
            Vs[r * LDV + j] = j < bw ? F.bot[(int64_t)r * F.ldb + kk0 + j] : T(0);
        }
        for (int e = tid; e < PB * PB; e += NTH) {
            const int i = e / PB, j = e - i * PB;
            Tp[i * LDV + j] = (i < bw && j < bw && i <= j) ? F.top[(int64_t)(kk0 + i) * F.ldt + kk0 + j] : T(0);
        }
        __syncthreads();
        for (int i = 0; i < bw; ++i) {
            // reflector i by warp 0: v = [1 ; x / (alpha - beta)], beta = -sign(alpha) |(alpha, x)|
            if (warp == 0) {
                T s = T(0);
                for (int r = lane; r < p; r += 32) s = fma(Vs[r * LDV + i], Vs[r * LDV + i], s);
                s = warp_sum(s);
                const T alpha = Tp[i * LDV + i];
                T g = T(0), tau = T(0), beta = alpha;
                if (s != T(0)) {
                    const T nrm = sqrt(fma(alpha, alpha, s));
                    beta = alpha >= T(0) ? -nrm : nrm;
                    g = T(1) / (alpha - beta);
                    tau = (beta - alpha) / beta;
                }
                for (int r = lane; r < p; r += 32) Vs[r * LDV + i] *= g;
                if (lane == 0) {
                    Tp[i * LDV + i] = beta;
                    tau_s[i] = tau;
                }
            }
            __syncthreads();
            const T tau = tau_s[i];
            for (int j = i + 1 + warp; j < bw; j += NW) {
                T d = T(0);
                for (int r = lane; r < p; r += 32) d = fma(Vs[r * LDV + i], Vs[r * LDV + j], d);
                d = warp_sum(d);
                const T sc = tau * (d + Tp[i * LDV + j]);
                for (int r = lane; r < p; r += 32) Vs[r * LDV + j] = fma(-sc, Vs[r * LDV + i], Vs[r * LDV + j]);
                if (lane == 0) Tp[i * LDV + j] -= sc;
            }
            __syncthreads();
        }
        for (int e = tid; e < bw * bw; e += NTH) {
            const int i = e / bw, j = e - i * bw;
            if (i <= j) F.top[(int64_t)(kk0 + i) * F.ldt + kk0 + j] = Tp[i * LDV + j];
        }
        for (int e = tid; e < PB * PB; e += NTH) {
            const int a = e / PB, b = e - a * PB;
            T s = T(0);
            if (a < b && b < bw)
                for (int r = 0; r < p; ++r) s = fma(Vs[r * LDV + a], Vs[r * LDV + b], s);
            Y[a * LDV + b] = s;
        }
        __syncthreads();
        if (warp == 0) wy_t_factor<T>(Tm, Y, tau_s, bw);
        __syncthreads();
        for (int c0 = kk0 + bw; c0 < n; c0 += CW_)
            big_apply_chunk<T>(F, c0, (n - c0) < CW_ ? (n - c0) : CW_, kk0, bw, p, sm);
        for (int b = 0; b < nc; ++b)
            for (int c0 = 0; c0 < C[b].ncols; c0 += CW_)
                big_apply_chunk<T>(C[b], c0, (C[b].ncols - c0) < CW_ ? (C[b].ncols - c0) : CW_, kk0, bw, p, sm);
    }
    __syncthreads();
}

// The QR of a level or whitening step: the register-panel form (with tensor cores in FP32) up
// to PMAX rows, the shared-memory-panel form above.
template <typename T, typename L = QrSmem>
__device__ __forceinline__ void tpqrt_any(int n, int p, const Blk<T>& F, const Blk<T>* C, int nc,
                                          T* sm, TcState* tc) {
    if constexpr (L::COMPACT) tpqrt_wy<T, L>(n, p, F, C, nc, sm, tc);   // n <= PMAX only
    else if (n > PMAX) tpqrt_big<T>(n, p, F, C, nc, sm);
    else tpqrt_wy<T, L>(n, p, F, C, nc, sm, tc);
}

// ------------------------------------------------------------------------------------------
// Level tile t (records in the generic layout; see the file comment).  L: the QR's
// shared-memory layout (QrSmemTc for the two-blocks-per-SM tensor-core kernel).
template <typename T, typename L = QrSmem>
__device__ void level_tile(int n, int64_t nc, int level, int64_t t, T* in, T* out, T* R,
                           double* resid, const double* cn2, const double* cd2,
                           unsigned long long* bad, T* sm, TcState* tc = nullptr) {
    const int tid = threadIdx.x;
    const int64_t nn = (int64_t)n * n;
    const int64_t CS = level_cs(n), RS = rstore_rs(n);
    const int64_t nt = nc / 2;
    const int64_t j = 2 * t, s = j + 1;
    const bool triple = (nc & 1) && (t == nt - 1);
    const int64_t oj = ((j + 1) << level) - 1;
    T* rj = in + j * CS;
    T* rs = in + s * CS;
    T* ro = out + t * CS;
    T* Rj = R + oj * RS;
    auto rec_C = [&](T* r) { return r; };
    auto rec_RC = [&](T* r) { return r + nn; };
    auto rec_E = [&](T* r) { return r + nn + n; };
    auto rec_RE = [&](T* r) { return r + 3 * nn + n; };

    // R row of column j: [Rd | Rl | Rr | y] <- [Chat_j | 0 | 0 | rC_j]
    for (int64_t e = tid; e < nn; e += NTH) {
        Rj[e] = rec_C(rj)[e];
        Rj[nn + e] = T(0);
        Rj[2 * nn + e] = T(0);
    }
    for (int r = tid; r < n; r += NTH) Rj[3 * nn + r] = rec_RC(rj)[r];
    __syncthreads();
    // step 1: [Chat_j ; -B_s], companions [0 ; D_s] (-> X_j, Dtilde_s) and [rC_j ; rE_s]
    {
        const Blk<T> F{Rj, n, rec_E(rs), 2 * n, n};
        const Blk<T> C[2] = {{Rj + 2 * nn, n, rec_E(rs) + n, 2 * n, n}, {Rj + 3 * nn, 1, rec_RE(rs), 1, 1}};
        tpqrt_any<T, L>(n, n, F, C, 2, sm, tc);
    }
    if (j >= 1) {
        // step 2: [Rtilde_j ; D_j], companions [0 ; -B_j] (left), [X_j ; 0] (right), [t_j ; rE_j];
        // the bottoms become the new column's coupling record.
        for (int64_t e = tid; e < nn; e += NTH) {
            const int64_t r = e / n, c = e - r * n;
            rec_E(ro)[r * 2 * n + c] = rec_E(rj)[r * 2 * n + c];
            rec_E(ro)[r * 2 * n + n + c] = T(0);
        }
        for (int r = tid; r < n; r += NTH) rec_RE(ro)[r] = rec_RE(rj)[r];
        __syncthreads();
        const Blk<T> F{Rj, n, rec_E(rj) + n, 2 * n, n};
        const Blk<T> C[3] = {{Rj + nn, n, rec_E(ro), 2 * n, n},
                             {Rj + 2 * nn, n, rec_E(ro) + n, 2 * n, n},
                             {Rj + 3 * nn, 1, rec_RE(ro), 1, 1}};
        tpqrt_any<T, L>(n, n, F, C, 3, sm, tc);
    }
    for (int c = tid; c < n; c += NTH)
        if (diag_is_singular<T>(Rj[(int64_t)c * n + c], cn2[oj * n + c] + cd2[oj * n + c], n))
            flag_error(bad, ST_SINGULAR, oj);
    // new column t: [Chat'_t | rC'_t] starts as [Chat_s | rC_s]
    for (int64_t e = tid; e < nn; e += NTH) rec_C(ro)[e] = rec_C(rs)[e];
    for (int r = tid; r < n; r += NTH) rec_RC(ro)[r] = rec_RC(rs)[r];
    T* re = nullptr;
    if (triple) {
        // tail column e: step 2 of [Chat_e ; D_e] with companions [0 ; -B_e] (-> Z_e), [rC_e ; rE_e]
        const int64_t e_ = j + 2;
        const int64_t oe = ((e_ + 1) << level) - 1;
        re = in + e_ * CS;
        T* Re = R + oe * RS;
        for (int64_t e = tid; e < nn; e += NTH) {
            Re[e] = rec_C(re)[e];
            Re[nn + e] = T(0);
            Re[2 * nn + e] = T(0);
        }
        for (int r = tid; r < n; r += NTH) Re[3 * nn + r] = rec_RC(re)[r];
        __syncthreads();
        const Blk<T> F{Re, n, rec_E(re) + n, 2 * n, n};
        const Blk<T> C[2] = {{Re + nn, n, rec_E(re), 2 * n, n}, {Re + 3 * nn, 1, rec_RE(re), 1, 1}};
        tpqrt_any<T, L>(n, n, F, C, 2, sm, tc);
        for (int c = tid; c < n; c += NTH)
            if (diag_is_singular<T>(Re[(int64_t)c * n + c], cn2[oe * n + c] + cd2[oe * n + c], n))
                flag_error(bad, ST_SINGULAR, oe);
    }
    __syncthreads();
    // step 3: [Chat_s ; Dtilde_s] with rhs [rC_s ; s_s]; for the tail a second pass over
    // [Chat'_s ; Z_e] with [rC'_s ; z_e] (same R and residual as the QR of the three blocks)
    {
        const Blk<T> F{rec_C(ro), n, rec_E(rs) + n, 2 * n, n};
        const Blk<T> C[1] = {{rec_RC(ro), 1, rec_RE(rs), 1, 1}};
        tpqrt_any<T, L>(n, n, F, C, 1, sm, tc);
    }
    if (triple) {
        const Blk<T> F{rec_C(ro), n, rec_E(re), 2 * n, n};
        const Blk<T> C[1] = {{rec_RC(ro), 1, rec_RE(re), 1, 1}};
        tpqrt_any<T, L>(n, n, F, C, 1, sm, tc);
    }
    if (threadIdx.x < 32) {
        double acc = 0.0;
        for (int r = threadIdx.x; r < n; r += 32) {
            const double v = (double)rec_RE(rs)[r];
            acc = fma(v, v, acc);
            if (triple) {
                const double z = (double)rec_RE(re)[r];
                acc = fma(z, z, acc);
            }
        }
        acc = warp_sum(acc);
        if (threadIdx.x == 0) resid[oj] = acc;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Whitening of step i.
__device__ __forceinline__ int tri_(int r) { return r * (r + 1) / 2; }

// Pivot j of the packed factor L by one warp: square root and reciprocal of L_jj, then column j
// scaled.  A non-positive or non-finite pivot flags ST_NOT_SPD at `step` and is replaced by 1.
__device__ __forceinline__ void chol_pivot_warp(double* L, int d, int j, int lane,
                                                unsigned long long* bad, int64_t step) {
    double ajj = L[tri_(j) + j];
    if (!(ajj > 0.0) || !isfinite(ajj)) {
        if (lane == 0) flag_error(bad, ST_NOT_SPD, step);
        ajj = 1.0;
    }
    const double dj = sqrt(ajj), inv = 1.0 / dj;
    __syncwarp();
    if (lane == 0) L[tri_(j) + j] = dj;
    for (int r = j + 1 + lane; r < d; r += 32) L[tri_(r) + j] *= inv;
    __syncwarp();
}

// Lower Cholesky factor of the d x d matrix held packed (row-major lower) in L, FP64, all
// threads, right-looking with look-ahead: during step j warp 0 updates column j+1 alone, takes
// pivot j+1 and scales that column, while warps 1-7 update the columns >= j+2 of the trailing
// triangle (row r by warp 1 + (r - j - 2) % 7, its columns by the lanes).  One barrier per pivot,
// and the pivot's latency overlaps the trailing update.  Warp 0 alone does the square root and
// reciprocal: an FP64 warp instruction occupies the FP64 pipe whatever its active lanes.  The
// caller synchronises after filling L.
__device__ inline void chol_packed(double* L, int d, unsigned long long* bad, int64_t step) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = NTH / 32;
    if (warp == 0) chol_pivot_warp(L, d, 0, lane, bad, step);
    __syncthreads();
    for (int j = 0; j + 1 < d; ++j) {
        if (warp == 0) {
            const double l1 = L[tri_(j + 1) + j];
            for (int r = j + 1 + lane; r < d; r += 32)
                L[tri_(r) + j + 1] = fma(-L[tri_(r) + j], l1, L[tri_(r) + j + 1]);
            __syncwarp();
            chol_pivot_warp(L, d, j + 1, lane, bad, step);
        } else {
            const int t = d - j - 2;
            for (int rr = warp - 1; rr < t; rr += NW - 1) {
                const int r = j + 2 + rr;
                double* Lr = L + tri_(r);
                const double lrj = Lr[j];
                for (int cc = lane; cc <= rr; cc += 32) {
                    const int c = j + 2 + cc;
                    Lr[c] = fma(-lrj, L[tri_(c) + j], Lr[c]);
                }
            }
        }
        __syncthreads();
    }
}

// X <- L^{-1} X for one column of X (row stride ldx), L packed lower (type T): 32 rows at a
// time in registers.
template <typename T>
__device__ void trsm_column(const T* L, int d, T* X, int64_t ldx) {
    for (int rb = 0; rb < d; rb += 32) {
        T acc[32];
#pragma unroll
        for (int ii = 0; ii < 32; ++ii) acc[ii] = (rb + ii < d) ? X[(int64_t)(rb + ii) * ldx] : T(0);
        // Unrolled so that the loads of the solved values (device memory) are issued in batches.
#pragma unroll 8
        for (int q = 0; q < rb; ++q) {
            const T xq = X[(int64_t)q * ldx];
#pragma unroll
            for (int ii = 0; ii < 32; ++ii)
                if (rb + ii < d) acc[ii] = fma(-L[tri_(rb + ii) + q], xq, acc[ii]);
        }
#pragma unroll
        for (int ii = 0; ii < 32; ++ii) {
            if (rb + ii < d) {
                const T x = acc[ii] / L[tri_(rb + ii) + rb + ii];
                acc[ii] = x;
#pragma unroll
                for (int i2 = ii + 1; i2 < 32; ++i2)
                    if (rb + i2 < d) acc[i2] = fma(-L[tri_(rb + i2) + rb + ii], x, acc[i2]);
            }
        }
#pragma unroll
        for (int ii = 0; ii < 32; ++ii)
            if (rb + ii < d) X[(int64_t)(rb + ii) * ldx] = acc[ii];
    }
}

// The same solve for one contiguous column by a whole warp (lane l holds rows l + 32 s).
template <typename T>
__device__ void trsm_column_warp(const T* L, int d, T* X) {
    const int lane = threadIdx.x & 31;
    T r[PMAX / 32];
#pragma unroll
    for (int s = 0; s < PMAX / 32; ++s) r[s] = (lane + 32 * s < d) ? X[lane + 32 * s] : T(0);
    for (int i = 0; i < d; ++i) {
        T x = T(0);
        if ((i & 31) == lane) {
#pragma unroll
            for (int s = 0; s < PMAX / 32; ++s)
                if ((i >> 5) == s) x = r[s] / L[tri_(i) + i];
        }
        x = __shfl_sync(0xffffffffu, x, i & 31);
#pragma unroll
        for (int s = 0; s < PMAX / 32; ++s) {
            const int ii = lane + 32 * s;
            if (ii > i && ii < d) r[s] = fma(-L[tri_(ii) + i], x, r[s]);
            if (ii == i) r[s] = x;
        }
    }
#pragma unroll
    for (int s = 0; s < PMAX / 32; ++s)
        if (lane + 32 * s < d) X[lane + 32 * s] = r[s];
}

struct WhitenSmem {
    // FP64 packed factor, then its working-precision copy; the QR's buffers overlay both.
    __host__ __device__ static size_t bytes(int n, bool fp32) {
        const size_t tri = (size_t)n * (n + 1) / 2;
        size_t chol = tri * sizeof(double) + (fp32 ? tri * sizeof(float) : 0);
        chol = (chol + 15) & ~(size_t)15;
        const size_t qr = (size_t)QrSmem::TOTAL * (fp32 ? sizeof(float) : sizeof(double));
        return chol > qr ? chol : qr;
    }
};

template <typename T>
__device__ void whiten_step(const WhitenArgs& a, int64_t i, unsigned char* smem, TcState* tc = nullptr) {
    const int n = a.n, tid = threadIdx.x;
    const int64_t nn = (int64_t)n * n, CS = level_cs(n);
    // Above PMAX the packed factors live in this block's slice of the global scratch (the shared
    // memory holds the QR's panel); below, in shared memory.
    double* Lpk = n > PMAX ? reinterpret_cast<double*>(reinterpret_cast<char*>(a.cta_scratch) +
                                                       blockIdx.x * a.cta_scratch_stride)
                           : reinterpret_cast<double*>(smem);
    const int tri = n * (n + 1) / 2;
    T* LT = sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(Lpk) : reinterpret_cast<T*>(Lpk + tri);
    T* out = reinterpret_cast<T*>(a.level0);
    T* rec = out + i * CS;
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
    for (int64_t e = tid; e < nn + n; e += NTH) rec[e] = T(0);   // [Chat_i | rC_i] <- 0
    T* En = out + (i + 1) * CS + nn + n;                         // E_{i+1}: [-B_i | D_i] (n x 2n)
    T* REn = En + 2 * nn;
    if (hasE) {
        const double* Ki = a.K + ti_step(a.ti, TI_K, i) * nn;
        const double* Fi = a.F + ti_step(a.ti, TI_F, i) * nn;
        const double* Hi = a.H + ti_step(a.ti, TI_H, i) * nn;
        for (int64_t e = tid; e < nn; e += NTH) {
            const int r = (int)(e / n), c = (int)(e - (int64_t)r * n);
            if (c <= r) Lpk[tri_(r) + c] = Ki[e];
            En[(int64_t)r * 2 * n + c] = (T)(-Fi[e]);
            En[(int64_t)r * 2 * n + n + c] = (T)Hi[e];
        }
        for (int r = tid; r < n; r += NTH) REn[r] = a.c ? (T)a.c[i * n + r] : T(0);
        __syncthreads();
        chol_packed(Lpk, n, a.bad, i);
        if (a.LK != nullptr) {
            double* lk = a.LK + i * nn;
            for (int64_t e = tid; e < nn; e += NTH) {
                const int r = (int)(e / n), c = (int)(e - (int64_t)r * n);
                lk[e] = c <= r ? Lpk[tri_(r) + c] : 0.0;
            }
        }
        if (sizeof(T) != sizeof(double)) {
            for (int e = tid; e < tri; e += NTH) LT[e] = (T)Lpk[e];
            __syncthreads();
        }
        for (int col = tid; col < 2 * n; col += NTH) trsm_column<T>(LT, n, En + col, 2 * n);
        if (2 * n < NTH) {
            if (tid == 2 * n) trsm_column<T>(LT, n, REn, 1);
        } else if (n > PMAX) {
            if (tid == 0) trsm_column<T>(LT, n, REn, 1);
        } else if (tid < 32) {
            trsm_column_warp<T>(LT, n, REn);
        }
        __syncthreads();
    }
    T* Gm = reinterpret_cast<T*>(a.scratch) + i * (int64_t)n * (n + 1);   // mi x (n + 1)
    if (mi > 0) {
        const double* Ci = a.C + ((a.ti & TI_C) ? 0 : co);
        const double* Gi = a.G + ((a.ti & TI_G) ? 0 : go) * n;
        for (int e = tid; e < mi * mi; e += NTH) {
            const int r = e / mi, c = e - r * mi;
            if (c <= r) Lpk[tri_(r) + c] = Ci[e];
        }
        for (int64_t e = tid; e < (int64_t)mi * n; e += NTH) {
            const int r = (int)(e / n), c = (int)(e - (int64_t)r * n);
            Gm[(int64_t)r * (n + 1) + c] = (T)Gi[e];
        }
        for (int r = tid; r < mi; r += NTH) Gm[(int64_t)r * (n + 1) + n] = (T)a.o[go + r];
        __syncthreads();
        chol_packed(Lpk, mi, a.bad, i);
        if (a.LC != nullptr) {
            for (int e = tid; e < mi * mi; e += NTH) {
                const int r = e / mi, c = e - r * mi;
                a.LC[co + e] = c <= r ? Lpk[tri_(r) + c] : 0.0;
            }
        }
        const int mtri = mi * (mi + 1) / 2;
        if (sizeof(T) != sizeof(double)) {
            T* LTm = reinterpret_cast<T*>(Lpk + mtri);
            for (int e = tid; e < mtri; e += NTH) LTm[e] = (T)Lpk[e];
            __syncthreads();
            for (int col = tid; col <= n; col += NTH) trsm_column<T>(LTm, mi, Gm + col, n + 1);
        } else {
            for (int col = tid; col <= n; col += NTH)
                trsm_column<T>(reinterpret_cast<T*>(Lpk), mi, Gm + col, n + 1);
        }
        __syncthreads();
        // [Chat_i | rC_i] = R of [0 ; L_C^{-1} [G_i | o_i]]
        const Blk<T> F{rec, n, Gm, n + 1, n};
        const Blk<T> C[1] = {{rec + nn, 1, Gm + n, n + 1, 1}};
        tpqrt_any<T>(n, mi, F, C, 1, reinterpret_cast<T*>(smem), tc);
    }
    if (tid < 32) {
        double acc = 0.0;
        for (int r = tid; r < mi; r += 32) {
            const double v = (double)Gm[(int64_t)r * (n + 1) + n];
            acc = fma(v, v, acc);
        }
        acc = warp_sum(acc);
        if (tid == 0) a.resid[i] = acc;
    }
    for (int col = tid; col < n; col += NTH) {
        double sc = 0.0, sb = 0.0, sd = 0.0;
        for (int r = 0; r <= col; ++r) {
            const double v = (double)rec[(int64_t)r * n + col];
            sc = fma(v, v, sc);
        }
        if (hasE) {
            for (int r = 0; r < n; ++r) {
                const double b = (double)En[(int64_t)r * 2 * n + col];
                const double d = (double)En[(int64_t)r * 2 * n + n + col];
                sb = fma(b, b, sb);
                sd = fma(d, d, sd);
            }
            a.cd2[(i + 1) * n + col] = sd;
        }
        a.cn2[i * n + col] = sc + sb;
        if (i == 0) a.cd2[col] = 0.0;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// SelInv: CTA GEMM over row blocks of 32 rows and column tiles of 128, 4 x 4 per thread.
constexpr int GM = 32, GN = 128, GK = 16;

struct SelSmem {
    static size_t bytes(int n, bool fp32) {
        return (size_t)(n * n + GK * GM + GK * GN) * (fp32 ? sizeof(float) : sizeof(double));
    }
};

// C[i][j] (i < M, j < N) = sum_{q = klo(i0) .. K-1} A(i, q) B(q, j), stored by st(i, j, acc) after
// all of the tile's reads; row blocks in ascending order.
template <typename T, typename FA, typename FB, typename FK, typename FS>
__device__ void gemm_rows(int M, int N, int K, FA A, FB B, FK klo, FS st, T* As, T* Bs) {
    const int tid = threadIdx.x;
    const int rg = tid >> 5, cg = tid & 31;
    for (int i0 = 0; i0 < M; i0 += GM) {
        for (int j0 = 0; j0 < N; j0 += GN) {
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
            for (int k0 = klo(i0); k0 < K; k0 += GK) {
                __syncthreads();
                for (int e = tid; e < GK * GM; e += NTH) {
                    const int i = e / GK, kk = e - i * GK;
                    As[kk * GM + i] = (i0 + i < M && k0 + kk < K) ? A(i0 + i, k0 + kk) : T(0);
                }
                for (int e = tid; e < GK * GN; e += NTH) {
                    const int kk = e / GN, jj = e - kk * GN;
                    Bs[kk * GN + jj] = (j0 + jj < N && k0 + kk < K) ? B(k0 + kk, j0 + jj) : T(0);
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < GK; ++kk) {
                    T av[4], bv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) av[a] = As[kk * GM + rg * 4 + a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) bv[b] = Bs[kk * GN + cg * 4 + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = i0 + rg * 4 + a, jx = j0 + cg * 4 + b;
                    if (i < M && jx < N) st(i, jx, acc[a][b]);
                }
        }
    }
    __syncthreads();
}

// Row q of level `level`.  Sx row c = [Sl (n x n) | Sr (n x n)], Sd = covariances (FP64).
template <typename T>
__device__ void selinv_row(int n, int64_t k, int level, int64_t q, const T* __restrict__ R, T* Sx,
                           double* Sd, unsigned long long* bad, T* sm, T* ri_global = nullptr) {
    const int tid = threadIdx.x;
    const int64_t nn = (int64_t)n * n;
    const int64_t c = ((2 * q + 1) << level) - 1;
    if (c >= k) return;
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    const bool ha = a >= 0, hb = b < k;
    int sab_src = 0;   // 1: S_ab = Sr_a, 2: S_ab = Sl_b^T
    if (ha && hb) sab_src = (ctz64(a + 1) == level + 1) ? 1 : 2;
    const T* Rc = R + c * rstore_rs(n);
    const T* Rd = Rc;
    const T* Rl = Rc + nn;
    const T* Rr = Rc + 2 * nn;
    T* Sl = Sx + c * 2 * nn;
    T* Sr = Sl + nn;
    // Rd^{-1}: in shared memory, or (state dimensions above PMAX) in this block's global scratch
    T* Ri = ri_global ? ri_global : sm;
    T* As = ri_global ? sm : sm + nn;
    T* Bs = As + GK * GM;
    double* slot = Sd + c * nn;
    // M and then S_cc share the FP64 covariance slot; in FP32 M sits in its second half so that
    // writing row block I of S_cc (doubles) only overwrites rows of M already consumed -- true
    // while one 128-column tile covers a row block.  Above that (n > GN, where ri_global is
    // given) M gets its own n x n after Rd^{-1} in the block's global slice.
    T* Mx = ri_global ? ri_global + nn
            : sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(slot) : reinterpret_cast<T*>(slot) + nn;

    // Ri = Rd^{-1} (upper triangular), one thread per column.
    for (int64_t e = tid; e < nn; e += NTH) Ri[e] = T(0);
    __syncthreads();
    for (int jc = tid; jc < n; jc += NTH) {
        for (int i = jc; i >= 0; --i) {
            T s = (i == jc) ? T(1) : T(0);
            for (int p = i + 1; p <= jc; ++p) s = fma(-Rd[(int64_t)i * n + p], Ri[(int64_t)p * n + jc], s);
            Ri[(int64_t)i * n + jc] = s / Rd[(int64_t)i * n + i];
        }
    }
    __syncthreads();
    auto Aop = [&](int i, int p) -> T {   // [Rl | Rr]
        return p < n ? (ha ? Rl[(int64_t)i * n + p] : T(0)) : (hb ? Rr[(int64_t)i * n + p - n] : T(0));
    };
    auto Sab = [&](int r, int cc) -> T {  // S_{a,b}
        if (sab_src == 1) return Sx[a * 2 * nn + nn + (int64_t)r * n + cc];
        if (sab_src == 2) return Sx[b * 2 * nn + (int64_t)cc * n + r];
        return T(0);
    };
    auto Sii = [&](int p, int qq) -> T {
        if (p < n) {
            if (qq < n) return ha ? (T)Sd[a * nn + (int64_t)p * n + qq] : T(0);
            return Sab(p, qq - n);
        }
        if (qq < n) return Sab(qq, p - n);
        return hb ? (T)Sd[b * nn + (int64_t)(p - n) * n + (qq - n)] : T(0);
    };
    auto k0 = [](int) { return 0; };
    // P = A S_II -> [Sl | Sr]
    gemm_rows<T>(n, 2 * n, 2 * n, Aop, Sii, k0,
                 [&](int i, int j, T v) { if (j < n) Sl[(int64_t)i * n + j] = v; else Sr[(int64_t)i * n + j - n] = v; },
                 As, Bs);
    // [Sl | Sr] = -Ri P (in place; row block i0 reads rows >= i0 only)
    auto Pop = [&](int p, int j) -> T { return j < n ? Sl[(int64_t)p * n + j] : Sr[(int64_t)p * n + j - n]; };
    gemm_rows<T>(n, 2 * n, n, [&](int i, int p) -> T { return Ri[(int64_t)i * n + p]; }, Pop,
                 [](int i0) { return (i0 / GK) * GK; },
                 [&](int i, int j, T v) { if (j < n) Sl[(int64_t)i * n + j] = -v; else Sr[(int64_t)i * n + j - n] = -v; },
                 As, Bs);
    // M = Ri - [Sl | Sr] A^T
    gemm_rows<T>(n, n, 2 * n, Pop, [&](int p, int j) -> T { return Aop(j, p); }, k0,
                 [&](int i, int j, T v) { Mx[(int64_t)i * n + j] = Ri[(int64_t)i * n + j] - v; }, As, Bs);
    // S_cc = M Ri^T, row block by row block in place (doubles)
    gemm_rows<T>(n, n, n, [&](int i, int p) -> T { return Mx[(int64_t)i * n + p]; },
                 [&](int p, int j) -> T { return Ri[(int64_t)j * n + p]; }, k0,
                 [&](int i, int j, T v) { slot[(int64_t)i * n + j] = (double)v; }, As, Bs);
    // symmetrise, check the diagonal
    for (int64_t e = tid; e < nn; e += NTH) {
        const int r = (int)(e / n), cc = (int)(e - (int64_t)r * n);
        if (r < cc) {
            const double v = 0.5 * (slot[(int64_t)r * n + cc] + slot[(int64_t)cc * n + r]);
            slot[(int64_t)r * n + cc] = v;
            slot[(int64_t)cc * n + r] = v;
        } else if (r == cc) {
            const T v = (T)slot[e];
            if (!(v > T(0))) flag_error(bad, ST_SINGULAR, c);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// SelInv on the tensor cores (FP32, state dimensions up to PMAX).  The four products of the
// reordered Algorithm 2 (see selinv_row) are dense contractions with M = n <= 128 output rows:
//     P = [Rl | Rr] S_II           K = 2n, N = 2n
//     [Sl | Sr] = -Ri P            K = n,  N = 2n
//     M = Ri - [Sl | Sr] [Rl | Rr]^T   K = 2n, N = n
//     S_cc = M Ri^T                K = n,  N = n
// Each runs as 3xTF32 tcgen05 MMAs (M = 128, N = the product's width rounded up to 16, K steps
// of 8) with the FP32 accumulator in TMEM.  Both operands are staged through shared memory in
// K-chunks of SKC: every thread converts four consecutive K elements of one operand row to a
// TF32 hi part and an FP32 lo remainder and stores them as 16-byte pieces of the K-major tiles
// (ks_tc.cuh).  The MMAs of a chunk complete (bounded mbarrier wait) before the next chunk
// overwrites the tiles; two blocks per SM (256 TMEM columns each) overlap one block's staging
// with the other's MMAs.  The whole product is in TMEM before its epilogue writes anything, so
// a product may overwrite its own operand (P -> [Sl | Sr]).
constexpr int SKC = 16;                    // K per staged chunk
constexpr uint32_t SEL_TM_COLS = 256;      // TMEM columns per block (N <= 256)
struct SelTcSmem {                         // byte offsets
    static constexpr int RI = 0;                                 // Rd^{-1}, PMAX x PMAX floats
    static constexpr int A = RI + PMAX * PMAX * 4;               // 128 x SKC, hi | lo
    static constexpr int B = A + 2 * 128 * SKC * 4;              // 256 x SKC, hi | lo
    static constexpr int MBAR = B + 2 * 256 * SKC * 4;
    static constexpr int SLOT = MBAR + 8;
    static constexpr int ABORT = SLOT + 4;
    static constexpr int BYTES = ABORT + 4;
};

struct SelTc {
    unsigned char* smem;
    uint32_t tmem, phase;
    unsigned long long* bad;
};

__device__ inline void sel_tc_setup(SelTc& st, unsigned char* smem, unsigned long long* bad) {
    st.smem = smem;
    st.phase = 0;
    st.bad = bad;
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + SelTcSmem::SLOT);
    if (threadIdx.x < 32) {
        tc::tmem_alloc(slot, SEL_TM_COLS);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(reinterpret_cast<uint64_t*>(smem + SelTcSmem::MBAR), 1);
        *reinterpret_cast<int*>(smem + SelTcSmem::ABORT) = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    st.tmem = *slot;
}

__device__ inline void sel_tc_teardown(SelTc& st) {
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(st.tmem, SEL_TM_COLS);
}

// Rows [0, R) x K-chunk [k0, k0 + SKC) of an operand, element (row, kk) = get(row, kk), as the
// hi | lo tiles at dst.  Unit u: four consecutive kk of one row; the eight units of a
// quarter-warp take eight consecutive rows of the same kk group (distinct 16-byte bank groups).
template <typename F>
__device__ __forceinline__ void sel_stage(unsigned char* dst, int R, int k0, F get) {
    constexpr int G = SKC / 4;
    float* hi = reinterpret_cast<float*>(dst);
    float* lo = reinterpret_cast<float*>(dst + R * SKC * 4);
    for (int u = threadIdx.x; u < R * G; u += NTH) {
        const int rl = u & 7, g = (u >> 3) % G, row = ((u >> 3) / G) * 8 + rl;
        float4 h, l;
        const float x0 = get(row, k0 + 4 * g), x1 = get(row, k0 + 4 * g + 1);
        const float x2 = get(row, k0 + 4 * g + 2), x3 = get(row, k0 + 4 * g + 3);
        h.x = tc::tf32_hi(x0); l.x = x0 - h.x;
        h.y = tc::tf32_hi(x1); l.y = x1 - h.y;
        h.z = tc::tf32_hi(x2); l.z = x2 - h.z;
        h.w = tc::tf32_hi(x3); l.w = x3 - h.w;
        const uint32_t o = tc::tile_off(R, row, 4 * g) >> 2;
        *reinterpret_cast<float4*>(hi + o) = h;
        *reinterpret_cast<float4*>(lo + o) = l;
    }
}

// D (TMEM columns [0, NP)) = sum_{kk < K} A(i, kk) B(kk, j) for the 128 rows i and NP columns j
// (NP a multiple of 16, <= 256).  A(i, kk) and B(kk, j) must return 0 outside the product.
// Whole block.
template <typename FA, typename FB>
__device__ void sel_tc_gemm(int K, int NP, FA A, FB B, SelTc& st) {
    int* abort = reinterpret_cast<int*>(st.smem + SelTcSmem::ABORT);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(st.smem + SelTcSmem::MBAR);
    unsigned char* As = st.smem + SelTcSmem::A;
    unsigned char* Bs = st.smem + SelTcSmem::B;
    const uint32_t idesc = tc::idesc_tf32(128, NP);
    for (int k0 = 0; k0 < K; k0 += SKC) {
        sel_stage(As, 128, k0, [&](int i, int kk) { return kk < K ? A(i, kk) : 0.f; });
        sel_stage(Bs, NP, k0, [&](int j, int kk) { return kk < K ? B(kk, j) : 0.f; });
        tc::fence_proxy_async_smem();
        tc::fence_before();
        __syncthreads();
        if (threadIdx.x == 0 && !*abort) {
            tc::fence_after();
            const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
            const uint32_t alo = 128 * SKC * 4, blo = (uint32_t)NP * SKC * 4;
            for (int s = 0; s < SKC / 8; ++s) {
                const uint64_t ah = tc::tile_desc(a0, 128, s), al = tc::tile_desc(a0 + alo, 128, s);
                const uint64_t bh = tc::tile_desc(b0, NP, s), bl = tc::tile_desc(b0 + blo, NP, s);
                const uint32_t first = (k0 == 0 && s == 0) ? 0u : 1u;
                tc::mma_ss(st.tmem, ah, bl, idesc, first);
                tc::mma_ss(st.tmem, al, bh, idesc, 1u);
                tc::mma_ss(st.tmem, ah, bh, idesc, 1u);
            }
            tc::commit(mbar);
        }
        bool ok = true;
        if (!*abort) ok = tc::mbar_wait(mbar, st.phase, TC_WAIT_LIMIT);
        st.phase ^= 1u;
        if (__syncthreads_or(!ok) && threadIdx.x == 0) {
            if (!*abort && st.bad != nullptr) flag_error(st.bad, ST_TIMEOUT, 0);
            *abort = 1;
        }
        tc::fence_after();
    }
}

// Epilogue: store(i, j, D[i][j]) for i < M, j < N.  Warp w reads the TMEM lanes of rows
// 32 (w % 4) .. + 31; the two warps of a lane quarter take alternate 32-column blocks.
template <typename FS>
__device__ void sel_tc_store(int M, int N, int NP, FS store, SelTc& st) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = 32 * (warp & 3) + lane, half = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    for (int cb = 32 * half; cb < NP; cb += 64) {
        float v[32];
        tc::tmem_ld32(st.tmem + lanes + (uint32_t)cb, v);
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int j = cb + t;
            if (i < M && j < N) store(i, j, v[t]);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// C = A B for M x N outputs and K terms as 128-row by 256-column tiles, each one product in
// TMEM and one epilogue; store(i, j, v) receives every output.  upper: A is upper triangular
// (A(i, kk) = 0 for kk < i), so row tile r0 starts its K range at r0.  The tiles of a row tile
// are stored before the next row tile is computed; with `upper` a product may therefore
// overwrite its B operand in place row tile by row tile (row tile r0 reads rows >= r0 of B).
template <typename FA, typename FB, typename FS>
__device__ void sel_tc_product(int M, int N, int K, FA A, FB B, FS store, SelTc& st, bool upper) {
    for (int r0 = 0; r0 < M; r0 += 128) {
        const int klo = upper ? r0 : 0;
        for (int c0 = 0; c0 < N; c0 += 256) {
            const int nw = (N - c0) < 256 ? (N - c0) : 256;
            const int NP = (nw + 15) & ~15;
            sel_tc_gemm(K - klo, NP, [&](int i, int kk) { return A(r0 + i, klo + kk); },
                        [&](int kk, int j) { return B(klo + kk, c0 + j); }, st);
            sel_tc_store((M - r0) < 128 ? (M - r0) : 128, nw, NP,
                         [&](int i, int j, float v) { store(r0 + i, c0 + j, v); }, st);
        }
    }
}

// Row q of level `level` with the products on the tensor cores (see selinv_row for the data).
// Above PMAX (ri_global != nullptr) Rd^{-1} and M live in this block's global slice and every
// product is tiled by sel_tc_product.
__device__ inline void selinv_row_tc(int n, int64_t k, int level, int64_t q, const float* __restrict__ R,
                                     float* Sx, double* Sd, unsigned long long* bad, SelTc& st,
                                     float* ri_global = nullptr) {
    const int tid = threadIdx.x;
    const int64_t nn = (int64_t)n * n;
    const int64_t c = ((2 * q + 1) << level) - 1;
    if (c >= k) return;
    const int64_t a = c - (1LL << level), b = c + (1LL << level);
    const bool ha = a >= 0, hb = b < k;
    int sab_src = 0;   // 1: S_ab = Sr_a, 2: S_ab = Sl_b^T
    if (ha && hb) sab_src = (ctz64(a + 1) == level + 1) ? 1 : 2;
    const float* Rc = R + c * rstore_rs(n);
    const float* Rd = Rc;
    const float* Rl = Rc + nn;
    const float* Rr = Rc + 2 * nn;
    float* Sl = Sx + c * 2 * nn;
    float* Sr = Sl + nn;
    float* Ri = ri_global ? ri_global : reinterpret_cast<float*>(st.smem + SelTcSmem::RI);
    double* slot = Sd + c * nn;
    // M: in the second half of the FP64 slot (n <= PMAX; S_cc is stored only after all of M is
    // read), else after Rd^{-1} in the global slice
    float* Mx = ri_global ? ri_global + nn : reinterpret_cast<float*>(slot) + nn;

    // Ri = Rd^{-1} (upper triangular), one thread per column.
    for (int64_t e = tid; e < nn; e += NTH) Ri[e] = 0.f;
    __syncthreads();
    for (int jc = tid; jc < n; jc += NTH) {
        for (int i = jc; i >= 0; --i) {
            float s = (i == jc) ? 1.f : 0.f;
            for (int p = i + 1; p <= jc; ++p) s = fmaf(-Rd[(int64_t)i * n + p], Ri[p * n + jc], s);
            Ri[i * n + jc] = s / Rd[(int64_t)i * n + i];
        }
    }
    __syncthreads();
    auto Aop = [&](int i, int p) -> float {   // [Rl | Rr], zero outside n x 2n
        if (i >= n) return 0.f;
        if (p < n) return ha ? Rl[(int64_t)i * n + p] : 0.f;
        return (p < 2 * n && hb) ? Rr[(int64_t)i * n + p - n] : 0.f;
    };
    auto Sab = [&](int r, int cc) -> float {
        if (sab_src == 1) return Sx[a * 2 * nn + nn + (int64_t)r * n + cc];
        if (sab_src == 2) return Sx[b * 2 * nn + (int64_t)cc * n + r];
        return 0.f;
    };
    auto Sii = [&](int p, int qq) -> float {   // 2n x 2n, zero outside
        if (p >= 2 * n || qq >= 2 * n) return 0.f;
        if (p < n) {
            if (qq < n) return ha ? (float)Sd[a * nn + (int64_t)p * n + qq] : 0.f;
            return Sab(p, qq - n);
        }
        if (qq < n) return Sab(qq, p - n);
        return hb ? (float)Sd[b * nn + (int64_t)(p - n) * n + (qq - n)] : 0.f;
    };
    auto SlSr = [&](int i, int j) -> float {   // [Sl | Sr], zero outside n x 2n
        if (i >= n || j >= 2 * n) return 0.f;
        return j < n ? Sl[(int64_t)i * n + j] : Sr[(int64_t)i * n + j - n];
    };
    auto put = [&](int i, int j, float v) {
        if (j < n) Sl[(int64_t)i * n + j] = v; else Sr[(int64_t)i * n + j - n] = v;
    };
    const int N2 = 2 * n;
    // P = [Rl | Rr] S_II -> [Sl | Sr]
    sel_tc_product(n, N2, N2, Aop, Sii, put, st, false);
    // [Sl | Sr] = -Ri P, in place (Ri upper triangular)
    sel_tc_product(n, N2, n, [&](int i, int p) { return (i < n && p < n) ? Ri[i * n + p] : 0.f; }, SlSr,
                   [&](int i, int j, float v) { put(i, j, -v); }, st, true);
    // M = Ri - [Sl | Sr] [Rl | Rr]^T
    sel_tc_product(n, n, N2, SlSr, [&](int p, int j) { return Aop(j, p); },
                   [&](int i, int j, float v) { Mx[(int64_t)i * n + j] = Ri[i * n + j] - v; }, st, false);
    // S_cc = M Ri^T (doubles into the slot; all of M is read before S_cc is stored)
    sel_tc_product(n, n, n, [&](int i, int p) { return (i < n && p < n) ? Mx[(int64_t)i * n + p] : 0.f; },
                   [&](int p, int j) { return (p < n && j < n) ? Ri[j * n + p] : 0.f; },
                   [&](int i, int j, float v) { slot[(int64_t)i * n + j] = (double)v; }, st, false);
    // symmetrise, check the diagonal
    for (int64_t e = tid; e < nn; e += NTH) {
        const int r = (int)(e / n), cc = (int)(e - (int64_t)r * n);
        if (r < cc) {
            const double v = 0.5 * (slot[(int64_t)r * n + cc] + slot[(int64_t)cc * n + r]);
            slot[(int64_t)r * n + cc] = v;
            slot[(int64_t)cc * n + r] = v;
        } else if (r == cc) {
            if (!(slot[e] > 0.0)) flag_error(bad, ST_SINGULAR, c);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// tc_off >= 0 (FP32 only): byte offset of the tensor-core region in shared memory; the block
// then holds TMEM for its whole life.  tc_off < 0: CUDA-core trailing updates.
template <typename T>
__global__ void __launch_bounds__(NTH) whiten_k(WhitenArgs a, int tc_off) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcState tcs;
    TcState* tc = nullptr;
    if (sizeof(T) == 4 && tc_off >= 0) {
        tc_setup(tcs, smem_raw + tc_off, a.bad);
        tc = &tcs;
    }
    for (int64_t i = blockIdx.x; i < a.k; i += gridDim.x) whiten_step<T>(a, i, smem_raw, tc);
    if (tc != nullptr) tc_teardown(tcs);
}

template <typename T>
__global__ void __launch_bounds__(NTH) level_k(int n, int64_t nc, int level, T* in, T* out, T* R,
                                               double* resid, const double* cn2, const double* cd2,
                                               unsigned long long* bad, int tc_off, int stall) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcState tcs;
    TcState* tc = nullptr;
    if (sizeof(T) == 4 && tc_off >= 0) {
        tc_setup(tcs, smem_raw + tc_off, bad, stall);
        tc = &tcs;
    }
    for (int64_t t = blockIdx.x; t < nc / 2; t += gridDim.x)
        level_tile<T>(n, nc, level, t, in, out, R, resid, cn2, cd2, bad, reinterpret_cast<T*>(smem_raw), tc);
    if (tc != nullptr) tc_teardown(tcs);
}

template <typename T>
__global__ void __launch_bounds__(NTH) selinv_k(int n, int64_t k, int level, const T* R, T* Sx,
                                                double* Sd, unsigned long long* bad, T* ri_scratch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t rows = (k >> level) - (k >> (level + 1));
    T* ri = ri_scratch ? ri_scratch + blockIdx.x * 2 * (int64_t)n * n : nullptr;   // Rd^{-1}, M
    for (int64_t q = blockIdx.x; q < rows; q += gridDim.x)
        selinv_row<T>(n, k, level, q, R, Sx, Sd, bad, reinterpret_cast<T*>(smem_raw), ri);
}

template <typename T, int OP>
__global__ void __launch_bounds__(NTH) batch_k(const BatchWork* wk, int tc_off) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchWork w = *wk;
    const int64_t total = w.off[w.np];
    TcState tcs;
    TcState* tc = nullptr;
    if (sizeof(T) == 4 && OP != B_SELINV && tc_off >= 0) {
        tc_setup(tcs, smem_raw + tc_off, w.np > 0 ? w.desc[w.probs[0]].bad : nullptr);
        tc = &tcs;
    }
    for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
        const int pi = batch_find(w.off, w.np, u);
        const ProbDesc& P = w.desc[w.probs[pi]];
        const int64_t x = u - w.off[pi];
        const int l = work_level(w, P);
        if (tc != nullptr) tc->bad = P.bad;
        if constexpr (OP == B_WHITEN) {
            whiten_step<T>(whiten_args_of(P), x, smem_raw, tc);
        } else if constexpr (OP == B_LEVEL) {
            level_tile<T>(P.n, P.k >> l, l, x, reinterpret_cast<T*>(P.lvl[l & 1]),
                          reinterpret_cast<T*>(P.lvl[(l + 1) & 1]), reinterpret_cast<T*>(P.R), P.resid,
                          P.cn2, P.cd2, P.bad, reinterpret_cast<T*>(smem_raw), tc);
        } else {
            selinv_row<T>(P.n, P.k, l, x, reinterpret_cast<const T*>(P.R), reinterpret_cast<T*>(P.Sx),
                          P.cov, P.bad, reinterpret_cast<T*>(smem_raw));
        }
    }
    if (tc != nullptr) tc_teardown(tcs);
}

// ---- host helpers of the launchers ----
inline unsigned grid_of(int64_t units, int per_sm) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int64_t g = (int64_t)sms * per_sm;
    return (unsigned)(units < g ? (units < 1 ? 1 : units) : g);
}

template <typename K>
inline void set_smem(K kern, size_t bytes) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline size_t qr_bytes(bool fp32) { return (size_t)QrSmem::TOTAL * (fp32 ? sizeof(float) : sizeof(double)); }

// Whether the FP32 kernels use the tensor cores (KS_NO_TC=1 selects the CUDA-core updates).
inline bool tc_enabled() {
    const char* v = getenv("KS_NO_TC");
    return !(v && *v && *v != '0');
}
// Test-only: KS_TEST_STALL_TC=1 makes the tensor-core level kernels take the stall mode.
inline int tc_stall_test() {
    const char* v = getenv("KS_TEST_STALL_TC");
    return (v && *v && *v != '0') ? 1 : 0;
}
// Blocks per SM of the FP32 tensor-core level kernel: 1 (the whole TMEM held for the block's
// life; the default) or 2 (KS_TC_BLOCKS=2: compact layout, TMEM per trailing update).  Two
// blocks per SM measured slower at n = 128 (81 against 68 ms for the level phase of k = 10^4):
// the in-place records of one tile take about 0.8 MB, so 152 tiles in flight already fill the
// 129 MB L2, and 304 spill to HBM.
inline int tc_blocks_per_sm() {
    const char* v = getenv("KS_TC_BLOCKS");
    return (v && *v == '2') ? 2 : 1;
}
// Shared memory of an FP32 kernel whose own layout takes `base` bytes: the tensor-core region
// follows at tc_align(base); *off receives that offset (-1 without tensor cores).
inline size_t with_tc(size_t base, bool fp32, int* off) {
    if (!fp32 || !tc_enabled()) {
        *off = -1;
        return base;
    }
    *off = (int)tc_align(base);
    return tc_align(base) + TcSmem::BYTES;
}
}  // namespace large
}  // namespace ks

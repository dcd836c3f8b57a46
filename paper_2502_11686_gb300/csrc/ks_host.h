// ks_host.h -- private host-side definitions shared by the C-ABI sources (context, factor
// handle, work memory, status words, phase timing).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "../../include/ks.h"
#include "ks_internal.cuh"

using namespace ks;


struct ks_fac {
    int64_t k = 0;
    int n = 0;
    int precision = 0;
    const SmallOps* small = nullptr;  // small-state path (element-major layouts) or generic
    void* R = nullptr;        // R store, k records of 3n^2+n elements (T)
    double* resid = nullptr;  // [2k]: residual parts of the level tiles and of the whitening
    int var_N = 0;                // ks_smooth_var: padded dimension (0 = a uniform problem)
    std::vector<int32_t> var_nd;  // ks_smooth_var: the caller's state dimensions n_i
};

struct ks_ctx {
    int device = 0;
    int precision = KS_FP64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    int sync = 1;
    std::string err;
    unsigned long long* d_bad = nullptr;
    unsigned long long* h_bad = nullptr;  // pinned
    double* h_scalar = nullptr;           // pinned
    void* ws = nullptr;
    size_t ws_size = 0;
    std::set<ks_fac*> facs;
    int smem_optin = 0;
    int profile = 0;
    ks_profile prof{};
    struct Pending { int phase; cudaEvent_t a, b; };
    std::vector<Pending> pending;     // recorded phase events not yet read
    std::vector<cudaEvent_t> spare;   // event pool
    // batched form
    std::string tune_cache;                          // file of tuned launch shapes ("" = none)
    std::map<std::string, int> tuned;                // class signature -> blocks per SM
    bool tune_loaded = false;
    void* bmeta = nullptr;                           // descriptors + work lists (fixed address)
    size_t bmeta_size = 0;
    std::map<std::string, cudaGraphExec_t> graphs;   // batch shape -> replayable launch graph
    std::set<std::string> shapes_seen;               // shapes already run once eagerly
    // variable state dimensions (ks_smooth_var): offsets, padded inputs and outputs
    void* vbuf = nullptr;
    size_t vbuf_size = 0;
    // Host inputs of ks_smooth are copied on `cin` into one of two staging buffers, so the copy
    // for the next call runs while this call's kernels run.  `ready` (on cin) orders the
    // kernels after the copy; `free` (on the ctx's stream, after the last kernel that reads the
    // inputs) orders the copy of the call after next after them.
    cudaStream_t cin = nullptr;
    struct Stage {
        void* p = nullptr;
        size_t size = 0;
        cudaEvent_t ready = nullptr, free = nullptr;
    };
    Stage in_stage[2];
    int in_next = 0;
    // ks_gauss_newton: linearizations, damped observation blocks, corrections
    void* gbuf = nullptr;
    size_t gbuf_size = 0;
};

namespace kshost {

constexpr int KS_NMAX_API = HUGE_NMAX;

inline ks_status fail(ks_ctx* ctx, ks_status s, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

#define KS_CUDA(ctx, call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? KS_ERR_OOM : KS_ERR_CUDA,  \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                   \
    } while (0)

inline bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Bump allocator over the ctx workspace (256-byte aligned pieces).
struct Plan {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    }
};

inline ks_status reserve(ks_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_size) return KS_OK;
    const size_t staged = ctx->in_stage[0].size + ctx->in_stage[1].size;
    if (ctx->budget && bytes + staged > ctx->budget)
        return fail(ctx, KS_ERR_OOM, "work memory %zu bytes exceeds the ctx budget %zu", bytes, ctx->budget);
    KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
    KS_CUDA(ctx, cudaMalloc(&ctx->ws, bytes));
    ctx->ws_size = bytes;
    return KS_OK;
}

inline int tile_smem_bytes(int n, bool fp32) { return tile_layout(n).total * (fp32 ? 4 : 8); }
inline int selinv_smem_bytes(int n, bool fp32) { return selinv_layout(n).total * (fp32 ? 4 : 8); }
inline int whiten_smem_bytes(int n, int m) { return whiten_layout(n, m).total * 8; }

inline int max_n_for(const ks_ctx* ctx) {
    const bool fp32 = ctx->precision == KS_FP32_REFINE;
    int best = 0;
    for (int n = 1; n <= KS_NMAX_API; ++n) {
        if (use_large(n, fp32)) {   // one thread block per unit, records in place
            if ((int)large_smem_bytes(n, fp32) > ctx->smem_optin) break;
            best = n;
            continue;
        }
        if (3 * n + 2 > 256) break;
        if (tile_smem_bytes(n, fp32) > ctx->smem_optin) break;
        if (selinv_smem_bytes(n, fp32) > ctx->smem_optin) break;
        if (whiten_smem_bytes(n, 0) > ctx->smem_optin) break;
        best = n;
    }
    return best;
}

inline int max_m_for(const ks_ctx* ctx, int n) {
    if (use_large(n, ctx->precision == KS_FP32_REFINE)) return n;
    int best = n;   // m <= n: the large-state whitening covers what the column-owner one cannot
    if ((int)large_smem_bytes(n, ctx->precision == KS_FP32_REFINE) > ctx->smem_optin) best = -1;
    for (int m = 0; m <= KS_NMAX_API; ++m) {
        if (n + m > 256) break;
        if (whiten_smem_bytes(n, m) > ctx->smem_optin) break;
        if (m > best) best = m;
    }
    return best;
}

// Input staging buffer number `b` of at least `bytes` bytes, with its events and the copy
// stream (created on first use).  Growing it waits for everything that may still use it.
inline ks_status stage_reserve(ks_ctx* ctx, int b, size_t bytes) {
    ks_ctx::Stage& s = ctx->in_stage[b];
    if (!ctx->cin) KS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cin, cudaStreamNonBlocking));
    if (!s.ready) KS_CUDA(ctx, cudaEventCreateWithFlags(&s.ready, cudaEventDisableTiming));
    if (!s.free) KS_CUDA(ctx, cudaEventCreateWithFlags(&s.free, cudaEventDisableTiming));
    if (bytes <= s.size) return KS_OK;
    size_t held = ctx->ws_size + ctx->in_stage[b ^ 1].size;
    if (ctx->budget && held + bytes > ctx->budget)
        return fail(ctx, KS_ERR_OOM, "staging %zu bytes of host inputs exceeds the ctx budget %zu", bytes, ctx->budget);
    KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    KS_CUDA(ctx, cudaStreamSynchronize(ctx->cin));
    if (s.p) cudaFree(s.p);
    s.p = nullptr;
    s.size = 0;
    KS_CUDA(ctx, cudaMalloc(&s.p, bytes));
    s.size = bytes;
    return KS_OK;
}

// Reads the device error words and resets them; returns the most severe code.
inline ks_status collect_status(ks_ctx* ctx, int64_t* info) {
    KS_CUDA(ctx, cudaMemcpyAsync(ctx->h_bad, ctx->d_bad, sizeof(unsigned long long) * ST_NCODES,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    KS_CUDA(ctx, cudaMemsetAsync(ctx->d_bad, 0xFF, sizeof(unsigned long long) * ST_NCODES, ctx->stream));
    for (int code : status_order) {
        if (ctx->h_bad[code] != ~0ULL) {
            if (info) *info = (int64_t)ctx->h_bad[code];
            return fail(ctx, (ks_status)code, "%s %lld", status_message(code), (long long)ctx->h_bad[code]);
        }
    }
    if (info) *info = -1;
    return KS_OK;
}

inline cudaEvent_t get_event(ks_ctx* ctx) {
    if (!ctx->spare.empty()) {
        cudaEvent_t e = ctx->spare.back();
        ctx->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets the launches of one phase: counts them and, with profiling on, records a pair of
// events on the ctx's stream around them.
struct Phase {
    ks_ctx* ctx;
    int phase;
    uint64_t l0;
    cudaEvent_t a = nullptr;
    Phase(ks_ctx* c, int ph) : ctx(c), phase(ph), l0(t_launches) {
        if (ctx->profile) {
            a = get_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~Phase() {
        const uint64_t nl = t_launches - l0;
        ctx->prof.launches += nl;
        ctx->prof.phase_launches[phase] += nl;
        if (ctx->profile && a) {
            cudaEvent_t b = get_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->pending.push_back({phase, a, b});
        }
    }
};

inline void drain_profile(ks_ctx* ctx) {
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->prof.phase_ms[p.phase] += ms;
        cudaGetLastError();
        ctx->spare.push_back(p.a);
        ctx->spare.push_back(p.b);
    }
    ctx->pending.clear();
}

}  // namespace kshost

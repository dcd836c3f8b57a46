// ks_static.cu -- ks_smooth_static: smoothing for callers that cannot allocate device memory.
//
// Who needs it: code that runs where device allocation is not allowed or not affordable -- a
// plugin inside a host application that owns the whole device-memory budget, or a real-time
// loop that must never wait on the allocator (cudaMalloc can block for a long time and cudaFree
// synchronizes the device).  Such a caller passes its inputs and outputs; everything else the
// smoother needs lives in g_scratch below, one fixed array of KS_STATIC_SCRATCH_BYTES bytes
// compiled into the library.  Every GPU that loads libks.so holds that array until the process
// exits.  No ks_ctx is involved, and nothing here calls cudaMalloc, cudaFree or any other
// allocating routine.
//
// Host code cannot use g_scratch's name as a device address (on the host it is only a stand-in
// symbol), so the first call on each device looks the address up with cudaGetSymbolAddress, with
// that device current, and caches it; the kernels receive that pointer.  All calls share the
// array and find the previous call's data in it: the parts that must start from a known value
// (error words, residual slots) are cleared on every call, and two calls that overlap on the GPU
// race.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/ks.h"
#include "ks_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_scratch[KS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

ks_status report(char* err, size_t len, ks_status s, const char* fmt, ...) {
    if (err && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, len, fmt, ap);
        va_end(ap);
    }
    return s;
}

bool on_device(const void* p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
           at.device == device;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" ks_status ks_smooth_static(int device, void* stream, int64_t k, int n, int m,
                                      const double* F, const double* H, const double* c,
                                      const double* K, const double* G, const double* o,
                                      const double* C, double* u_out, double* cov_out,
                                      int64_t* info, char* err, size_t err_len) {
    using namespace ks;
    if (info) *info = -1;
    if (err && err_len) err[0] = '\0';
    if (device < 0 || device >= kMaxDevices)
        return report(err, err_len, KS_ERR_ARG, "device %d out of range", device);
    if (k < 1) return report(err, err_len, KS_ERR_ARG, "k must be >= 1 (got %lld)", (long long)k);
    if (n < 1 || n > SMALL_NMAX)
        return report(err, err_len, KS_ERR_ARG, "n = %d outside [1, %d]", n, SMALL_NMAX);
    if (m < 0 || m > n) return report(err, err_len, KS_ERR_ARG, "m = %d outside [0, n = %d]", m, n);

    // Work memory of this call, carved from the static array.
    const size_t nt = (size_t)n * (n + 1) / 2;
    const size_t cs = nt + 2 * (size_t)n + 2 * (size_t)n * n;   // level record
    const size_t rs = nt + 2 * (size_t)n * n + n;               // R record
    const size_t ss = 2 * (size_t)n * n;                        // SelInv record
    // Every state needs at least one level record and one R record, so a k above this bound
    // cannot fit; rejecting it first also keeps the byte counts below from overflowing.
    const int64_t k_fit = (int64_t)(KS_STATIC_SCRATCH_BYTES / (sizeof(double) * (cs + rs)));
    if (k > k_fit)
        return report(err, err_len, KS_ERR_ARG,
                      "k = %lld, n = %d needs more work memory than the %zu bytes of the static "
                      "scratch array (at most %lld states at this n); use ks_smooth for this size",
                      (long long)k, n, (size_t)KS_STATIC_SCRATCH_BYTES, (long long)k_fit);
    size_t off = 0;
    const size_t o_bad = off; off += round256(sizeof(unsigned long long) * ST_NCODES);
    const size_t o_a = off;   off += round256((size_t)k * cs * sizeof(double));
    const size_t o_b = off;   off += round256((size_t)(k / 2 + 1) * cs * sizeof(double));
    const size_t o_r = off;   off += round256((size_t)k * rs * sizeof(double));
    const size_t o_res = off; off += round256((size_t)2 * k * sizeof(double));
    const size_t o_cn = off;  off += round256((size_t)k * n * sizeof(double));
    const size_t o_cd = off;  off += round256((size_t)k * n * sizeof(double));
    const size_t o_s = off;   if (cov_out) off += round256((size_t)k * ss * sizeof(double));
    if (off > (size_t)KS_STATIC_SCRATCH_BYTES)
        return report(err, err_len, KS_ERR_ARG,
                      "k = %lld, n = %d%s needs %zu bytes of work memory, more than the %zu bytes "
                      "of the static scratch array; use ks_smooth for this size",
                      (long long)k, n, cov_out ? " with covariances" : "", off,
                      (size_t)KS_STATIC_SCRATCH_BYTES);

    const bool need_evo = k > 1, need_obs = m > 0;
    if (!u_out || (need_evo && (!F || !H || !K)) || (need_obs && (!G || !o || !C)))
        return report(err, err_len, KS_ERR_ARG, "a required array pointer is NULL");
    const void* ptrs[] = {F, H, c, K, G, o, C, u_out, cov_out};
    for (const void* p : ptrs)
        if (p && !on_device(p, device))
            return report(err, err_len, KS_ERR_ARG,
                          "every array must be device memory of device %d (got %p)", device, p);

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return report(err, err_len, KS_ERR_CUDA, "cudaGetDevice failed");
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return report(err, err_len, KS_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    }
    struct Restore {
        int dev;
        ~Restore() { if (dev >= 0) cudaSetDevice(dev); }
    } restore{prev};

    // One-time set-up per device: the device address of g_scratch.
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_addr[device] == nullptr) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || p == nullptr)
                return report(err, err_len, KS_ERR_CUDA, "cudaGetSymbolAddress failed: %s",
                              cudaGetErrorString(e));
            g_addr[device] = p;
        }
        base = g_addr[device];
    }
    char* ws = static_cast<char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The call ends by waiting for its own work on `stream`; a wait inside a stream capture
    // would invalidate the caller's capture, so a capturing stream is refused up front.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return report(err, err_len, KS_ERR_CUDA, "cudaStreamIsCapturing failed");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return report(err, err_len, KS_ERR_ARG,
                      "stream is capturing; ks_smooth_static synchronizes its stream and cannot "
                      "run inside a capture");
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(ws + o_bad);
    double* resid = reinterpret_cast<double*>(ws + o_res);
    const SmallOps* ops = small_ops(n);

#define KS_STATIC_CUDA(call)                                                                     \
    do {                                                                                         \
        const cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                                   \
            return report(err, err_len, KS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

    // What the previous call left must not leak into this one.
    KS_STATIC_CUDA(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long) * ST_NCODES, st));
    KS_STATIC_CUDA(cudaMemsetAsync(resid, 0, (size_t)k * sizeof(double), st));

    WhitenArgs wa{};
    wa.k = k;
    wa.n = n;
    wa.mmax = m;
    wa.m_uniform = m;
    wa.F = F; wa.H = H; wa.c = c; wa.K = K; wa.G = G; wa.o = o; wa.C = C;
    wa.level0 = ws + o_a;
    wa.resid = resid + k;
    wa.cn2 = reinterpret_cast<double*>(ws + o_cn);
    wa.cd2 = reinterpret_cast<double*>(ws + o_cd);
    wa.bad = bad;
    KS_STATIC_CUDA(ops->whiten(wa, false, st));
    void* bufs[2] = {ws + o_a, ws + o_b};
    void* R = ws + o_r;
    int64_t nc = k;
    int level = 0, cur = 0;
    while (nc > 1) {
        KS_STATIC_CUDA(ops->level(nc, level, k, bufs[cur], bufs[cur ^ 1], R, resid, wa.cn2, wa.cd2,
                                  bad, false, st));
        nc /= 2;
        ++level;
        cur ^= 1;
    }
    const int L = level;
    KS_STATIC_CUDA(ops->base(k, L, bufs[cur], R, wa.cn2, wa.cd2, bad, false, st));
    for (int l = L; l >= 0; --l) KS_STATIC_CUDA(ops->backsub(k, l, R, nullptr, u_out, false, st));
    if (cov_out)
        for (int l = L; l >= 0; --l)
            KS_STATIC_CUDA(ops->selinv(k, l, R, ws + o_s, cov_out, bad, false, st));

    unsigned long long words[ST_NCODES];
    KS_STATIC_CUDA(cudaMemcpyAsync(words, bad, sizeof(words), cudaMemcpyDeviceToHost, st));
    KS_STATIC_CUDA(cudaStreamSynchronize(st));
#undef KS_STATIC_CUDA
    for (int code : status_order) {
        if (words[code] != ~0ULL) {
            if (info) *info = (int64_t)words[code];
            return report(err, err_len, (ks_status)code, "%s %lld", status_message(code),
                          (long long)words[code]);
        }
    }
    return KS_OK;
}

// ks_api.cu -- the C ABI declared in include/ks.h: argument checks, device work memory, staging
// of host arrays, and the launch sequence of one smoothing call:
//   whitening -> level 0 .. L-1 of the odd-even factorization -> base -> back substitution
//   (levels L .. 0) [-> FP64 refinement in KS_FP32_REFINE mode] -> copy-out -> status.
#include <cstdlib>

#include "ks_host.h"

using namespace ks;

namespace ks {
extern const SmallOps small_ops_1, small_ops_2, small_ops_3, small_ops_4, small_ops_5,
    small_ops_6, small_ops_7, small_ops_8;
const SmallOps* small_ops(int n) {
    static const SmallOps* table[SMALL_NMAX + 1] = {nullptr,      &small_ops_1, &small_ops_2,
                                                    &small_ops_3, &small_ops_4, &small_ops_5,
                                                    &small_ops_6, &small_ops_7, &small_ops_8};
    return (n >= 1 && n <= SMALL_NMAX) ? table[n] : nullptr;
}

extern const MedOps med_ops_12, med_ops_16, med_ops_24, med_ops_32, med_ops_48, med_ops_64;
static const MedOps* med_table(int n) {
    if (const char* v = getenv("KS_NO_MED")) { if (*v && *v != '0') return nullptr; }
    switch (n) {
        case 12: return &med_ops_12;
        case 16: return &med_ops_16;
        case 24: return &med_ops_24;
        case 32: return &med_ops_32;
        case 48: return &med_ops_48;
        case 64: return &med_ops_64;
        default: return nullptr;
    }
}
const MedOps* med_ops(int n, bool fp32) {
    const MedOps* m = med_table(n);
    return (m != nullptr && (fp32 || m->fp64)) ? m : nullptr;
}
const MedOps* med_whiten_ops(int n, int mmax, bool fp32) {
    const MedOps* m = med_table(n);
    return (m != nullptr && mmax <= n && (fp32 || m->wfp64)) ? m : nullptr;
}
}  // namespace ks

using namespace kshost;

extern "C" {

void ks_default_options(ks_options* opt) {
    if (!opt) return;
    opt->device = 0;
    opt->precision = KS_FP64;
    opt->stream = nullptr;
    opt->mem_budget = 0;
    opt->sync = 1;
    opt->profile = 0;
    opt->tune_cache = nullptr;
}

ks_status ks_create(ks_ctx** out, const ks_options* opt) {
    if (!out) return KS_ERR_ARG;
    *out = nullptr;
    ks_options o;
    ks_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != KS_FP64 && o.precision != KS_FP32_REFINE) return KS_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
        cudaGetLastError();
        return KS_ERR_CUDA;
    }
    ks_ctx* ctx = new ks_ctx();
    ctx->device = o.device;
    ctx->precision = o.precision;
    ctx->budget = o.mem_budget;
    ctx->sync = o.sync;
    ctx->profile = o.profile;
    if (o.tune_cache) ctx->tune_cache = o.tune_cache;
    if (cudaSetDevice(o.device) != cudaSuccess) { delete ctx; return KS_ERR_CUDA; }
    if (o.stream) {
        ctx->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return KS_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, o.device);
    if (cudaMalloc(&ctx->d_bad, sizeof(unsigned long long) * ST_NCODES) != cudaSuccess ||
        cudaMallocHost(&ctx->h_bad, sizeof(unsigned long long) * ST_NCODES) != cudaSuccess ||
        cudaMallocHost(&ctx->h_scalar, sizeof(double)) != cudaSuccess) {
        ks_destroy(ctx);
        return KS_ERR_OOM;
    }
    cudaMemsetAsync(ctx->d_bad, 0xFF, sizeof(unsigned long long) * ST_NCODES, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        ks_destroy(ctx);
        return KS_ERR_CUDA;
    }
    *out = ctx;
    return KS_OK;
}

int ks_max_n(const ks_ctx* ctx) { return ctx ? max_n_for(ctx) : 0; }

int ks_max_m(const ks_ctx* ctx, int n) { return ctx ? max_m_for(ctx, n) : -1; }

const char* ks_last_error(const ks_ctx* ctx) { return ctx ? ctx->err.c_str() : "null ctx"; }

ks_status ks_smooth(ks_ctx* ctx, int64_t k, int n, const int32_t* m, const double* F,
                    const double* H, const double* c, const double* K, const double* G,
                    const double* o, const double* C, double* u_out, ks_handle* keep,
                    int64_t* info) {
    if (!ctx) return KS_ERR_ARG;
    if (info) *info = -1;
    ks_fac* reuse = nullptr;
    if (keep) {
        if (*keep && ctx->facs.count(*keep)) reuse = *keep;
        *keep = nullptr;
    }
    ctx->err.clear();
    if (k < 1) return fail(ctx, KS_ERR_ARG, "k must be >= 1 (got %lld)", (long long)k);
    const int maxn = max_n_for(ctx);
    if (n < 1 || n > maxn) return fail(ctx, KS_ERR_ARG, "n = %d outside [1, %d]", n, maxn);
    if (!m || !u_out) return fail(ctx, KS_ERR_ARG, "m and u_out must not be NULL");
    if (k > 1 && (!F || !H || !K)) return fail(ctx, KS_ERR_ARG, "F, H and K must not be NULL when k > 1");
    const bool fp32 = ctx->precision == KS_FP32_REFINE;
    const int maxm = max_m_for(ctx, n);
    int mmax = 0;
    int64_t tot_m = 0, tot_m2 = 0;
    bool uniform = true;
    for (int64_t i = 0; i < k; ++i) {
        const int mi = m[i];
        if (mi < 0 || mi > maxm) return fail(ctx, KS_ERR_ARG, "m[%lld] = %d outside [0, %d]", (long long)i, mi, maxm);
        mmax = std::max(mmax, mi);
        tot_m += mi;
        tot_m2 += (int64_t)mi * mi;
        uniform = uniform && (mi == m[0]);
    }
    if (tot_m > 0 && (!G || !o || !C)) return fail(ctx, KS_ERR_ARG, "G, o and C must not be NULL when some m_i > 0");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    // Small states with at most n observations per step run one thread per unit of work.
    const SmallOps* sops = (mmax <= n) ? small_ops(n) : nullptr;

    const size_t T = fp32 ? 4 : 8;
    const int64_t CS = level_cs(n), RS = rstore_rs(n);
    const int64_t nn = (int64_t)n * n;
    const int64_t ke = k > 1 ? k - 1 : 0;
    struct Src { const double* p; size_t count; bool dev; size_t off; };
    Src src[7] = {{F, (size_t)(ke * nn), false, 0}, {H, (size_t)(ke * nn), false, 0},
                  {c, (size_t)(ke * n), false, 0},  {K, (size_t)(ke * nn), false, 0},
                  {G, (size_t)(tot_m * n), false, 0}, {o, (size_t)tot_m, false, 0},
                  {C, (size_t)tot_m2, false, 0}};
    Plan plan, splan;   // work memory; staging of host inputs
    const size_t o_lvlA = plan.take((size_t)k * CS * T);
    const size_t o_lvlB = plan.take((size_t)(k / 2 + 1) * CS * T);
    for (auto& s : src) {
        s.dev = s.p == nullptr || s.count == 0 || is_device_ptr(s.p);
        if (!s.dev) s.off = splan.take(s.count * sizeof(double));
    }
    const bool u_dev = is_device_ptr(u_out);
    const size_t o_u = u_dev ? 0 : plan.take((size_t)k * n * sizeof(double));
    size_t o_moff = 0, o_goff = 0, o_coff = 0;
    if (!uniform) {
        o_moff = plan.take((size_t)k * sizeof(int32_t));
        o_goff = plan.take((size_t)(k + 1) * sizeof(int64_t));
        o_coff = plan.take((size_t)(k + 1) * sizeof(int64_t));
    }
    size_t o_R = 0, o_res = 0;
    if (!keep) {
        o_R = plan.take((size_t)k * RS * T);
        o_res = plan.take((size_t)2 * k * sizeof(double));
    }
    const bool huge = n > LARGE_NMAX;   // factors of the whitening in per-block global slices
    const size_t o_wscr = huge ? plan.take((size_t)huge_grid(k) * huge_whiten_scratch_bytes(n)) : 0;
    const size_t o_cn2 = plan.take((size_t)k * n * sizeof(double));
    const size_t o_cd2 = plan.take((size_t)k * n * sizeof(double));
    size_t o_LK = 0, o_LC = 0, o_g = 0, o_q = 0, o_w = 0, o_d = 0;
    if (fp32) {
        o_LK = plan.take((size_t)ke * nn * sizeof(double));
        o_LC = plan.take((size_t)std::max<int64_t>(tot_m2, 1) * sizeof(double));
        o_g = plan.take((size_t)k * n * sizeof(double));
        o_q = plan.take((size_t)std::max<int64_t>(ke, 1) * n * sizeof(double));
        o_w = plan.take((size_t)k * n * sizeof(double));
        o_d = plan.take((size_t)k * n * sizeof(double));
    }
    ks_status rs = reserve(ctx, plan.off);
    if (rs != KS_OK) return rs;
    int ib = -1;   // input staging buffer of this call
    if (splan.off > 0) {
        ib = ctx->in_next;
        rs = stage_reserve(ctx, ib, splan.off);
        if (rs != KS_OK) return rs;
        ctx->in_next ^= 1;
    }
    char* ws = (char*)ctx->ws;
    cudaStream_t st = ctx->stream;

    ks_fac* fac = nullptr;
    void* R;
    double* resid;
    if (keep && reuse && reuse->k == k && reuse->n == n && reuse->precision == ctx->precision &&
        reuse->small == sops) {
        fac = reuse;
        R = fac->R;
        resid = fac->resid;
    } else if (keep) {
        fac = new ks_fac();
        fac->k = k;
        fac->n = n;
        fac->precision = ctx->precision;
        fac->small = sops;
        cudaError_t e1 = cudaMalloc(&fac->R, (size_t)k * RS * T);
        cudaError_t e2 = e1 == cudaSuccess ? cudaMalloc((void**)&fac->resid, (size_t)2 * k * sizeof(double)) : e1;
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cudaGetLastError();
            if (fac->R) cudaFree(fac->R);
            delete fac;
            return fail(ctx, KS_ERR_OOM, "cannot allocate the retained factor (%zu bytes)", (size_t)k * RS * T);
        }
        R = fac->R;
        resid = fac->resid;
    } else {
        R = ws + o_R;
        resid = (double*)(ws + o_res);
    }

    ctx->prof.calls++;
    // Stage host inputs.
    const double* dptr[7];
    double* u = u_dev ? u_out : (double*)(ws + o_u);
    std::vector<int64_t> goff, coff;
    {
    Phase ph_copy(ctx, KS_PHASE_COPY);
    if (ib >= 0) {
        // The copies wait only for the kernels of the call that last read this buffer (two calls
        // back), not for the previous call, whose kernels they overlap.
        ks_ctx::Stage& sb = ctx->in_stage[ib];
        KS_CUDA(ctx, cudaStreamWaitEvent(ctx->cin, sb.free, 0));
        for (int i = 0; i < 7; ++i)
            if (!src[i].dev)
                KS_CUDA(ctx, cudaMemcpyAsync((char*)sb.p + src[i].off, src[i].p,
                                             src[i].count * sizeof(double), cudaMemcpyHostToDevice,
                                             ctx->cin));
        KS_CUDA(ctx, cudaEventRecord(sb.ready, ctx->cin));
        KS_CUDA(ctx, cudaStreamWaitEvent(st, sb.ready, 0));
    }
    for (int i = 0; i < 7; ++i)
        dptr[i] = src[i].dev ? src[i].p : (const double*)((char*)ctx->in_stage[ib].p + src[i].off);
    if (!uniform) {
        goff.resize(k + 1);
        coff.resize(k + 1);
        goff[0] = coff[0] = 0;
        for (int64_t i = 0; i < k; ++i) {
            goff[i + 1] = goff[i] + m[i];
            coff[i + 1] = coff[i] + (int64_t)m[i] * m[i];
        }
        KS_CUDA(ctx, cudaMemcpyAsync(ws + o_moff, m, (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        KS_CUDA(ctx, cudaMemcpyAsync(ws + o_goff, goff.data(), (size_t)(k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        KS_CUDA(ctx, cudaMemcpyAsync(ws + o_coff, coff.data(), (size_t)(k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    }
    }

    WhitenArgs wa{};
    wa.ti = 0;
    wa.k = k;
    wa.n = n;
    wa.mmax = mmax;
    wa.m_uniform = uniform ? m[0] : -1;
    wa.m = uniform ? nullptr : (const int32_t*)(ws + o_moff);
    wa.goff = uniform ? nullptr : (const int64_t*)(ws + o_goff);
    wa.coff = uniform ? nullptr : (const int64_t*)(ws + o_coff);
    wa.F = dptr[0]; wa.H = dptr[1]; wa.c = c ? dptr[2] : nullptr; wa.K = dptr[3];
    wa.G = dptr[4]; wa.o = dptr[5]; wa.C = dptr[6];
    wa.level0 = ws + o_lvlA;
    wa.resid = resid + k;
    wa.LK = fp32 ? (double*)(ws + o_LK) : nullptr;
    wa.LC = fp32 ? (double*)(ws + o_LC) : nullptr;
    wa.cn2 = (double*)(ws + o_cn2);
    wa.cd2 = (double*)(ws + o_cd2);
    wa.bad = ctx->d_bad;
    wa.scratch = ws + o_lvlB;
    wa.cta_scratch = huge ? ws + o_wscr : nullptr;
    wa.cta_scratch_stride = huge ? (int64_t)huge_whiten_scratch_bytes(n) : 0;
    KS_CUDA(ctx, cudaMemsetAsync(resid, 0, (size_t)k * sizeof(double), st));
    {
        Phase ph(ctx, KS_PHASE_WHITEN);
        KS_CUDA(ctx, sops ? sops->whiten(wa, fp32, st) : launch_whiten(wa, fp32, st));
        KS_CUDA(ctx, launch_check_finite(wa, st));
    }
    // FP64: nothing after the whitening reads the inputs, so the staging buffer is free.
    if (ib >= 0 && !fp32) KS_CUDA(ctx, cudaEventRecord(ctx->in_stage[ib].free, st));

    // Odd-even levels.
    void* bufs[2] = {ws + o_lvlA, ws + o_lvlB};
    int64_t nc = k;
    int level = 0, cur = 0;
    {
        Phase ph(ctx, KS_PHASE_LEVEL);
        while (nc > 1) {
            if (sops)
                KS_CUDA(ctx, sops->level(nc, level, k, bufs[cur], bufs[cur ^ 1], R, resid, wa.cn2, wa.cd2, ctx->d_bad, fp32, st));
            else if (const MedOps* mops = med_ops(n, fp32))
                KS_CUDA(ctx, mops->level(nc, level, k, bufs[cur], bufs[cur ^ 1], R, resid, wa.cn2, wa.cd2, ctx->d_bad, fp32, st));
            else
                KS_CUDA(ctx, launch_level(n, nc, level, k, bufs[cur], bufs[cur ^ 1], R, resid, wa.cn2, wa.cd2, ctx->d_bad, fp32, st));
            nc /= 2;
            ++level;
            cur ^= 1;
        }
    }
    const int L = level;
    {
        Phase ph(ctx, KS_PHASE_BACKSUB);
        if (sops) {
            KS_CUDA(ctx, sops->base(k, L, bufs[cur], R, wa.cn2, wa.cd2, ctx->d_bad, fp32, st));
            for (int l = L; l >= 0; --l) KS_CUDA(ctx, sops->backsub(k, l, R, nullptr, u, fp32, st));
        } else {
            KS_CUDA(ctx, launch_base(n, k, L, bufs[cur], R, wa.cn2, wa.cd2, ctx->d_bad, fp32, st));
            for (int l = L; l >= 0; --l) KS_CUDA(ctx, launch_backsub_warp(n, k, l, R, fp32, u, st));
        }
    }

    if (fp32) {
        Phase ph(ctx, KS_PHASE_REFINE);
        RefineArgs ra{};
        ra.ti = 0;
        ra.k = k;
        ra.n = n;
        ra.m_uniform = wa.m_uniform;
        ra.m = wa.m;
        ra.goff = wa.goff;
        ra.coff = wa.coff;
        ra.F = wa.F; ra.H = wa.H; ra.c = wa.c; ra.G = wa.G; ra.o = wa.o;
        ra.LK = wa.LK; ra.LC = wa.LC;
        ra.u = u;
        ra.g = (double*)(ws + o_g);
        ra.q = (double*)(ws + o_q);
        double* w = (double*)(ws + o_w);
        double* d = (double*)(ws + o_d);
        if (sops) {
            // FP32 correction solve; the scratch vectors reuse the FP64 ones' space.
            KS_CUDA(ctx, sops->refine(ra, (float*)ra.q, (float*)ra.g, (float*)w, (float*)d, R, L, st));
        } else {
            KS_CUDA(ctx, launch_refine_warp(ra, (float*)ra.q, (float*)ra.g, (float*)w, (float*)d, R, L, st));
        }
        // FP32 + refinement: the refinement re-reads the inputs; after it the buffer is free.
        if (ib >= 0) KS_CUDA(ctx, cudaEventRecord(ctx->in_stage[ib].free, st));
    }
    if (!u_dev) {
        Phase ph(ctx, KS_PHASE_COPY);
        KS_CUDA(ctx, cudaMemcpyAsync(u_out, u, (size_t)k * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }

    if (fac) {
        ctx->facs.insert(fac);
        *keep = fac;
    }
    (void)reuse;
    if (ctx->sync) {
        ks_status s = collect_status(ctx, info);
        if (s != KS_OK && fac) {
            // the handle stays valid (memory owned by ctx) but the factor is unusable
        }
        return s;
    }
    return KS_OK;
}

ks_status ks_covariances(ks_ctx* ctx, ks_handle h, double* cov_out, double* cross_out) {
    if (!ctx) return KS_ERR_ARG;
    ctx->err.clear();
    if (!h || !ctx->facs.count(h)) return fail(ctx, KS_ERR_NO_FACTOR, "unknown or released handle");
    if (!cov_out) return fail(ctx, KS_ERR_ARG, "cov_out must not be NULL");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    const bool fp32 = h->precision == KS_FP32_REFINE;
    const int n = h->n;
    const int64_t k = h->k, nn = (int64_t)n * n;
    const size_t T = fp32 ? 4 : 8;
    Plan plan;
    const size_t o_S = plan.take((size_t)k * 2 * nn * T);
    const bool huge = n > LARGE_NMAX;   // Rd^{-1} and M of every block in a global slice
    const size_t o_ri = huge ? plan.take((size_t)huge_grid((k + 1) / 2) * 2 * nn * T) : 0;
    const bool cov_dev = is_device_ptr(cov_out);
    const size_t o_cov = cov_dev ? 0 : plan.take((size_t)k * nn * sizeof(double));
    const bool cross_dev = cross_out == nullptr || is_device_ptr(cross_out);
    const size_t o_cross = cross_dev ? 0 : plan.take((size_t)std::max<int64_t>(k - 1, 1) * nn * sizeof(double));
    ks_status rs = reserve(ctx, plan.off);
    if (rs != KS_OK) return rs;
    char* ws = (char*)ctx->ws;
    cudaStream_t st = ctx->stream;
    double* Sd = cov_dev ? cov_out : (double*)(ws + o_cov);
    void* Sx = ws + o_S;
    int L = 0;
    while ((k >> (L + 1)) >= 1) ++L;
    ctx->prof.calls++;
    double* cr = cross_out ? (cross_dev ? cross_out : (double*)(ws + o_cross)) : nullptr;
    {
        Phase ph(ctx, KS_PHASE_SELINV);
        const SmallOps* sops = h->small;
        for (int l = L; l >= 0; --l)
            KS_CUDA(ctx, sops ? sops->selinv(k, l, h->R, Sx, Sd, ctx->d_bad, fp32, st)
                         : huge ? launch_selinv_huge(n, k, l, h->R, Sx, Sd, ws + o_ri, ctx->d_bad, fp32, st)
                                : launch_selinv(n, k, l, h->R, Sx, Sd, ctx->d_bad, fp32, st));
        if (cr) KS_CUDA(ctx, sops ? sops->cross(k, Sx, cr, fp32, st) : launch_cross(n, k, Sx, cr, fp32, st));
    }
    {
        Phase ph(ctx, KS_PHASE_COPY);
        if (cr && !cross_dev && k > 1)
            KS_CUDA(ctx, cudaMemcpyAsync(cross_out, cr, (size_t)(k - 1) * nn * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (!cov_dev)
            KS_CUDA(ctx, cudaMemcpyAsync(cov_out, Sd, (size_t)k * nn * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (ctx->sync) return collect_status(ctx, nullptr);
    return KS_OK;
}

ks_status ks_residual(ks_ctx* ctx, ks_handle h, double* out) {
    if (!ctx) return KS_ERR_ARG;
    if (!h || !ctx->facs.count(h)) return fail(ctx, KS_ERR_NO_FACTOR, "unknown or released handle");
    if (!out) return fail(ctx, KS_ERR_ARG, "out must not be NULL");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    Plan plan;
    const size_t o_s = plan.take(sizeof(double));
    ks_status rs = reserve(ctx, plan.off);
    if (rs != KS_OK) return rs;
    double* d = (double*)((char*)ctx->ws + o_s);
    KS_CUDA(ctx, launch_sum(h->resid, 2 * h->k, d, ctx->stream));
    KS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scalar, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *out = *ctx->h_scalar;
    return KS_OK;
}

ks_status ks_release(ks_ctx* ctx, ks_handle h) {
    if (!ctx) return KS_ERR_ARG;
    if (!h) return KS_OK;
    if (!ctx->facs.count(h)) return fail(ctx, KS_ERR_NO_FACTOR, "unknown or released handle");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(h->R);
    cudaFree(h->resid);
    ctx->facs.erase(h);
    delete h;
    return KS_OK;
}

ks_status ks_sync(ks_ctx* ctx, int64_t* info) {
    if (!ctx) return KS_ERR_ARG;
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    return collect_status(ctx, info);
}

ks_status ks_profile_read(ks_ctx* ctx, ks_profile* out, int reset) {
    if (!ctx || !out) return KS_ERR_ARG;
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    drain_profile(ctx);
    *out = ctx->prof;
    if (reset) ctx->prof = ks_profile{};
    return KS_OK;
}

ks_status ks_destroy(ks_ctx* ctx) {
    if (!ctx) return KS_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drain_profile(ctx);
    for (cudaEvent_t e : ctx->spare) cudaEventDestroy(e);
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
    if (ctx->bmeta) cudaFree(ctx->bmeta);
    if (ctx->vbuf) cudaFree(ctx->vbuf);
    if (ctx->gbuf) cudaFree(ctx->gbuf);
    for (ks_fac* f : ctx->facs) {
        cudaFree(f->R);
        cudaFree(f->resid);
        delete f;
    }
    ctx->facs.clear();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->cin) cudaStreamSynchronize(ctx->cin);
    for (auto& sb : ctx->in_stage) {
        if (sb.p) cudaFree(sb.p);
        if (sb.ready) cudaEventDestroy(sb.ready);
        if (sb.free) cudaEventDestroy(sb.free);
    }
    if (ctx->cin) cudaStreamDestroy(ctx->cin);
    if (ctx->d_bad) cudaFree(ctx->d_bad);
    if (ctx->h_bad) cudaFreeHost(ctx->h_bad);
    if (ctx->h_scalar) cudaFreeHost(ctx->h_scalar);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return KS_OK;
}

}  // extern "C"

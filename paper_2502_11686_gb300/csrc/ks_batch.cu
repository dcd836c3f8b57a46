// ks_batch.cu -- ks_smooth_batch: many independent problems of different lengths and state
// dimensions smoothed together.
//
// Problems are grouped by (n, path): the small-state path (n <= 8, every m_i <= n; one thread per
// unit) or the column-owner path (one thread block per unit).  For each group, every operation
// of the method -- whitening, each level of the odd-even factorization, the base, each level of
// back substitution, the refinement steps, each level of SelInv -- is ONE launch whose persistent
// thread blocks walk the units of all problems of the group (a device work list: a prefix sum of
// the units per problem, searched per unit).  Problems whose recursion is shallower simply have
// no units at the deeper levels.
//
// The descriptors and work lists live at fixed offsets of one device buffer, so the launch
// sequence of a batch shape (groups, deepest level per group, precision, covariances) is captured
// once as a CUDA graph and replayed for later batches of that shape: only the contents of the
// buffer change.  The persistent grid of the level and SelInv launches of each group is chosen by
// timing candidate grids on the first batch that contains the group (the project's autotuner); the
// choices are kept in the ctx and, if ks_options.tune_cache is set, in that file.
#include <fstream>
#include <sstream>

#include "ks_host.h"

using namespace ks;
using namespace kshost;

namespace {

struct Group {
    int n = 0;
    bool small = false;
    int mmax = 0;
    int L = 0;
    bool cov = false;
    std::vector<int> probs;
    const SmallOps* sops = nullptr;
    std::string sig(bool fp32) const {
        std::ostringstream os;
        os << (fp32 ? "f32" : "f64") << ":n" << n << (small ? ":s" : ":g") << ":m" << mmax;
        return os.str();
    }
};

struct Launch {
    int group, op, level;
    size_t work_off;  // BatchWork in the meta buffer
    size_t off_off;   // its prefix array
};

int64_t units_of(int op, int level, int64_t k, int n) {
    switch (op) {
        case B_WHITEN: return k;
        case B_LEVEL: return (k >> level) >> 1;
        case B_BASE: return 1;
        case B_BACKSUB:
        case B_SELINV:
        case B_BACKSUB_W: return (k >> level) - (k >> (level + 1));
        case B_REFINE_Q: return k - 1;
        case B_REFINE_G: return k;
        case B_RT_SOLVE: return k >> level;
        case B_ADD: return k * n;
    }
    return 0;
}

int floor_log2(int64_t k) {
    int L = 0;
    while ((k >> (L + 1)) >= 1) ++L;
    return L;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int TUNE_FAMILY = 64;   // tuned value = family * TUNE_FAMILY + blocks per SM

void load_tuning(ks_ctx* ctx) {
    if (ctx->tune_loaded) return;
    ctx->tune_loaded = true;
    if (ctx->tune_cache.empty()) return;
    std::ifstream in(ctx->tune_cache);
    std::string sig;
    int bps;
    while (in >> sig >> bps)
        if (bps > 0) ctx->tuned[sig] = bps;
}

void save_tuning(ks_ctx* ctx) {
    if (ctx->tune_cache.empty()) return;
    std::ofstream out(ctx->tune_cache, std::ios::trunc);
    for (auto& kv : ctx->tuned) out << kv.first << " " << kv.second << "\n";
}

}  // namespace

extern "C" ks_status ks_smooth_batch(ks_ctx* ctx, int nprob, const ks_problem* probs, int* status,
                                     int64_t* info) {
    if (!ctx) return KS_ERR_ARG;
    ctx->err.clear();
    if (nprob < 1 || !probs) return fail(ctx, KS_ERR_ARG, "nprob must be >= 1 and probs not NULL");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    const bool fp32 = ctx->precision == KS_FP32_REFINE;
    const size_t T = fp32 ? 4 : 8;
    const int maxn = std::min(max_n_for(ctx), LARGE_NMAX);   // batched kernels stop at 128
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    load_tuning(ctx);

    // ---- validate and group ----
    std::vector<int> mmax(nprob), m0(nprob);
    std::vector<char> uniform(nprob);
    std::vector<int64_t> tot_m(nprob), tot_m2(nprob);
    std::map<std::pair<int, int>, Group> gmap;
    for (int p = 0; p < nprob; ++p) {
        const ks_problem& P = probs[p];
        if (P.k < 1 || P.n < 1 || P.n > maxn || !P.m || !P.u_out)
            return fail(ctx, KS_ERR_ARG, "problem %d: bad k / n / m / u_out", p);
        if (P.k > 1 && (!P.F || !P.H || !P.K)) return fail(ctx, KS_ERR_ARG, "problem %d: F, H, K needed", p);
        const int maxm = max_m_for(ctx, P.n);
        int mm = 0;
        int64_t t1 = 0, t2 = 0;
        bool uni = true;
        for (int64_t i = 0; i < P.k; ++i) {
            const int mi = P.m[i];
            if (mi < 0 || mi > maxm) return fail(ctx, KS_ERR_ARG, "problem %d: m[%lld] = %d", p, (long long)i, mi);
            mm = std::max(mm, mi);
            t1 += mi;
            t2 += (int64_t)mi * mi;
            uni = uni && mi == P.m[0];
        }
        if (t1 > 0 && (!P.G || !P.o || !P.C)) return fail(ctx, KS_ERR_ARG, "problem %d: G, o, C needed", p);
        if ((P.time_invariant & (KS_TI_G | KS_TI_C)) && !uni)
            return fail(ctx, KS_ERR_ARG, "problem %d: time-invariant G / C need the same m at every step", p);
        mmax[p] = mm;
        m0[p] = P.m[0];
        uniform[p] = uni;
        tot_m[p] = t1;
        tot_m2[p] = t2;
        const SmallOps* sops = (mm <= P.n) ? small_ops(P.n) : nullptr;
        Group& g = gmap[{P.n, sops ? 1 : 0}];
        g.n = P.n;
        g.small = sops != nullptr;
        g.sops = sops;
        g.mmax = std::max(g.mmax, mm);
        g.L = std::max(g.L, floor_log2(P.k));
        g.cov = g.cov || P.cov_out != nullptr;
        g.probs.push_back(p);
    }
    std::vector<Group> groups;
    for (auto& kv : gmap) groups.push_back(kv.second);

    // ---- per-problem work memory ----
    struct Mem {
        size_t stage[7], m, goff, coff, lvl0, lvl1, R, cn2, cd2, u, LK, LC, q, g, w, d, Sx, cov;
    };
    std::vector<Mem> mem(nprob);
    Plan plan;
    const size_t o_bad = plan.take((size_t)nprob * ST_NCODES * sizeof(unsigned long long));
    std::vector<size_t> o_res(nprob);
    for (int p = 0; p < nprob; ++p) o_res[p] = plan.take((size_t)2 * probs[p].k * sizeof(double));
    const size_t res_end = plan.off;
    const size_t res_begin = o_res[0];
    for (int p = 0; p < nprob; ++p) {
        const ks_problem& P = probs[p];
        const int64_t k = P.k, n = P.n, nn = n * n, ke = k > 1 ? k - 1 : 0;
        const bool small = mmax[p] <= n && small_ops(P.n) != nullptr;
        const int64_t nt = n * (n + 1) / 2;
        const int64_t CS = small ? nt + 2 * n + 2 * nn : level_cs((int)n);
        const int64_t RS = small ? nt + 2 * nn + n : rstore_rs((int)n);
        Mem& M = mem[p];
        const double* src[7] = {P.F, P.H, P.c, P.K, P.G, P.o, P.C};
        const unsigned ti = P.time_invariant;
        const int64_t kf = (ti & KS_TI_F) ? 1 : ke, kh = (ti & KS_TI_H) ? 1 : ke, kk = (ti & KS_TI_K) ? 1 : ke;
        const size_t cnt[7] = {(size_t)(kf * nn), (size_t)(kh * nn), (size_t)(ke * n), (size_t)(kk * nn),
                               (size_t)((ti & KS_TI_G) ? (int64_t)m0[p] * n : tot_m[p] * n), (size_t)tot_m[p],
                               (size_t)((ti & KS_TI_C) ? (int64_t)m0[p] * m0[p] : tot_m2[p])};
        for (int a = 0; a < 7; ++a)
            M.stage[a] = (src[a] && cnt[a] && !is_device_ptr(src[a])) ? plan.take(cnt[a] * sizeof(double)) + 1 : 0;
        M.m = M.goff = M.coff = 0;
        if (!uniform[p]) {
            M.m = plan.take((size_t)k * sizeof(int32_t));
            M.goff = plan.take((size_t)(k + 1) * sizeof(int64_t));
            M.coff = plan.take((size_t)(k + 1) * sizeof(int64_t));
        }
        M.lvl0 = plan.take((size_t)k * CS * T);
        M.lvl1 = plan.take((size_t)(k / 2 + 1) * CS * T);
        M.R = plan.take((size_t)k * RS * T);
        M.cn2 = plan.take((size_t)k * n * sizeof(double));
        M.cd2 = plan.take((size_t)k * n * sizeof(double));
        M.u = is_device_ptr(P.u_out) ? 0 : plan.take((size_t)k * n * sizeof(double)) + 1;
        M.LK = M.LC = M.q = M.g = M.w = M.d = 0;
        if (fp32) {
            M.LK = plan.take((size_t)std::max<int64_t>(ke, 1) * nn * sizeof(double));
            M.LC = plan.take((size_t)std::max<int64_t>(tot_m2[p], 1) * sizeof(double));
            const size_t vb = small ? sizeof(float) : sizeof(double);
            M.q = plan.take((size_t)std::max<int64_t>(ke, 1) * n * vb);
            M.g = plan.take((size_t)k * n * vb);
            M.w = plan.take((size_t)k * n * vb);
            M.d = plan.take((size_t)k * n * vb);
        }
        M.Sx = M.cov = 0;
        if (P.cov_out) {
            M.Sx = plan.take((size_t)k * 2 * nn * T);
            M.cov = is_device_ptr(P.cov_out) ? 0 : plan.take((size_t)k * nn * sizeof(double)) + 1;
        }
    }
    ks_status rs = reserve(ctx, plan.off);
    if (rs != KS_OK) return rs;
    char* ws = static_cast<char*>(ctx->ws);
    cudaStream_t st = ctx->stream;

    // ---- descriptors (host) and staging copies ----
    std::vector<ProbDesc> desc(nprob);
    std::vector<std::vector<int64_t>> offs_host(nprob);
    {
        Phase ph(ctx, KS_PHASE_COPY);
        for (int p = 0; p < nprob; ++p) {
            const ks_problem& P = probs[p];
            const Mem& M = mem[p];
            ProbDesc& D = desc[p];
            memset(&D, 0, sizeof(D));
            D.k = P.k;
            D.n = P.n;
            D.mmax = mmax[p];
            D.L = floor_log2(P.k);
            D.m_uniform = uniform[p] ? m0[p] : -1;
            const double* src[7] = {P.F, P.H, P.c, P.K, P.G, P.o, P.C};
            const double* dst[7];
            const int64_t ke = P.k > 1 ? P.k - 1 : 0, nn = (int64_t)P.n * P.n;
            const unsigned ti = P.time_invariant;
            const int64_t kf = (ti & KS_TI_F) ? 1 : ke, kh = (ti & KS_TI_H) ? 1 : ke, kk = (ti & KS_TI_K) ? 1 : ke;
            const size_t cnt[7] = {(size_t)(kf * nn), (size_t)(kh * nn), (size_t)(ke * P.n), (size_t)(kk * nn),
                                   (size_t)((ti & KS_TI_G) ? (int64_t)m0[p] * P.n : tot_m[p] * P.n), (size_t)tot_m[p],
                                   (size_t)((ti & KS_TI_C) ? (int64_t)m0[p] * m0[p] : tot_m2[p])};
            D.ti = ti;
            for (int a = 0; a < 7; ++a) {
                if (M.stage[a]) {
                    KS_CUDA(ctx, cudaMemcpyAsync(ws + M.stage[a] - 1, src[a], cnt[a] * sizeof(double),
                                                 cudaMemcpyHostToDevice, st));
                    dst[a] = (const double*)(ws + M.stage[a] - 1);
                } else {
                    dst[a] = src[a];
                }
            }
            D.F = dst[0]; D.H = dst[1]; D.c = P.c ? dst[2] : nullptr; D.K = dst[3];
            D.G = dst[4]; D.o = dst[5]; D.C = dst[6];
            if (!uniform[p]) {
                std::vector<int64_t>& go = offs_host[p];
                go.resize(2 * (P.k + 1));
                int64_t* g = go.data();
                int64_t* c2 = g + P.k + 1;
                g[0] = c2[0] = 0;
                for (int64_t i = 0; i < P.k; ++i) {
                    g[i + 1] = g[i] + P.m[i];
                    c2[i + 1] = c2[i] + (int64_t)P.m[i] * P.m[i];
                }
                KS_CUDA(ctx, cudaMemcpyAsync(ws + M.m, P.m, (size_t)P.k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
                KS_CUDA(ctx, cudaMemcpyAsync(ws + M.goff, g, (size_t)(P.k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
                KS_CUDA(ctx, cudaMemcpyAsync(ws + M.coff, c2, (size_t)(P.k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
                D.m = (const int32_t*)(ws + M.m);
                D.goff = (const int64_t*)(ws + M.goff);
                D.coff = (const int64_t*)(ws + M.coff);
            }
            D.lvl[0] = ws + M.lvl0;
            D.lvl[1] = ws + M.lvl1;
            D.R = ws + M.R;
            D.resid = (double*)(ws + o_res[p]);
            D.cn2 = (double*)(ws + M.cn2);
            D.cd2 = (double*)(ws + M.cd2);
            D.u = M.u ? (double*)(ws + M.u - 1) : P.u_out;
            if (fp32) {
                D.LK = (double*)(ws + M.LK);
                D.LC = (double*)(ws + M.LC);
                D.q = ws + M.q;
                D.g = ws + M.g;
                D.w = ws + M.w;
                D.d = ws + M.d;
            }
            if (P.cov_out) {
                D.Sx = ws + M.Sx;
                D.cov = M.cov ? (double*)(ws + M.cov - 1) : P.cov_out;
            }
            D.bad = (unsigned long long*)(ws + o_bad) + (size_t)p * ST_NCODES;
        }
    }

    // ---- launch list and the meta buffer layout (fixed for a batch shape) ----
    int cap = 16;
    while (cap < nprob) cap *= 2;
    std::vector<Launch> launches;
    size_t moff = 0;
    const size_t o_desc = moff;
    moff += align256((size_t)cap * sizeof(ProbDesc));
    std::vector<size_t> o_probs(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        o_probs[gi] = moff;
        moff += align256((size_t)cap * sizeof(int));
    }
    auto add = [&](int gi, int op, int level) {
        Launch l;
        l.group = gi;
        l.op = op;
        l.level = level;
        l.work_off = moff;
        moff += align256(sizeof(BatchWork));
        l.off_off = moff;
        moff += align256((size_t)(cap + 1) * sizeof(int64_t));
        launches.push_back(l);
    };
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const Group& g = groups[gi];
        add((int)gi, B_WHITEN, 0);
        for (int l = 0; l < g.L; ++l) add((int)gi, B_LEVEL, l);
        add((int)gi, B_BASE, 0);
        for (int l = g.L; l >= 0; --l) add((int)gi, B_BACKSUB, l);
        if (fp32) {
            add((int)gi, B_REFINE_Q, 0);
            add((int)gi, B_REFINE_G, 0);
            for (int l = 0; l <= g.L; ++l) add((int)gi, B_RT_SOLVE, l);
            for (int l = g.L; l >= 0; --l) add((int)gi, B_BACKSUB_W, l);
            add((int)gi, B_ADD, 0);
        }
        if (g.cov)
            for (int l = g.L; l >= 0; --l) add((int)gi, B_SELINV, l);
    }
    if (moff > ctx->bmeta_size) {
        KS_CUDA(ctx, cudaStreamSynchronize(st));
        for (auto& gr : ctx->graphs) cudaGraphExecDestroy(gr.second);
        ctx->graphs.clear();
        if (ctx->bmeta) cudaFree(ctx->bmeta);
        ctx->bmeta = nullptr;
        ctx->bmeta_size = 0;
        KS_CUDA(ctx, cudaMalloc(&ctx->bmeta, moff * 2));
        ctx->bmeta_size = moff * 2;
    }
    char* meta = static_cast<char*>(ctx->bmeta);
    std::vector<char> blob(moff, 0);
    memcpy(blob.data() + o_desc, desc.data(), (size_t)nprob * sizeof(ProbDesc));
    for (size_t gi = 0; gi < groups.size(); ++gi)
        memcpy(blob.data() + o_probs[gi], groups[gi].probs.data(), groups[gi].probs.size() * sizeof(int));
    for (const Launch& l : launches) {
        const Group& g = groups[l.group];
        BatchWork w;
        w.desc = (const ProbDesc*)(meta + o_desc);
        w.probs = (const int*)(meta + o_probs[l.group]);
        w.off = (const int64_t*)(meta + l.off_off);
        w.np = (int)g.probs.size();
        w.level = l.level;
        memcpy(blob.data() + l.work_off, &w, sizeof(w));
        int64_t* off = (int64_t*)(blob.data() + l.off_off);
        off[0] = 0;
        for (size_t i = 0; i < g.probs.size(); ++i) {
            const ks_problem& P = probs[g.probs[i]];
            int64_t u = units_of(l.op, l.level, P.k, P.n);
            if (l.op == B_SELINV && !P.cov_out) u = 0;
            off[i + 1] = off[i] + u;
        }
    }
    KS_CUDA(ctx, cudaMemcpyAsync(meta, blob.data(), moff, cudaMemcpyHostToDevice, st));
    KS_CUDA(ctx, cudaMemsetAsync(ws + o_bad, 0xFF, (size_t)nprob * ST_NCODES * sizeof(unsigned long long), st));
    KS_CUDA(ctx, cudaMemsetAsync(ws + res_begin, 0, res_end - res_begin, st));

    // ---- one launch of the sequence ----
    // A tuned value is family * TUNE_FAMILY + blocks per SM (family: the level kernel of a
    // generic group, 0 = register-column, 1 = column owner; see launch_batch_generic).
    auto grid_of = [&](const Group& g, int op) -> unsigned {
        const int tuned = ctx->tuned.count(g.sig(fp32)) ? ctx->tuned[g.sig(fp32)] % TUNE_FAMILY : 0;
        int bps;
        if (g.small) bps = (op == B_LEVEL || op == B_SELINV) ? (tuned ? tuned : 8) : 16;
        else if (op == B_WHITEN || op == B_LEVEL || op == B_SELINV) bps = (op == B_WHITEN) ? 8 : (tuned ? tuned : 8);
        else if (op == B_BASE) bps = 2;
        else bps = 8;
        return (unsigned)(nsm * bps);
    };
    auto family_of = [&](const Group& g) -> int {
        return ctx->tuned.count(g.sig(fp32)) ? ctx->tuned[g.sig(fp32)] / TUNE_FAMILY : 0;
    };
    auto issue_f = [&](const Launch& l, unsigned grid, int family) -> cudaError_t {
        const Group& g = groups[l.group];
        const BatchWork* wk = (const BatchWork*)(meta + l.work_off);
        if (g.small) return g.sops->batch(l.op, wk, fp32, grid, st);
        return launch_batch_generic(l.op, g.n, g.mmax, wk, fp32, grid, st, family);
    };
    auto issue = [&](const Launch& l, unsigned grid) -> cudaError_t {
        return issue_f(l, grid, family_of(groups[l.group]));
    };

    // Batch shape: groups, their deepest levels, covariances, precision, capacity and grids.
    auto shape_key = [&]() {
        std::ostringstream key;
        key << (fp32 ? "f32" : "f64") << "|cap" << cap;
        for (const Group& g : groups)
            key << "|" << g.sig(fp32) << ":L" << g.L << (g.cov ? ":c" : "") << ":t"
                << (ctx->tuned.count(g.sig(fp32)) ? ctx->tuned[g.sig(fp32)] : 0);
        return key.str();
    };

    // ---- the first batch of a shape runs eagerly; groups seen for the first time are tuned
    //      there by timing candidate grids of their level-0 launch (it only reads the whitened
    //      level 0 and rewrites its outputs, so it can be repeated -- except the large-state
    //      kernel, which works in place and keeps a fixed grid) ----
    bool tuning = false;
    for (const Group& g : groups)
        if (!ctx->tuned.count(g.sig(fp32)) && g.L >= 1) tuning = true;
    ctx->prof.calls++;
    auto op_phase = [](int op) {
        switch (op) {
            case B_WHITEN: return (int)KS_PHASE_WHITEN;
            case B_LEVEL: return (int)KS_PHASE_LEVEL;
            case B_BASE:
            case B_BACKSUB: return (int)KS_PHASE_BACKSUB;
            case B_SELINV: return (int)KS_PHASE_SELINV;
            default: return (int)KS_PHASE_REFINE;
        }
    };
    if (ctx->profile && !tuning) {
        // Profiling: the same launches issued one by one, each timed into its phase.
        for (const Launch& l : launches) {
            Phase ph(ctx, op_phase(l.op));
            KS_CUDA(ctx, issue(l, grid_of(groups[l.group], l.op)));
        }
    } else if (tuning || !ctx->shapes_seen.count(shape_key())) {
        Phase ph(ctx, KS_PHASE_BATCH);
        cudaEvent_t e0 = get_event(ctx), e1 = get_event(ctx);
        for (size_t i = 0; i < launches.size(); ++i) {
            const Launch& l = launches[i];
            const Group& g = groups[l.group];
            const std::string sig = g.sig(fp32);
            if (l.op == B_LEVEL && l.level == 0 && !ctx->tuned.count(sig) && !g.small &&
                use_large(g.n, fp32)) {
                ctx->tuned[sig] = 2;   // the large-state level kernel works in place: not repeatable
            } else if (l.op == B_LEVEL && l.level == 0 && !ctx->tuned.count(sig)) {
                // Candidates: the persistent grid (blocks per SM) and, where the state dimension
                // has a register-column level kernel, that kernel or the column-owner one.
                static const int cand[] = {1, 2, 4, 8, 16, 32};
                const int nfam = (!g.small && med_ops(g.n, fp32) != nullptr) ? 2 : 1;
                float best = 1e30f;
                int best_val = 8;
                for (int fam = 0; fam < nfam; ++fam) {
                    for (int bps : cand) {
                        for (int rep = 0; rep < 2; ++rep) {   // first repetition warms up
                            KS_CUDA(ctx, cudaEventRecord(e0, st));
                            KS_CUDA(ctx, issue_f(l, (unsigned)(nsm * bps), fam));
                            KS_CUDA(ctx, cudaEventRecord(e1, st));
                            KS_CUDA(ctx, cudaEventSynchronize(e1));
                            float ms = 0.f;
                            cudaEventElapsedTime(&ms, e0, e1);
                            if (rep == 1 && ms < best) {
                                best = ms;
                                best_val = fam * TUNE_FAMILY + bps;
                            }
                        }
                    }
                }
                ctx->tuned[sig] = best_val;
            }
            KS_CUDA(ctx, issue(l, grid_of(g, l.op)));
        }
        ctx->spare.push_back(e0);
        ctx->spare.push_back(e1);
        if (tuning) save_tuning(ctx);
        ctx->shapes_seen.insert(shape_key());
    } else {
        // Replay (or capture, then replay) the launch graph of this batch shape.
        const std::string k = shape_key();
        auto it = ctx->graphs.find(k);
        if (it == ctx->graphs.end()) {
            cudaGraph_t graph = nullptr;
            KS_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaSuccess;
            for (const Launch& l : launches) {
                ce = issue(l, grid_of(groups[l.group], l.op));
                if (ce != cudaSuccess) break;
            }
            const cudaError_t ee = cudaStreamEndCapture(st, &graph);
            if (ce != cudaSuccess || ee != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return fail(ctx, KS_ERR_CUDA, "graph capture of the batch failed: %s",
                            cudaGetErrorString(ce != cudaSuccess ? ce : ee));
            }
            cudaGraphExec_t exec = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return fail(ctx, KS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            it = ctx->graphs.emplace(k, exec).first;
        }
        const uint64_t l0 = t_launches;
        {
            Phase ph(ctx, KS_PHASE_BATCH);
            KS_CUDA(ctx, cudaGraphLaunch(it->second, st));
            t_launches = l0 + launches.size();   // kernels replayed by the graph
        }
    }

    // ---- outputs and statuses ----
    {
        Phase ph(ctx, KS_PHASE_COPY);
        for (int p = 0; p < nprob; ++p) {
            const ks_problem& P = probs[p];
            const Mem& M = mem[p];
            if (M.u)
                KS_CUDA(ctx, cudaMemcpyAsync(P.u_out, ws + M.u - 1, (size_t)P.k * P.n * sizeof(double),
                                             cudaMemcpyDeviceToHost, st));
            if (P.cov_out && M.cov)
                KS_CUDA(ctx, cudaMemcpyAsync(P.cov_out, ws + M.cov - 1,
                                             (size_t)P.k * P.n * P.n * sizeof(double),
                                             cudaMemcpyDeviceToHost, st));
        }
    }
    std::vector<unsigned long long> words((size_t)nprob * ST_NCODES);
    KS_CUDA(ctx, cudaMemcpyAsync(words.data(), ws + o_bad, words.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
    KS_CUDA(ctx, cudaStreamSynchronize(st));
    ks_status first = KS_OK;
    for (int p = 0; p < nprob; ++p) {
        int sp = KS_OK;
        int64_t ip = -1;
        for (int code : status_order)
            if (words[(size_t)p * ST_NCODES + code] != ~0ULL) {
                sp = code;
                ip = (int64_t)words[(size_t)p * ST_NCODES + code];
                break;
            }
        if (status) status[p] = sp;
        if (info) info[p] = ip;
        if (sp != KS_OK && first == KS_OK) {
            first = (ks_status)sp;
            fail(ctx, first, "problem %d: status %d at index %lld", p, sp, (long long)ip);
        }
    }
    return first;
}

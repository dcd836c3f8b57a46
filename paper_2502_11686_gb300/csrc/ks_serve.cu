// ks_serve.cu -- the serving loop: continuous batching of smoothing requests on one GPU.
//
// A scheduler thread admits requests in arrival order while device memory (a budget) and slots
// allow, and runs "ticks".  A tick advances every admitted request by one stage of its plan
//   whitening, level 0 .. L-1, base, back substitution L .. 0,
//   [FP32 mode: refinement q, g, R^T w = g levels 0 .. L, R d = w levels L .. 0, u += d],
//   [covariances: SelInv levels L .. 0]
// and issues, per state-dimension group, ONE launch per kind of stage over all requests that
// are at it -- each request at its own recursion level (the batched kernels read the level from
// the request's descriptor).  Requests that arrive while others run join at the next tick, so
// their work shares launches with requests that are further along.  Stages advance
// deterministically, so the next tick is prepared while the previous one runs (two descriptor
// buffers); a request is complete when the tick of its last stage has finished on the device.
// Memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the server stream).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "ks_host.h"

namespace ks {
cudaError_t launch_generate(int64_t k, int n, int m, uint64_t seed, double f_scale, double* F,
                            double* H, double* K, double* G, double* C, double* o,
                            cudaStream_t st);
cudaError_t launch_generate_steps(int64_t k, int n, int m, uint64_t seed, double f_scale, double* F,
                                  double* H, double* K, double* G, double* C, double* o,
                                  cudaStream_t st);
}

using namespace ks;
using namespace kshost;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    int64_t id = 0;
    ks_problem prob{};
    bool synthetic = false;
    uint64_t seed = 0;
    int want_cov = 0;
    int64_t follow_of = -1;
    int64_t k = 0;
    int n = 0, mmax = 0, m0 = 0, L = 0;
    bool uniform = true;
    int64_t tot_m = 0, tot_m2 = 0;
    std::vector<int32_t> m_copy;
    std::vector<int64_t> offs;              // goff | coff (ragged m)
    const SmallOps* sops = nullptr;
    std::vector<std::pair<int, int>> stages;  // (operation, level)
    size_t stage = 0;
    void* arena = nullptr;
    size_t bytes = 0;
    ProbDesc desc{};
    double* u_host = nullptr;                // caller's host outputs (copied back at completion)
    double* cov_host = nullptr;
    double* cov_dev = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
    int status = KS_OK;
    int64_t info = -1;
    int state = 0;                           // 0 queued, 1 active, 2 last stage issued, 3 done
    int followers = 0;                       // covariance follow-ups not yet done
};

int floor_log2(int64_t k) {
    int L = 0;
    while ((k >> (L + 1)) >= 1) ++L;
    return L;
}

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

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct ks_server {
    ks_ctx* ctx = nullptr;
    ks_server_options opt{};
    bool fp32 = false;
    int nsm = 0;
    cudaStream_t st = nullptr, cst = nullptr;
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    int64_t next_id = 1;
    std::deque<Req*> queue;
    std::vector<Req*> active;
    std::unordered_map<int64_t, Req*> all;
    size_t used = 0;
    void* meta[2] = {nullptr, nullptr};
    size_t meta_size[2] = {0, 0};
    struct Tick {
        cudaEvent_t ev;
        std::vector<Req*> finishing;
        int buf;
    };
    std::deque<Tick> inflight;
    std::vector<cudaEvent_t> events;
    int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_ticks = 0, n_launches = 0;
    int64_t n_shared_launches = 0;   // launches that carried work of two or more requests
    int64_t max_per_launch = 0;      // most requests carried by one launch
    std::string err;
};

namespace {

// Work memory of a request, carved from one stream-ordered allocation.
size_t plan_request(ks_server* S, Req* r, bool apply) {
    const bool fp32 = S->fp32;
    const size_t T = fp32 ? 4 : 8;
    const int64_t k = r->k, n = r->n, nn = n * n, ke = k > 1 ? k - 1 : 0;
    const bool small = r->sops != nullptr;
    const int64_t ntri = n * (n + 1) / 2;
    const int64_t CS = small ? ntri + 2 * n + 2 * nn : level_cs((int)n);
    const int64_t RS = small ? ntri + 2 * nn + n : rstore_rs((int)n);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += align256(b);
        return o;
    };
    char* base = (char*)r->arena;
    auto P = [&](size_t o) { return (void*)(base + o); };
    ProbDesc& D = r->desc;
    if (r->follow_of >= 0) {   // covariance follow-up: SelInv store + error words (+ output)
        const size_t o_bad = take(ST_NCODES * sizeof(unsigned long long));
        const size_t o_sx = take((size_t)k * 2 * nn * T);
        const size_t o_cov = take((size_t)k * nn * sizeof(double));
        if (apply) {
            D.bad = (unsigned long long*)P(o_bad);
            D.Sx = P(o_sx);
            r->cov_dev = (double*)P(o_cov);
            D.cov = r->cov_dev;
            cudaMemsetAsync(D.bad, 0xFF, ST_NCODES * sizeof(unsigned long long), S->st);
        }
        return off;
    }
    const size_t o_bad = take(ST_NCODES * sizeof(unsigned long long));
    const size_t o_res = take((size_t)2 * k * sizeof(double));
    const ks_problem& Q = r->prob;
    const unsigned ti = r->synthetic ? (KS_TI_F | KS_TI_H | KS_TI_K | KS_TI_G | KS_TI_C) : Q.time_invariant;
    size_t o_in[7] = {0, 0, 0, 0, 0, 0, 0};
    size_t cnt[7] = {0, 0, 0, 0, 0, 0, 0};
    const double* src[7] = {Q.F, Q.H, Q.c, Q.K, Q.G, Q.o, Q.C};
    const int64_t kf = (ti & KS_TI_F) ? 1 : ke, kh = (ti & KS_TI_H) ? 1 : ke, kk = (ti & KS_TI_K) ? 1 : ke;
    cnt[0] = kf * nn; cnt[1] = kh * nn; cnt[2] = Q.c ? ke * n : 0; cnt[3] = kk * nn;
    cnt[4] = (ti & KS_TI_G) ? (size_t)r->m0 * n : (size_t)r->tot_m * n;
    cnt[5] = r->tot_m;
    cnt[6] = (ti & KS_TI_C) ? (size_t)r->m0 * r->m0 : (size_t)r->tot_m2;
    for (int a = 0; a < 7; ++a) {
        const bool stage_it = r->synthetic ? (a != 2 && cnt[a] > 0) : (src[a] && cnt[a] && !is_device_ptr(src[a]));
        o_in[a] = stage_it ? take(cnt[a] * sizeof(double)) + 1 : 0;
    }
    size_t o_m = 0, o_goff = 0, o_coff = 0;
    if (!r->uniform) {
        o_m = take((size_t)k * sizeof(int32_t));
        o_goff = take((size_t)(k + 1) * sizeof(int64_t));
        o_coff = take((size_t)(k + 1) * sizeof(int64_t));
    }
    const size_t o_l0 = take((size_t)k * CS * T), o_l1 = take((size_t)(k / 2 + 1) * CS * T);
    const size_t o_R = take((size_t)k * RS * T);
    const size_t o_cn = take((size_t)k * n * sizeof(double)), o_cd = take((size_t)k * n * sizeof(double));
    const bool own_u = r->synthetic || !is_device_ptr(Q.u_out);
    const size_t o_u = own_u ? take((size_t)k * n * sizeof(double)) : 0;
    size_t o_LK = 0, o_LC = 0, o_q = 0, o_g = 0, o_w = 0, o_d = 0;
    if (fp32) {
        o_LK = take((size_t)std::max<int64_t>(ke, 1) * nn * sizeof(double));
        o_LC = take((size_t)std::max<int64_t>(r->tot_m2, 1) * sizeof(double));
        o_q = take((size_t)std::max<int64_t>(ke, 1) * n * sizeof(float));
        o_g = take((size_t)k * n * sizeof(float));
        o_w = take((size_t)k * n * sizeof(float));
        o_d = take((size_t)k * n * sizeof(float));
    }
    size_t o_sx = 0, o_cov = 0;
    const bool own_cov = r->want_cov && (r->synthetic || (Q.cov_out && !is_device_ptr(Q.cov_out)));
    if (r->want_cov) {
        o_sx = take((size_t)k * 2 * nn * T);
        if (own_cov) o_cov = take((size_t)k * nn * sizeof(double));
    }
    if (!apply) return off;
    memset(&D, 0, sizeof(D));
    D.ti = ti;
    D.k = k;
    D.n = r->n;
    D.mmax = r->mmax;
    D.L = r->L;
    D.m_uniform = r->uniform ? r->m0 : -1;
    const double* dst[7];
    for (int a = 0; a < 7; ++a) dst[a] = o_in[a] ? (const double*)P(o_in[a] - 1) : src[a];
    D.F = dst[0]; D.H = dst[1]; D.c = r->synthetic ? nullptr : (Q.c ? dst[2] : nullptr); D.K = dst[3];
    D.G = dst[4]; D.o = dst[5]; D.C = dst[6];
    if (!r->uniform) {
        D.m = (const int32_t*)P(o_m);
        D.goff = (const int64_t*)P(o_goff);
        D.coff = (const int64_t*)P(o_coff);
    }
    D.lvl[0] = P(o_l0);
    D.lvl[1] = P(o_l1);
    D.R = P(o_R);
    D.resid = (double*)P(o_res);
    D.cn2 = (double*)P(o_cn);
    D.cd2 = (double*)P(o_cd);
    D.u = own_u ? (double*)P(o_u) : Q.u_out;
    r->u_host = (!r->synthetic && own_u) ? Q.u_out : nullptr;
    if (fp32) {
        D.LK = (double*)P(o_LK);
        D.LC = (double*)P(o_LC);
        D.q = P(o_q);
        D.g = P(o_g);
        D.w = P(o_w);
        D.d = P(o_d);
    }
    if (r->want_cov) {
        D.Sx = P(o_sx);
        r->cov_dev = own_cov ? (double*)P(o_cov) : Q.cov_out;
        D.cov = r->cov_dev;
        r->cov_host = (!r->synthetic && own_cov) ? Q.cov_out : nullptr;
    }
    D.bad = (unsigned long long*)P(o_bad);
    // stage the inputs (copies or generation) and clear what must start at zero
    cudaStream_t st = S->st;
    if (r->synthetic) {
        launch_generate(k, r->n, r->m0, r->seed, 0.99, (double*)dst[0], (double*)dst[1], (double*)dst[3],
                        (double*)dst[4], (double*)dst[6], (double*)dst[5], st);
    } else {
        for (int a = 0; a < 7; ++a)
            if (o_in[a]) cudaMemcpyAsync(P(o_in[a] - 1), src[a], cnt[a] * sizeof(double), cudaMemcpyHostToDevice, st);
        if (!r->uniform) {
            cudaMemcpyAsync(P(o_m), r->m_copy.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(P(o_goff), r->offs.data(), (size_t)(k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(P(o_coff), r->offs.data() + k + 1, (size_t)(k + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, st);
        }
    }
    cudaMemsetAsync(D.bad, 0xFF, ST_NCODES * sizeof(unsigned long long), st);
    cudaMemsetAsync(D.resid, 0, (size_t)k * sizeof(double), st);
    return off;
}

void make_stages(ks_server* S, Req* r) {
    r->stages.clear();
    const int L = r->L;
    if (r->follow_of >= 0) {
        for (int l = L; l >= 0; --l) r->stages.push_back({B_SELINV, l});
        return;
    }
    r->stages.push_back({B_WHITEN, 0});
    for (int l = 0; l < L; ++l) r->stages.push_back({B_LEVEL, l});
    r->stages.push_back({B_BASE, 0});
    for (int l = L; l >= 0; --l) r->stages.push_back({B_BACKSUB, l});
    if (S->fp32) {
        r->stages.push_back({B_REFINE_Q, 0});
        r->stages.push_back({B_REFINE_G, 0});
        for (int l = 0; l <= L; ++l) r->stages.push_back({B_RT_SOLVE, l});
        for (int l = L; l >= 0; --l) r->stages.push_back({B_BACKSUB_W, l});
        r->stages.push_back({B_ADD, 0});
    }
    if (r->want_cov)
        for (int l = L; l >= 0; --l) r->stages.push_back({B_SELINV, l});
}

cudaEvent_t take_event(ks_server* S) {
    if (!S->events.empty()) {
        cudaEvent_t e = S->events.back();
        S->events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// One tick over the schedulable requests: per group and kind of stage one launch.
void issue_tick(ks_server* S, const std::vector<Req*>& sched) {
    struct Launch {
        int n;
        const SmallOps* sops;
        int mmax;
        int op;
        std::vector<int> idx;
    };
    std::vector<Launch> launches;
    std::map<std::tuple<int, const SmallOps*, int>, size_t> where;
    for (size_t i = 0; i < sched.size(); ++i) {
        Req* r = sched[i];
        const int op = r->stages[r->stage].first;
        auto key = std::make_tuple(r->n, r->sops, op);
        auto it = where.find(key);
        if (it == where.end()) {
            it = where.emplace(key, launches.size()).first;
            launches.push_back({r->n, r->sops, 0, op, {}});
        }
        Launch& L = launches[it->second];
        L.mmax = std::max(L.mmax, r->mmax);
        L.idx.push_back((int)i);
    }
    // meta blob: descriptors, then per launch (work, probs, offsets)
    size_t off = align256(sched.size() * sizeof(ProbDesc));
    std::vector<size_t> o_work(launches.size()), o_probs(launches.size()), o_off(launches.size());
    for (size_t l = 0; l < launches.size(); ++l) {
        o_work[l] = off;
        off += align256(sizeof(BatchWork));
        o_probs[l] = off;
        off += align256(launches[l].idx.size() * sizeof(int));
        o_off[l] = off;
        off += align256((launches[l].idx.size() + 1) * sizeof(int64_t));
    }
    const int b = S->inflight.empty() ? 0 : 1 - S->inflight.back().buf;
    if (off > S->meta_size[b]) {
        if (S->meta[b]) cudaFreeAsync(S->meta[b], S->st);
        S->meta[b] = nullptr;
        cudaMallocAsync(&S->meta[b], off * 2, S->st);
        S->meta_size[b] = off * 2;
    }
    char* meta = (char*)S->meta[b];
    std::vector<char> blob(off, 0);
    for (size_t i = 0; i < sched.size(); ++i) {
        ProbDesc d = sched[i]->desc;
        d.cur_level = sched[i]->stages[sched[i]->stage].second;
        memcpy(blob.data() + i * sizeof(ProbDesc), &d, sizeof(ProbDesc));
    }
    for (size_t l = 0; l < launches.size(); ++l) {
        BatchWork w;
        w.desc = (const ProbDesc*)meta;
        w.probs = (const int*)(meta + o_probs[l]);
        w.off = (const int64_t*)(meta + o_off[l]);
        w.np = (int)launches[l].idx.size();
        w.level = -1;
        memcpy(blob.data() + o_work[l], &w, sizeof(w));
        memcpy(blob.data() + o_probs[l], launches[l].idx.data(), launches[l].idx.size() * sizeof(int));
        int64_t* o = (int64_t*)(blob.data() + o_off[l]);
        o[0] = 0;
        for (size_t i = 0; i < launches[l].idx.size(); ++i) {
            Req* r = sched[launches[l].idx[i]];
            o[i + 1] = o[i] + units_of(launches[l].op, r->stages[r->stage].second, r->k, r->n);
        }
    }
    cudaMemcpyAsync(meta, blob.data(), off, cudaMemcpyHostToDevice, S->st);
    for (size_t l = 0; l < launches.size(); ++l) {
        const Launch& L = launches[l];
        const BatchWork* wk = (const BatchWork*)(meta + o_work[l]);
        const bool per_block = L.sops == nullptr &&
                               (L.op == B_WHITEN || L.op == B_LEVEL || L.op == B_BASE || L.op == B_SELINV);
        const unsigned grid = (unsigned)(S->nsm * (per_block ? 8 : 16));
        if (L.sops)
            L.sops->batch(L.op, wk, S->fp32, grid, S->st);
        else
            launch_batch_generic(L.op, L.n, L.mmax, wk, S->fp32, grid, S->st);
    }
    S->n_launches += (int64_t)launches.size();
    S->n_ticks++;
    for (const Launch& L : launches) {
        const int64_t np = (int64_t)L.idx.size();
        if (np >= 2) S->n_shared_launches++;
        if (np > S->max_per_launch) S->max_per_launch = np;
    }
    ks_server::Tick t;
    t.ev = take_event(S);
    t.buf = b;
    cudaEventRecord(t.ev, S->st);
    for (Req* r : sched) {
        r->stage++;
        if (r->stage == r->stages.size()) {
            r->state = 2;
            t.finishing.push_back(r);
        }
    }
    S->inflight.push_back(t);
}

// Completes the oldest in-flight tick: statuses and outputs of the requests that finished in it.
void complete_oldest(ks_server* S) {
    ks_server::Tick t = S->inflight.front();
    S->inflight.pop_front();
    cudaEventSynchronize(t.ev);
    if (!t.finishing.empty()) {
        std::vector<unsigned long long> words(t.finishing.size() * ST_NCODES);
        cudaStreamWaitEvent(S->cst, t.ev, 0);
        for (size_t i = 0; i < t.finishing.size(); ++i) {
            Req* r = t.finishing[i];
            cudaMemcpyAsync(words.data() + i * ST_NCODES, r->desc.bad, ST_NCODES * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, S->cst);
            if (r->u_host)
                cudaMemcpyAsync(r->u_host, r->desc.u, (size_t)r->k * r->n * sizeof(double), cudaMemcpyDeviceToHost, S->cst);
            if (r->cov_host && r->follow_of < 0)
                cudaMemcpyAsync(r->cov_host, r->cov_dev, (size_t)r->k * r->n * r->n * sizeof(double),
                                cudaMemcpyDeviceToHost, S->cst);
            if (r->follow_of >= 0 && r->cov_host)
                cudaMemcpyAsync(r->cov_host, r->cov_dev, (size_t)r->k * r->n * r->n * sizeof(double),
                                cudaMemcpyDeviceToHost, S->cst);
        }
        cudaStreamSynchronize(S->cst);
        std::lock_guard<std::mutex> lk(S->mu);
            const auto now = Clock::now();
        for (size_t i = 0; i < t.finishing.size(); ++i) {
            Req* r = t.finishing[i];
            for (int code : status_order)
                if (words[i * ST_NCODES + code] != ~0ULL) {
                    r->status = code;
                    r->info = (int64_t)words[i * ST_NCODES + code];
                    break;
                }
            r->t_done = now;
            r->state = 3;
            S->n_completed++;
            if (r->follow_of >= 0) {
                auto b = S->all.find(r->follow_of);
                if (b != S->all.end()) b->second->followers--;
            }
            S->active.erase(std::find(S->active.begin(), S->active.end(), r));
            const bool keep = S->opt.keep_factors && r->follow_of < 0 && r->status == KS_OK;
            if (!keep && r->follow_of < 0 && !r->synthetic) {
                cudaFreeAsync(r->arena, S->st);
                S->used -= r->bytes;
                r->arena = nullptr;
            }
        }
        S->cv_done.notify_all();
    }
    S->events.push_back(t.ev);
}

void scheduler(ks_server* S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        auto schedulable = [&]() {
            for (Req* r : S->active)
                if (r->state == 1) return true;
            return false;
        };
        S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || schedulable() || !S->inflight.empty(); });
        if (S->stop && S->queue.empty() && S->active.empty() && S->inflight.empty()) break;
        // Admission.  Covariance follow-ups go first, from any queue position: they run on a
        // factor that is already resident, and the caller may hold that factor (and its memory)
        // until the follow-up is done, so a follow-up waiting behind a new request that needs
        // that memory would never be admitted.  New requests then go in arrival order.
        auto fail_oom = [&](Req* r) {
            r->status = KS_ERR_OOM;
            r->state = 3;
            r->t_done = Clock::now();
            S->n_completed++;
            S->cv_done.notify_all();
        };
        // Allocates and plans r (removed from the queue by the caller); 0 admitted, 1 no memory
        // now (r not admitted), 2 rejected with KS_ERR_OOM.
        auto admit = [&](Req* r, size_t need) -> int {
            lk.unlock();
            void* p = nullptr;
            const cudaError_t e = cudaMallocAsync(&p, need, S->st);
            lk.lock();
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (S->active.empty() && S->inflight.empty()) {   // nothing will free memory
                    fail_oom(r);
                    return 2;
                }
                return 1;
            }
            r->arena = p;
            r->bytes = need;
            S->used += need;
            lk.unlock();
            plan_request(S, r, true);
            lk.lock();
            make_stages(S, r);
            r->stage = 0;
            r->state = 1;
            r->t_admit = Clock::now();
            S->n_admitted++;
            S->active.push_back(r);
            return 0;
        };
        const size_t budget = S->opt.mem_budget;
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            Req* r = *it;
            if (r->follow_of < 0) {
                ++it;
                continue;
            }
            const size_t need = plan_request(S, r, false);
            if (need > budget) {
                it = S->queue.erase(it);
                fail_oom(r);
                continue;
            }
            if ((int)S->active.size() >= S->opt.max_active || S->used + need > budget) {
                ++it;
                continue;
            }
            const size_t pos = (size_t)(it - S->queue.begin());
            S->queue.erase(it);
            if (admit(r, need) == 1) {
                S->queue.insert(S->queue.begin() + pos, r);
                break;
            }
            it = S->queue.begin() + pos;
        }
        while (!S->queue.empty()) {
            Req* r = S->queue.front();
            const size_t need = plan_request(S, r, false);
            if (need > budget) {
                S->queue.pop_front();
                fail_oom(r);
                continue;
            }
            if ((int)S->active.size() >= S->opt.max_active || S->used + need > budget) break;
            S->queue.pop_front();
            if (admit(r, need) == 1) {
                S->queue.push_front(r);
                break;
            }
        }
        std::vector<Req*> sched;
        for (Req* r : S->active)
            if (r->state == 1) sched.push_back(r);
        lk.unlock();
        if (!sched.empty()) {
            while (S->inflight.size() >= 2) complete_oldest(S);
            issue_tick(S, sched);
        } else if (!S->inflight.empty()) {
            complete_oldest(S);
        }
        lk.lock();
    }
}

Req* find_req(ks_server* S, int64_t id) {
    auto it = S->all.find(id);
    return it == S->all.end() ? nullptr : it->second;
}

ks_status fill_shape(ks_server* S, Req* r) {
    const int maxn = std::min(max_n_for(S->ctx), LARGE_NMAX);   // batched kernels stop at 128
    if (r->k < 1 || r->n < 1 || r->n > maxn) {
        S->err = "bad k or n";
        return KS_ERR_ARG;
    }
    r->L = floor_log2(r->k);
    if (r->synthetic) {
        r->mmax = r->m0;
        r->tot_m = r->k * r->m0;
        r->tot_m2 = r->k * (int64_t)r->m0 * r->m0;
        r->uniform = true;
    } else {
        const ks_problem& Q = r->prob;
        if (!Q.m || !Q.u_out || (r->k > 1 && (!Q.F || !Q.H || !Q.K))) {
            S->err = "missing arrays";
            return KS_ERR_ARG;
        }
        r->m_copy.assign(Q.m, Q.m + r->k);
        r->m0 = Q.m[0];
        const int maxm = max_m_for(S->ctx, r->n);
        for (int32_t mi : r->m_copy) {
            if (mi < 0 || mi > maxm) {
                S->err = "bad m";
                return KS_ERR_ARG;
            }
            r->mmax = std::max(r->mmax, (int)mi);
            r->tot_m += mi;
            r->tot_m2 += (int64_t)mi * mi;
            r->uniform = r->uniform && mi == r->m0;
        }
        if (r->tot_m > 0 && (!Q.G || !Q.o || !Q.C)) {
            S->err = "missing G / o / C";
            return KS_ERR_ARG;
        }
        if ((Q.time_invariant & (KS_TI_G | KS_TI_C)) && !r->uniform) {
            S->err = "time-invariant G / C need uniform m";
            return KS_ERR_ARG;
        }
        r->want_cov = Q.cov_out != nullptr;
        if (!r->uniform) {
            r->offs.resize(2 * (r->k + 1));
            r->offs[0] = r->offs[r->k + 1] = 0;
            for (int64_t i = 0; i < r->k; ++i) {
                r->offs[i + 1] = r->offs[i] + r->m_copy[i];
                r->offs[r->k + 1 + i + 1] = r->offs[r->k + 1 + i] + (int64_t)r->m_copy[i] * r->m_copy[i];
            }
        }
        r->prob.m = r->m_copy.data();
    }
    r->sops = (r->mmax <= r->n) ? small_ops(r->n) : nullptr;
    return KS_OK;
}

ks_status enqueue(ks_server* S, Req* r, int64_t* id) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    S->all[r->id] = r;
    S->queue.push_back(r);
    S->n_submitted++;
    if (id) *id = r->id;
    S->cv_work.notify_one();
    return KS_OK;
}

}  // namespace

extern "C" {

ks_status ks_server_create(ks_ctx* ctx, const ks_server_options* opt, ks_server** out) {
    if (!ctx || !out) return KS_ERR_ARG;
    *out = nullptr;
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    ks_server* S = new ks_server();
    S->ctx = ctx;
    if (opt) S->opt = *opt;
    S->fp32 = ctx->precision == KS_FP32_REFINE;
    cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (S->opt.max_active <= 0) S->opt.max_active = 4096;
    if (S->opt.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->opt.mem_budget = fr / 4 * 3;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t thr = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->cst, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return fail(ctx, KS_ERR_CUDA, "cannot create the server streams");
    }
    S->thr = std::thread(scheduler, S);
    *out = S;
    return KS_OK;
}

ks_status ks_server_submit(ks_server* S, const ks_problem* prob, int64_t* id) {
    if (!S || !prob) return KS_ERR_ARG;
    Req* r = new Req();
    r->prob = *prob;
    r->k = prob->k;
    r->n = prob->n;
    const ks_status s = fill_shape(S, r);
    if (s != KS_OK) {
        delete r;
        return s;
    }
    return enqueue(S, r, id);
}

ks_status ks_server_submit_synthetic(ks_server* S, int64_t k, int n, int m, uint64_t seed,
                                     int want_cov, int64_t* id) {
    if (!S || m < 0) return KS_ERR_ARG;
    Req* r = new Req();
    r->synthetic = true;
    r->k = k;
    r->n = n;
    r->m0 = m;
    r->seed = seed;
    r->want_cov = want_cov;
    if (m > max_m_for(S->ctx, n)) {
        delete r;
        return KS_ERR_ARG;
    }
    const ks_status s = fill_shape(S, r);
    if (s != KS_OK) {
        delete r;
        return s;
    }
    return enqueue(S, r, id);
}

ks_status ks_server_covariances(ks_server* S, int64_t id, double* cov_out, int64_t* follow_id) {
    if (!S) return KS_ERR_ARG;
    Req* base;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        base = find_req(S, id);
        if (!base || base->state != 3 || base->follow_of >= 0 || base->arena == nullptr) return KS_ERR_NO_FACTOR;
        base->followers++;
    }
    Req* r = new Req();
    r->follow_of = id;
    r->k = base->k;
    r->n = base->n;
    r->L = base->L;
    r->mmax = base->mmax;
    r->sops = base->sops;
    r->desc = base->desc;   // its factor; plan_request(apply) sets the SelInv store and output
    r->cov_host = (cov_out && !is_device_ptr(cov_out)) ? cov_out : nullptr;
    r->want_cov = 1;
    return enqueue(S, r, follow_id);
}

ks_status ks_server_wait(ks_server* S, int64_t id, double timeout_ms, ks_request_info* out) {
    if (!S) return KS_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    Req* r = find_req(S, id);
    if (!r) return KS_ERR_ARG;
    auto ready = [&] { return r->state == 3; };
    if (timeout_ms < 0)
        S->cv_done.wait(lk, ready);
    else
        S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
    if (out) {
        out->done = r->state == 3;
        out->status = r->status;
        out->info = r->info;
        out->k = r->k;
        out->n = r->n;
        const auto t_admit = r->state >= 1 ? r->t_admit : Clock::now();
        out->queue_ms = std::chrono::duration<double, std::milli>(t_admit - r->t_submit).count();
        out->latency_ms = r->state == 3 ? std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count() : -1.0;
    }
    return r->state == 3 ? (ks_status)r->status : KS_ERR_TIMEOUT;
}

ks_status ks_server_result(ks_server* S, int64_t id, double* u_out, double* cov_out) {
    if (!S) return KS_ERR_ARG;
    Req* r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r = find_req(S, id);
        if (!r || r->state != 3 || r->arena == nullptr) return KS_ERR_NO_FACTOR;
    }
    if (u_out && r->follow_of < 0)
        KS_CUDA(S->ctx, cudaMemcpyAsync(u_out, r->desc.u, (size_t)r->k * r->n * sizeof(double), cudaMemcpyDefault, S->cst));
    if (cov_out && r->cov_dev)
        KS_CUDA(S->ctx, cudaMemcpyAsync(cov_out, r->cov_dev, (size_t)r->k * r->n * r->n * sizeof(double),
                                        cudaMemcpyDefault, S->cst));
    KS_CUDA(S->ctx, cudaStreamSynchronize(S->cst));
    return KS_OK;
}

ks_status ks_server_release(ks_server* S, int64_t id) {
    if (!S) return KS_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Req* r = find_req(S, id);
    if (!r) return KS_ERR_ARG;
    if (r->state != 3 || r->followers > 0) return KS_ERR_ARG;   // still running, or a follow-up uses its factor
    if (r->arena) {
        cudaFreeAsync(r->arena, S->st);
        S->used -= r->bytes;
        r->arena = nullptr;
    }
    S->all.erase(id);
    delete r;
    return KS_OK;
}

ks_status ks_server_stats(ks_server* S, ks_server_counters* out) {
    if (!S || !out) return KS_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->n_submitted;
    out->admitted = S->n_admitted;
    out->completed = S->n_completed;
    out->active = (int64_t)S->active.size();
    out->queued = (int64_t)S->queue.size();
    out->ticks = S->n_ticks;
    out->launches = S->n_launches;
    out->shared_launches = S->n_shared_launches;
    out->max_requests_per_launch = S->max_per_launch;
    out->bytes_in_use = S->used;
    out->bytes_budget = S->opt.mem_budget;
    return KS_OK;
}

ks_status ks_server_destroy(ks_server* S) {
    if (!S) return KS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->thr.joinable()) S->thr.join();
    cudaSetDevice(S->ctx->device);
    cudaStreamSynchronize(S->st);
    for (auto& kv : S->all) {
        if (kv.second->arena) cudaFreeAsync(kv.second->arena, S->st);
        delete kv.second;
    }
    for (int b = 0; b < 2; ++b)
        if (S->meta[b]) cudaFreeAsync(S->meta[b], S->st);
    cudaStreamSynchronize(S->st);
    for (cudaEvent_t e : S->events) cudaEventDestroy(e);
    cudaStreamDestroy(S->st);
    cudaStreamDestroy(S->cst);
    delete S;
    return KS_OK;
}

ks_status ks_generate(ks_ctx* ctx, int64_t k, int n, int m, uint64_t seed, double f_scale,
                      double* F, double* H, double* K, double* G, double* C, double* o) {
    if (!ctx || k < 1 || n < 1 || m < 0 || !F || !H || !K || (m > 0 && (!G || !C || !o))) return KS_ERR_ARG;
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    KS_CUDA(ctx, launch_generate(k, n, m, seed, f_scale, F, H, K, G, C, o, ctx->stream));
    if (ctx->sync) KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return KS_OK;
}

ks_status ks_generate_steps(ks_ctx* ctx, int64_t k, int n, int m, uint64_t seed, double f_scale,
                            double* F, double* H, double* K, double* G, double* C, double* o) {
    if (!ctx || k < 1 || n < 1 || m < 0 || (k > 1 && (!F || !H || !K)) ||
        (m > 0 && (!G || !C || !o)))
        return KS_ERR_ARG;
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    KS_CUDA(ctx, launch_generate_steps(k, n, m, seed, f_scale, F, H, K, G, C, o, ctx->stream));
    if (ctx->sync) KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return KS_OK;
}

}  // extern "C"

// ks_var.cu -- ks_smooth_var / ks_covariances_var: problems whose state dimension varies from
// step to step, with rectangular H_i (Section 2: u_i has n_i entries, evolution equation i has
// l_i rows, H_i is l_i x n_{i+1}; Section 3: block rows and block columns may have any sizes).
//
// GB300 design: the odd-even kernels run on uniform tiles, so a variable-dimension problem is
// embedded, on the device, into a uniform one of dimension N = max_i max(n_i, l_i):
//   * state i becomes u'_i = [u_i ; z_i] with N - n_i padding components z_i;
//   * every padding component gets one observation row  1 * z = 0  with unit variance, so it is
//     determined (z = 0) and coupled to nothing else;
//   * evolution equation i keeps its l_i rows, padded with zero columns for the padding
//     components, and N - l_i zero rows (unit variance, zero right-hand side) are appended.
// The whitened matrix of the padded problem is, up to a permutation of columns and zero rows,
// diag(U A, I): the normal matrix is block diagonal between real and padding components, so
// the smoothed states and their covariance blocks are exactly those of the original problem.
// The cost is the uniform problem's, (N / n_i)^3 per step at worst: worth it while the
// dimensions stay within a small factor of each other, which is the regime of this interface.
// pad_kernel builds the padded arrays (one thread block per step); unpad kernels gather the
// states and covariance blocks back into the caller's packed layout.
#include <numeric>

#include "ks_host.h"

using namespace kshost;

namespace {

// Per-step offsets into the caller's packed arrays and into the padded ones.
struct VarOffsets {
    const int32_t *nd, *l, *m;       // [k], [k-1], [k]
    const int64_t *fo, *ho, *eo, *ko;  // evolution i: F, H, c, K offsets [k]
    const int64_t *gv, *go, *co;     // observation i: G values, o rows, C values [k]
    const int64_t *pgo, *pco;        // padded observation i: rows, C values [k]
};

__global__ void pad_kernel(int64_t k, int N, VarOffsets off, const double* F, const double* H,
                           const double* c, const double* K, const double* G, const double* o,
                           const double* C, double* Fp, double* Hp, double* cp, double* Kp,
                           double* Gp, double* op, double* Cp) {
    const int64_t NN = (int64_t)N * N;
    for (int64_t i = blockIdx.x; i < k; i += gridDim.x) {
        const int ni = off.nd[i], mi = off.m[i], mp = mi + (N - ni);
        if (i + 1 < k) {
            const int li = off.l[i], nj = off.nd[i + 1];
            double* Fi = Fp + i * NN;
            double* Hi = Hp + i * NN;
            double* Ki = Kp + i * NN;
            for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
                const int r = e / N, q = e - r * N;
                Fi[e] = (r < li && q < ni) ? F[off.fo[i] + (int64_t)r * ni + q] : 0.0;
                Hi[e] = (r < li && q < nj) ? H[off.ho[i] + (int64_t)r * nj + q] : 0.0;
                Ki[e] = (r < li && q < li) ? K[off.ko[i] + (int64_t)r * li + q] : (r == q ? 1.0 : 0.0);
            }
            for (int r = threadIdx.x; r < N; r += blockDim.x)
                cp[i * N + r] = (c != nullptr && r < li) ? c[off.eo[i] + r] : 0.0;
        }
        double* Gi = Gp + off.pgo[i] * N;
        for (int64_t e = threadIdx.x; e < (int64_t)mp * N; e += blockDim.x) {
            const int r = (int)(e / N), q = (int)(e - (int64_t)r * N);
            double v;
            if (r < mi) v = q < ni ? G[off.gv[i] + (int64_t)r * ni + q] : 0.0;
            else v = (q == ni + (r - mi)) ? 1.0 : 0.0;   // padding component r - mi
            Gi[e] = v;
        }
        for (int r = threadIdx.x; r < mp; r += blockDim.x) op[off.pgo[i] + r] = r < mi ? o[off.go[i] + r] : 0.0;
        double* Ci = Cp + off.pco[i];
        for (int64_t e = threadIdx.x; e < (int64_t)mp * mp; e += blockDim.x) {
            const int r = (int)(e / mp), q = (int)(e - (int64_t)r * mp);
            Ci[e] = (r < mi && q < mi) ? C[off.co[i] + (int64_t)r * mi + q] : (r == q ? 1.0 : 0.0);
        }
    }
}

// u_out[uoff_i + q] = up[i][q], q < n_i (one thread per padded entry).
__global__ void unpad_states_kernel(int64_t k, int N, const int32_t* nd, const int64_t* uoff,
                                    const double* up, double* u) {
    const int64_t total = k * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N;
        const int q = (int)(e - i * N);
        if (q < nd[i]) u[uoff[i] + q] = up[e];
    }
}

// cov[soff_i + r n_i + q] = Sp[i][r][q], r, q < n_i.
__global__ void unpad_cov_kernel(int64_t k, int N, const int32_t* nd, const int64_t* soff,
                                 const double* Sp, double* cov) {
    const int64_t NN = (int64_t)N * N, total = k * NN;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / NN;
        const int rq = (int)(e - i * NN), r = rq / N, q = rq - r * N;
        const int ni = nd[i];
        if (r < ni && q < ni) cov[soff[i] + (int64_t)r * ni + q] = Sp[e];
    }
}

unsigned grid_for(int64_t work, int per_block) {
    const int64_t b = (work + per_block - 1) / per_block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

namespace {
// Grows ctx's variable-dimension buffer (kept apart from the work memory, which ks_smooth may
// reallocate while the padded inputs are in use).
ks_status var_reserve(ks_ctx* ctx, size_t bytes, char** out) {
    if (bytes > ctx->vbuf_size) {
        KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->vbuf) cudaFree(ctx->vbuf);
        ctx->vbuf = nullptr;
        ctx->vbuf_size = 0;
        KS_CUDA(ctx, cudaMalloc(&ctx->vbuf, bytes));
        ctx->vbuf_size = bytes;
    }
    *out = (char*)ctx->vbuf;
    return KS_OK;
}
}  // namespace

extern "C" {

ks_status ks_smooth_var(ks_ctx* ctx, int64_t k, const int32_t* nd, const int32_t* l,
                        const int32_t* m, const double* F, const double* H, const double* c,
                        const double* K, const double* G, const double* o, const double* C,
                        double* u_out, ks_handle* keep, int64_t* info) {
    if (!ctx) return KS_ERR_ARG;
    if (info) *info = -1;
    ctx->err.clear();
    if (k < 1) return fail(ctx, KS_ERR_ARG, "k must be >= 1 (got %lld)", (long long)k);
    if (!nd || !m || !u_out || (k > 1 && !l)) return fail(ctx, KS_ERR_ARG, "nd, l, m and u_out must not be NULL");
    int N = 0;
    int64_t sF = 0, sH = 0, sc = 0, sK = 0, sG = 0, so = 0, sC = 0, sU = 0;
    for (int64_t i = 0; i < k; ++i) {
        if (nd[i] < 1) return fail(ctx, KS_ERR_ARG, "nd[%lld] = %d must be >= 1", (long long)i, nd[i]);
        if (m[i] < 0) return fail(ctx, KS_ERR_ARG, "m[%lld] = %d must be >= 0", (long long)i, m[i]);
        N = std::max(N, (int)nd[i]);
        sU += nd[i];
        sG += (int64_t)m[i] * nd[i];
        so += m[i];
        sC += (int64_t)m[i] * m[i];
        if (i + 1 < k) {
            if (l[i] < 0) return fail(ctx, KS_ERR_ARG, "l[%lld] = %d must be >= 0", (long long)i, l[i]);
            N = std::max(N, (int)l[i]);
            sF += (int64_t)l[i] * nd[i];
            sH += (int64_t)l[i] * nd[i + 1];
            sc += l[i];
            sK += (int64_t)l[i] * l[i];
        }
    }
    const int maxn = ks_max_n(ctx);
    if (N > maxn)
        return fail(ctx, KS_ERR_ARG, "max(n_i, l_i) = %d above the largest supported state dimension %d", N, maxn);
    const int maxm = ks_max_m(ctx, N);
    for (int64_t i = 0; i < k; ++i)
        if (m[i] + (N - nd[i]) > maxm)
            return fail(ctx, KS_ERR_ARG,
                        "step %lld: m_i + (N - n_i) = %d above %d (padded to N = %d, every padding "
                        "component takes one observation row)", (long long)i, m[i] + (N - nd[i]), maxm, N);
    if (sK > 0 && (!F || !H || !K)) return fail(ctx, KS_ERR_ARG, "F, H and K must not be NULL when some l_i > 0");
    if (so > 0 && (!G || !o || !C)) return fail(ctx, KS_ERR_ARG, "G, o and C must not be NULL when some m_i > 0");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));

    // Host offsets (caller layout and padded layout).
    std::vector<int64_t> fo(k), ho(k), eo(k), ko(k), gv(k), go(k), co(k), pgo(k + 1), pco(k + 1), uoff(k + 1);
    std::vector<int32_t> mp(k), lv(k, 0);
    {
        int64_t a = 0, b = 0, e = 0, q = 0, g1 = 0, g2 = 0, g3 = 0;
        pgo[0] = pco[0] = uoff[0] = 0;
        for (int64_t i = 0; i < k; ++i) {
            fo[i] = a; ho[i] = b; eo[i] = e; ko[i] = q; gv[i] = g1; go[i] = g2; co[i] = g3;
            if (i + 1 < k) {
                lv[i] = l[i];
                a += (int64_t)l[i] * nd[i];
                b += (int64_t)l[i] * nd[i + 1];
                e += l[i];
                q += (int64_t)l[i] * l[i];
            }
            g1 += (int64_t)m[i] * nd[i];
            g2 += m[i];
            g3 += (int64_t)m[i] * m[i];
            mp[i] = m[i] + (N - nd[i]);
            pgo[i + 1] = pgo[i] + mp[i];
            pco[i + 1] = pco[i] + (int64_t)mp[i] * mp[i];
            uoff[i + 1] = uoff[i] + nd[i];
        }
    }
    const int64_t ke = k > 1 ? k - 1 : 0;
    const int64_t NN = (int64_t)N * N;
    Plan plan;
    const size_t o_nd = plan.take(k * sizeof(int32_t)), o_l = plan.take(k * sizeof(int32_t)),
                 o_m = plan.take(k * sizeof(int32_t));
    size_t o_off[9];
    for (int j = 0; j < 9; ++j) o_off[j] = plan.take((size_t)k * sizeof(int64_t));
    const size_t o_uoff = plan.take((size_t)(k + 1) * sizeof(int64_t));
    struct Src { const double* p; int64_t count; size_t off; bool dev; };
    Src src[7] = {{F, sF, 0, true}, {H, sH, 0, true}, {c, sc, 0, true}, {K, sK, 0, true},
                  {G, sG, 0, true}, {o, so, 0, true}, {C, sC, 0, true}};
    for (auto& s : src) {
        s.dev = s.p == nullptr || s.count == 0 || is_device_ptr(s.p);
        if (!s.dev) s.off = plan.take((size_t)s.count * sizeof(double));
    }
    const size_t o_Fp = plan.take((size_t)std::max<int64_t>(ke, 1) * NN * 8);
    const size_t o_Hp = plan.take((size_t)std::max<int64_t>(ke, 1) * NN * 8);
    const size_t o_cp = plan.take((size_t)std::max<int64_t>(ke, 1) * N * 8);
    const size_t o_Kp = plan.take((size_t)std::max<int64_t>(ke, 1) * NN * 8);
    const size_t o_Gp = plan.take((size_t)std::max<int64_t>(pgo[k], 1) * N * 8);
    const size_t o_op = plan.take((size_t)std::max<int64_t>(pgo[k], 1) * 8);
    const size_t o_Cp = plan.take((size_t)std::max<int64_t>(pco[k], 1) * 8);
    const size_t o_up = plan.take((size_t)k * N * 8);
    const bool u_dev = is_device_ptr(u_out);
    const size_t o_u = u_dev ? 0 : plan.take((size_t)sU * 8);
    char* vb = nullptr;
    ks_status rs = var_reserve(ctx, plan.off, &vb);
    if (rs != KS_OK) return rs;
    cudaStream_t st = ctx->stream;
    KS_CUDA(ctx, cudaMemcpyAsync(vb + o_nd, nd, k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    KS_CUDA(ctx, cudaMemcpyAsync(vb + o_l, lv.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    KS_CUDA(ctx, cudaMemcpyAsync(vb + o_m, m, k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const std::vector<int64_t>* offs[9] = {&fo, &ho, &eo, &ko, &gv, &go, &co, &pgo, &pco};
    for (int j = 0; j < 9; ++j)
        KS_CUDA(ctx, cudaMemcpyAsync(vb + o_off[j], offs[j]->data(), k * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    KS_CUDA(ctx, cudaMemcpyAsync(vb + o_uoff, uoff.data(), (k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    const double* d[7];
    for (int j = 0; j < 7; ++j) {
        if (src[j].dev) {
            d[j] = src[j].count > 0 ? src[j].p : nullptr;
        } else {
            KS_CUDA(ctx, cudaMemcpyAsync(vb + src[j].off, src[j].p, (size_t)src[j].count * 8, cudaMemcpyHostToDevice, st));
            d[j] = (const double*)(vb + src[j].off);
        }
    }
    VarOffsets vo;
    vo.nd = (const int32_t*)(vb + o_nd);
    vo.l = (const int32_t*)(vb + o_l);
    vo.m = (const int32_t*)(vb + o_m);
    vo.fo = (const int64_t*)(vb + o_off[0]);
    vo.ho = (const int64_t*)(vb + o_off[1]);
    vo.eo = (const int64_t*)(vb + o_off[2]);
    vo.ko = (const int64_t*)(vb + o_off[3]);
    vo.gv = (const int64_t*)(vb + o_off[4]);
    vo.go = (const int64_t*)(vb + o_off[5]);
    vo.co = (const int64_t*)(vb + o_off[6]);
    vo.pgo = (const int64_t*)(vb + o_off[7]);
    vo.pco = (const int64_t*)(vb + o_off[8]);
    double* Fp = (double*)(vb + o_Fp);
    double* Hp = (double*)(vb + o_Hp);
    double* cp = (double*)(vb + o_cp);
    double* Kp = (double*)(vb + o_Kp);
    double* Gp = (double*)(vb + o_Gp);
    double* op = (double*)(vb + o_op);
    double* Cp = (double*)(vb + o_Cp);
    double* up = (double*)(vb + o_up);
    {
        Phase ph(ctx, KS_PHASE_COPY);
        pad_kernel<<<grid_for(k, 1), 128, 0, st>>>(k, N, vo, d[0], d[1], d[2], d[3], d[4], d[5], d[6],
                                                  Fp, Hp, cp, Kp, Gp, op, Cp);
        ++t_launches;
        KS_CUDA(ctx, cudaGetLastError());
    }
    ks_status s = ks_smooth(ctx, k, N, mp.data(), Fp, Hp, cp, Kp, Gp, op, Cp, up, keep, info);
    if (s != KS_OK) return s;
    {
        Phase ph(ctx, KS_PHASE_COPY);
        double* u = u_dev ? u_out : (double*)(vb + o_u);
        unpad_states_kernel<<<grid_for(k * N, 256), 256, 0, st>>>(k, N, vo.nd, (const int64_t*)(vb + o_uoff), up, u);
        ++t_launches;
        KS_CUDA(ctx, cudaGetLastError());
        if (!u_dev) KS_CUDA(ctx, cudaMemcpyAsync(u_out, u, (size_t)sU * 8, cudaMemcpyDeviceToHost, st));
    }
    if (keep && *keep) {
        (*keep)->var_N = N;
        (*keep)->var_nd.assign(nd, nd + k);
    }
    if (ctx->sync) KS_CUDA(ctx, cudaStreamSynchronize(st));
    return KS_OK;
}

ks_status ks_covariances_var(ks_ctx* ctx, ks_handle h, double* cov_out) {
    if (!ctx) return KS_ERR_ARG;
    ctx->err.clear();
    if (!h || !ctx->facs.count(h)) return fail(ctx, KS_ERR_NO_FACTOR, "unknown or released handle");
    if (h->var_N == 0)
        return fail(ctx, KS_ERR_ARG, "the handle was not made by ks_smooth_var (use ks_covariances)");
    if (!cov_out) return fail(ctx, KS_ERR_ARG, "cov_out must not be NULL");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t k = h->k;
    const int N = h->var_N;
    const std::vector<int32_t>& vnd = h->var_nd;
    std::vector<int64_t> soff(k + 1, 0);
    for (int64_t i = 0; i < k; ++i) soff[i + 1] = soff[i] + (int64_t)vnd[i] * vnd[i];
    Plan plan;
    const size_t o_nd = plan.take(k * sizeof(int32_t));
    const size_t o_soff = plan.take((size_t)(k + 1) * sizeof(int64_t));
    const size_t o_Sp = plan.take((size_t)k * N * N * 8);
    const bool dev = is_device_ptr(cov_out);
    const size_t o_cov = dev ? 0 : plan.take((size_t)soff[k] * 8);
    char* vb = nullptr;
    ks_status rs = var_reserve(ctx, plan.off, &vb);
    if (rs != KS_OK) return rs;
    cudaStream_t st = ctx->stream;
    KS_CUDA(ctx, cudaMemcpyAsync(vb + o_nd, vnd.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    KS_CUDA(ctx, cudaMemcpyAsync(vb + o_soff, soff.data(), (k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    double* Sp = (double*)(vb + o_Sp);
    ks_status s = ks_covariances(ctx, h, Sp, nullptr);
    if (s != KS_OK) return s;
    Phase ph(ctx, KS_PHASE_COPY);
    double* cov = dev ? cov_out : (double*)(vb + o_cov);
    unpad_cov_kernel<<<grid_for(k * N * N, 256), 256, 0, st>>>(k, N, (const int32_t*)(vb + o_nd),
                                                               (const int64_t*)(vb + o_soff), Sp, cov);
    ++t_launches;
    KS_CUDA(ctx, cudaGetLastError());
    if (!dev) KS_CUDA(ctx, cudaMemcpyAsync(cov_out, cov, (size_t)soff[k] * 8, cudaMemcpyDeviceToHost, st));
    if (ctx->sync) KS_CUDA(ctx, cudaStreamSynchronize(st));
    return KS_OK;
}

}  // extern "C"

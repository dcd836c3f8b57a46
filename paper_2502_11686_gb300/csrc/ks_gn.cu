// ks_gn.cu -- ks_gauss_newton: nonlinear smoothing by Levenberg-Marquardt over the states-only
// linear smoother (Section 2: for nonlinear evolution maps f_i and observation maps g_i every
// Gauss-Newton step is a linear smoothing problem whose matrices are the Jacobians at the current
// iterate, possibly concatenated with a diagonal matrix; the covariances are not needed).
//
// One iteration at the iterate u (all on the device; the host only takes the accept / stop
// decisions from three scalars):
//   1. the caller's linearization at u: J_i = df_i(u_i), e_i = f_i(u_i) - u_{i+1},
//      Gj_i = dg_i(u_i), r_i = o_i - g_i(u_i)   (kept from the previous accepted trial);
//   2. damped observations: G'_i = [Gj_i ; I], o'_i = [r_i ; 0], C'_i = diag(C_i, I / lambda)
//      (the Levenberg-Marquardt rows sqrt(lambda) d_i = 0 in whitened form);
//   3. ks_smooth of  d_{i+1} = J_i d_i + e_i (cov K_i),  o'_i = G'_i d_i (cov C'_i)  -> d;
//   4. stop if ||d|| <= xtol (||u|| + xtol);
//   5. trial t = u + d, linearization at t, Phi(t); accept if Phi(t) < Phi(u) (lambda /= 3),
//      else reject (lambda *= 4);
//   6. stop after an accepted step with Phi(u) - Phi(t) <= ftol Phi(t), or lambda > 1e16.
// Phi(u) = sum ||L_K,i^{-1} e_i||^2 + sum ||L_C,i^{-1} r_i||^2 is evaluated in FP64 by one thread
// per step (Cholesky of K_i and C_i in registers), then summed in a fixed order.
#include "ks_host.h"

using namespace kshost;

namespace {

constexpr int GN_NMAX = 16;   // largest n and m of the objective kernel

// Per step: the objective part, ||d_i||^2 and ||u_i||^2 (d and u may be null).
__global__ void gn_parts_kernel(int64_t k, int n, int m, const double* K, const double* C,
                                const double* e, const double* r, const double* d, const double* u,
                                double* parts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        double phi = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            const int dd = pass == 0 ? n : m;
            if (dd == 0 || (pass == 0 && i + 1 >= k)) continue;
            const double* A = pass == 0 ? K + i * (int64_t)n * n : C + i * (int64_t)m * m;
            const double* v = pass == 0 ? e + i * n : r + i * m;
            double L[GN_NMAX * (GN_NMAX + 1) / 2], w[GN_NMAX];
            for (int j = 0; j < dd; ++j) {
                for (int q = 0; q <= j; ++q) {
                    double s = A[j * dd + q];
                    for (int p = 0; p < q; ++p) s -= L[j * (j + 1) / 2 + p] * L[q * (q + 1) / 2 + p];
                    L[j * (j + 1) / 2 + q] = (q == j) ? sqrt(s) : s / L[q * (q + 1) / 2 + q];
                }
            }
            for (int j = 0; j < dd; ++j) {
                double s = v[j];
                for (int p = 0; p < j; ++p) s -= L[j * (j + 1) / 2 + p] * w[p];
                w[j] = s / L[j * (j + 1) / 2 + j];
                phi = fma(w[j], w[j], phi);
            }
        }
        double d2 = 0.0, u2 = 0.0;
        for (int j = 0; j < n; ++j) {
            if (d) d2 = fma(d[i * n + j], d[i * n + j], d2);
            if (u) u2 = fma(u[i * n + j], u[i * n + j], u2);
        }
        parts[i] = phi;
        parts[k + i] = d2;
        parts[2 * k + i] = u2;
    }
}

// Damped observation blocks of step 2 (one thread per entry of the largest array).
__global__ void gn_damp_kernel(int64_t k, int n, int m, double lambda, const double* Gj,
                               const double* r, const double* C, double* Gd, double* od,
                               double* Cd) {
    const int mp = m + n;
    const int64_t per = (int64_t)mp * mp > (int64_t)mp * n ? (int64_t)mp * mp : (int64_t)mp * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * per;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / per;
        const int x = (int)(e - i * per);
        if (x < mp * n) {
            const int row = x / n, col = x - row * n;
            Gd[i * mp * n + x] = row < m ? Gj[(i * m + row) * n + col] : (row - m == col ? 1.0 : 0.0);
        }
        if (x < mp * mp) {
            const int row = x / mp, col = x - row * mp;
            Cd[i * (int64_t)mp * mp + x] = (row < m && col < m) ? C[(i * m + row) * m + col]
                                           : (row == col ? 1.0 / lambda : 0.0);
        }
        if (x < mp) od[i * mp + x] = x < m ? r[i * m + x] : 0.0;
    }
}

__global__ void gn_identity_kernel(int64_t count, int n, double* H) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count * n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % ((int64_t)n * n));
        H[e] = (x / n == x % n) ? 1.0 : 0.0;
    }
}

__global__ void gn_axpy_kernel(int64_t count, const double* u, const double* d, double* t) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        t[e] = u[e] + d[e];
}

// The pendulum's linearization (symplectic Euler step of dt; observation sin(theta)).
__global__ void pendulum_kernel(int64_t k, double dt, double gr, const double* o, const double* u,
                                double* J, double* e, double* Gj, double* r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double th = u[2 * i], w = u[2 * i + 1];
        double sn, cs;
        sincos(th, &sn, &cs);
        if (i + 1 < k) {
            const double w1 = w - gr * sn * dt;
            const double a = gr * cs * dt;
            J[4 * i + 0] = 1.0 - a * dt;
            J[4 * i + 1] = dt;
            J[4 * i + 2] = -a;
            J[4 * i + 3] = 1.0;
            e[2 * i] = th + w1 * dt - u[2 * (i + 1)];
            e[2 * i + 1] = w1 - u[2 * (i + 1) + 1];
        }
        Gj[2 * i] = cs;
        Gj[2 * i + 1] = 0.0;
        r[i] = o[i] - sn;
    }
}

unsigned blocks_for(int64_t work) {
    const int64_t b = (work + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

namespace {
ks_status gn_reserve(ks_ctx* ctx, size_t bytes, char** out) {
    if (bytes > ctx->gbuf_size) {
        KS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->gbuf) cudaFree(ctx->gbuf);
        ctx->gbuf = nullptr;
        ctx->gbuf_size = 0;
        KS_CUDA(ctx, cudaMalloc(&ctx->gbuf, bytes));
        ctx->gbuf_size = bytes;
    }
    *out = (char*)ctx->gbuf;
    return KS_OK;
}
}  // namespace

extern "C" {

void ks_gn_default_options(ks_gn_options* opt) {
    if (!opt) return;
    opt->max_iter = 50;
    opt->lambda0 = 1e-3;
    opt->ftol = 1e-12;
    opt->xtol = 1e-10;
}

int ks_pendulum_linearize(void* user, int64_t k, int n, int m, const double* u, double* J,
                          double* e, double* Gj, double* r, void* stream) {
    const ks_pendulum* p = static_cast<const ks_pendulum*>(user);
    if (!p || n != 2 || m != 1 || !p->o) return 1;
    pendulum_kernel<<<blocks_for(k), 256, 0, (cudaStream_t)stream>>>(k, p->dt, p->gravity, p->o, u,
                                                                    J, e, Gj, r);
    ++t_launches;
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

ks_status ks_gauss_newton(ks_ctx* ctx, int64_t k, int n, int m, ks_linearize_fn fn, void* user,
                          const double* K, const double* C, double* u, const ks_gn_options* opt,
                          ks_gn_report* rep) {
    if (!ctx) return KS_ERR_ARG;
    ctx->err.clear();
    ks_gn_options o;
    ks_gn_default_options(&o);
    if (opt) o = *opt;
    if (k < 2 || n < 1 || n > GN_NMAX || m < 0 || m > GN_NMAX || !fn || !u || !K || (m > 0 && !C))
        return fail(ctx, KS_ERR_ARG, "ks_gauss_newton: need k >= 2, 1 <= n <= %d, 0 <= m <= %d, a "
                    "linearization and device arrays K, C, u", GN_NMAX, GN_NMAX);
    if (!(o.lambda0 > 0.0) || o.max_iter < 1) return fail(ctx, KS_ERR_ARG, "lambda0 must be > 0, max_iter >= 1");
    if (!is_device_ptr(u) || !is_device_ptr(K) || (m > 0 && !is_device_ptr(C)))
        return fail(ctx, KS_ERR_ARG, "ks_gauss_newton: K, C and u must be device arrays");
    KS_CUDA(ctx, cudaSetDevice(ctx->device));
    const int mp = m + n;
    const int64_t nn = (int64_t)n * n;
    Plan plan;
    size_t oJ[2], oe[2], oG[2], orr[2];
    for (int s = 0; s < 2; ++s) {   // linearization at the iterate (s = cur) and at the trial
        oJ[s] = plan.take((size_t)(k - 1) * nn * 8);
        oe[s] = plan.take((size_t)(k - 1) * n * 8);
        oG[s] = plan.take((size_t)k * m * n * 8 + 8);
        orr[s] = plan.take((size_t)k * m * 8 + 8);
    }
    const size_t oH = plan.take((size_t)(k - 1) * nn * 8);
    const size_t oGd = plan.take((size_t)k * mp * n * 8);
    const size_t ood = plan.take((size_t)k * mp * 8);
    const size_t oCd = plan.take((size_t)k * mp * mp * 8);
    const size_t od = plan.take((size_t)k * n * 8);
    const size_t ot = plan.take((size_t)k * n * 8);
    const size_t oparts = plan.take((size_t)3 * k * 8);
    const size_t osums = plan.take(3 * 8);
    char* b = nullptr;
    ks_status rs = gn_reserve(ctx, plan.off, &b);
    if (rs != KS_OK) return rs;
    cudaStream_t st = ctx->stream;
    const int saved_sync = ctx->sync;
    ctx->sync = 1;   // the inner solves report their status before each decision
    struct Restore { ks_ctx* c; int s; ~Restore() { c->sync = s; } } restore{ctx, saved_sync};
    auto P = [&](size_t off) { return (double*)(b + off); };
    int cur = 0;
    std::vector<int32_t> mv(k, mp);
    double sums[3];
    auto linearize = [&](const double* x, int s) -> ks_status {
        if (fn(user, k, n, m, x, P(oJ[s]), P(oe[s]), P(oG[s]), P(orr[s]), (void*)st) != 0)
            return fail(ctx, KS_ERR_ARG, "the linearization callback failed");
        KS_CUDA(ctx, cudaGetLastError());
        return KS_OK;
    };
    auto reduce = [&](int s, const double* d, const double* x) -> ks_status {
        gn_parts_kernel<<<blocks_for(k), 256, 0, st>>>(k, n, m, K, C, P(oe[s]), P(orr[s]), d, x, P(oparts));
        ++t_launches;
        KS_CUDA(ctx, cudaGetLastError());
        for (int j = 0; j < 3; ++j) KS_CUDA(ctx, launch_sum(P(oparts) + j * k, k, P(osums) + j, st));
        KS_CUDA(ctx, cudaMemcpyAsync(sums, P(osums), sizeof sums, cudaMemcpyDeviceToHost, st));
        KS_CUDA(ctx, cudaStreamSynchronize(st));
        return KS_OK;
    };
    gn_identity_kernel<<<blocks_for((k - 1) * nn), 256, 0, st>>>(k - 1, n, P(oH));
    ++t_launches;
    ks_status s = linearize(u, cur);
    if (s != KS_OK) return s;
    if ((s = reduce(cur, nullptr, nullptr)) != KS_OK) return s;
    double phi = sums[0], lam = o.lambda0;
    ks_gn_report R{};
    R.objective0 = phi;
    for (int it = 0; it < o.max_iter; ++it) {
        R.iterations = it + 1;
        gn_damp_kernel<<<blocks_for(k * (int64_t)mp * std::max(mp, n)), 256, 0, st>>>(
            k, n, m, lam, P(oG[cur]), P(orr[cur]), C, P(oGd), P(ood), P(oCd));
        ++t_launches;
        KS_CUDA(ctx, cudaGetLastError());
        int64_t info = -1;
        s = ks_smooth(ctx, k, n, mv.data(), P(oJ[cur]), P(oH), P(oe[cur]), K, P(oGd), P(ood), P(oCd),
                      P(od), nullptr, &info);
        if (s != KS_OK) return s;
        gn_axpy_kernel<<<blocks_for(k * n), 256, 0, st>>>(k * n, u, P(od), P(ot));
        ++t_launches;
        if ((s = linearize(P(ot), cur ^ 1)) != KS_OK) return s;
        if ((s = reduce(cur ^ 1, P(od), u)) != KS_OK) return s;
        const double phi_t = sums[0], dn = sqrt(sums[1]), un = sqrt(sums[2]);
        if (dn <= o.xtol * (un + o.xtol)) {
            R.converged = 1;
            break;
        }
        if (phi_t < phi) {
            const double dec = phi - phi_t;
            KS_CUDA(ctx, cudaMemcpyAsync(u, P(ot), (size_t)k * n * 8, cudaMemcpyDeviceToDevice, st));
            cur ^= 1;
            phi = phi_t;
            lam /= 3.0;
            R.accepted++;
            if (dec <= o.ftol * phi) {
                R.converged = 1;
                break;
            }
        } else {
            lam *= 4.0;
            if (lam > 1e16) break;
        }
    }
    KS_CUDA(ctx, cudaStreamSynchronize(st));
    R.objective = phi;
    R.lambda = lam;
    if (rep) *rep = R;
    return KS_OK;
}

}  // extern "C"

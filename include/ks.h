/*
 * ks.h -- C ABI of the GB300 odd-even Kalman smoother (libks.so).
 *
 * Method: Gargir & Toledo, "Parallel-in-Time Kalman Smoothing Using Orthogonal
 * Transformations" (IPDPS 2025).  The smoother solves the generalized least-squares problem of
 * Section 2 (eq. of the generalized least-squares estimator)
 *
 *     u_hat = argmin_u  sum_i || V_i (H_i u_{i+1} - F_i u_i - c_i) ||^2
 *                     + sum_i || W_i (o_i - G_i u_i) ||^2,     V_i^T V_i = K_i^{-1},
 *                                                               W_i^T W_i = C_i^{-1},
 *
 * by the odd-even block QR factorization of Section 3 (Householder QR of pairs of block rows,
 * even block columns eliminated first, recursion on the odd ones), back substitution through
 * the same recursion (Section 3.1), and the covariances cov(u_hat_i) -- the diagonal blocks of
 * (R^T R)^{-1} -- by the odd-even block SelInv of Section 4 (Algorithm 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - k is the NUMBER OF STATES u_0..u_{k-1} (the paper numbers them 0..k, so its k is ours
 *    minus one).  Evolution equation i (0 <= i < k-1) links u_i to u_{i+1}:
 *    H_i u_{i+1} = F_i u_i + c_i + eps_i, cov(eps_i) = K_i.  It is the paper's equation i+1.
 *  - Observation i: o_i = G_i u_i + delta_i with m_i rows (0 allowed), cov(delta_i) = C_i.
 *    C_i is the paper's L_i.  There is no prior on u_0 (the paper's unknown initial state).
 *  - All matrices are FP64, row-major, step-major:
 *      F, H, K : [k-1][n][n]        c : [k-1][n]  (NULL means c = 0)
 *      G : packed, observation i occupies m_i*n values, in step order
 *      o : packed, sum(m_i) values
 *      C : packed, observation i occupies m_i*m_i values (SPD)
 *      u_out : [k][n]               cov_out : [k][n][n]
 *  - Every array pointer may be a DEVICE pointer (e.g. torch.Tensor.data_ptr() on the ctx's
 *    device) or a HOST pointer (pageable or pinned); the library detects which with
 *    cudaPointerGetAttributes and stages host arrays through its own device buffers on the
 *    ctx's stream.  `m` is always a host array.  The caller keeps ownership of every array.
 *  - Calls are ordered on the ctx's stream.  With ks_options.sync = 1 (the default) every
 *    call returns after its work is complete and reports device-detected errors; with
 *    sync = 0 calls return after enqueueing and ks_sync() reports errors.
 *  - No call throws.  On failure the return value says why, *info (when given) holds the
 *    first failing step / column, and ks_last_error() a message.  Outputs are undefined
 *    unless the call returned KS_OK.
 *  - One ks_ctx must not be used from two host threads at the same time.
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ks_ctx ks_ctx;
typedef struct ks_fac ks_fac;
typedef ks_fac *ks_handle;

typedef enum {
    KS_OK = 0,
    KS_ERR_ARG = 1,        /* bad size, NULL pointer, unsupported n for this precision */
    KS_ERR_NOT_SPD = 2,    /* a K_i or C_i has no Cholesky factor; info = step i */
    KS_ERR_SINGULAR = 3,   /* a diagonal block of R is singular or not finite (the states are
                              not determined by the data); info = state index */
    KS_ERR_OOM = 4,        /* device allocation failed */
    KS_ERR_CUDA = 5,       /* a CUDA runtime call failed; see ks_last_error */
    KS_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up (the tensor-core completion
                              waits of the FP32 large-state kernels, about a second each); the
                              call's outputs are undefined, the ctx stays usable */
    KS_ERR_NO_FACTOR = 7,  /* the handle holds no factorization */
    KS_ERR_NONFINITE = 8   /* ks_smooth: an input value that enters the equations of state i is
                              NaN or infinite (F_i, c_i, G_i, o_i, or H_{i-1}, which multiplies
                              u_i); info = i.  A non-finite K_i or C_i has no Cholesky factor and
                              gives KS_ERR_NOT_SPD instead */
} ks_status;

typedef enum {
    KS_FP64 = 0,         /* every step of the method in FP64 */
    KS_FP32_REFINE = 1   /* FP64 Cholesky factors of K_i, C_i; whitened blocks, Householder QR,
                            back substitution and SelInv in FP32; then one FP64 iterative-
                            refinement step of the states (FP64 residual of the least-squares
                            system, corrected semi-normal equations with the FP32 R) */
} ks_precision;

typedef struct {
    int device;         /* CUDA device ordinal */
    int precision;      /* ks_precision */
    void *stream;       /* cudaStream_t to run on; NULL = a stream owned by the ctx */
    size_t mem_budget;  /* bytes of device work memory the ctx may hold; 0 = no limit */
    int sync;           /* 1 = each call waits for its work and reports device errors */
    int profile;        /* 1 = time every phase with CUDA events on the ctx's stream */
    const char *tune_cache; /* file where ks_smooth_batch keeps its tuned launch shapes (read at
                               the first batch, rewritten after tuning); NULL = keep them in the
                               ctx only.  One line per problem group: its signature, then
                               family * 64 + blocks per SM, family 0 = the default level kernel
                               of that state dimension, 1 = the column-owner kernel */
} ks_options;

/* Phases reported by ks_profile_read (indices of phase_ms / phase_launches). */
typedef enum {
    KS_PHASE_WHITEN = 0,   /* Cholesky factors, whitened blocks, observation pre-reduction */
    KS_PHASE_LEVEL = 1,    /* the odd-even levels of the QR factorization (all levels) */
    KS_PHASE_BACKSUB = 2,  /* base block and back substitution (all levels) */
    KS_PHASE_REFINE = 3,   /* FP64 residual, R^T w = g, R d = w, u += d */
    KS_PHASE_SELINV = 4,   /* odd-even SelInv (all levels) and the lag-one gather */
    KS_PHASE_COPY = 5,     /* staging of host arrays in and out */
    KS_PHASE_BATCH = 6,    /* ks_smooth_batch: the whole launch sequence (one CUDA graph) */
    KS_NPHASES = 7
} ks_phase;

typedef struct {
    uint64_t launches;                  /* kernels this ctx launched */
    uint64_t phase_launches[KS_NPHASES];
    double phase_ms[KS_NPHASES];        /* GPU time per phase (profile = 1 only) */
    uint64_t calls;                     /* ks_smooth + ks_covariances calls */
} ks_profile;

/* Fills *opt with the defaults: device 0, KS_FP64, ctx-owned stream, no budget, sync = 1,
 * profile = 0, tune_cache = NULL. */
void ks_default_options(ks_options *opt);

/* Creates a context.  opt may be NULL (defaults).  Returns KS_OK, KS_ERR_ARG or KS_ERR_CUDA. */
ks_status ks_create(ks_ctx **out, const ks_options *opt);

/*
 * Smoothed states (Section 3: factorization, transformation of the right-hand side and back
 * substitution).  Arrays as in the header comment; u_out receives [k][n] FP64.
 * keep: NULL, or receives a handle that retains the factorization for ks_covariances; the
 *       handle owns device memory until ks_release or ks_destroy.  If *keep already holds a
 *       live handle of this ctx with the same k, n and precision, its memory is reused (no
 *       allocation) and the same handle is returned; any other non-NULL *keep is ignored.
 * info: NULL, or receives the first failing step / state index (-1 if none).
 * n must satisfy 1 <= n <= ks_max_n(ctx) and every m_i <= ks_max_m(ctx, n).
 */
ks_status ks_smooth(ks_ctx *ctx, int64_t k, int n, const int32_t *m,
                    const double *F, const double *H, const double *c, const double *K,
                    const double *G, const double *o, const double *C,
                    double *u_out, ks_handle *keep, int64_t *info);

/*
 * Smoothed states of a problem whose state dimension varies from step to step (Section 2: u_i
 * has n_i entries; evolution equation i has l_i rows, H_i u_{i+1} = F_i u_i + c_i + eps_i with
 * H_i of size l_i x n_{i+1} -- rectangular when the dimension changes -- and F_i of size
 * l_i x n_i; Section 3 allows blocks of any size).
 *   nd [k], l [k-1], m [k]: host int32 arrays of n_i (>= 1), l_i (>= 0), m_i (>= 0).
 *   Packed FP64 row-major arrays in step order: F (l_i*n_i values per equation), H (l_i*n_{i+1}),
 *   c (l_i, or NULL = 0), K (l_i*l_i, SPD), G (m_i*n_i per observation), o (m_i), C (m_i*m_i).
 *   u_out: packed [sum n_i].  keep / info as in ks_smooth (info indexes steps and states).
 * Host or device pointers, as everywhere.  The problem is embedded on the device into a uniform
 * one of dimension N = max(n_i, l_i) (every padding component pinned by a unit observation, so
 * the results are exactly the original problem's) and smoothed by the same kernels; requires
 * N <= ks_max_n(ctx) and m_i + N - n_i <= ks_max_m(ctx, N).  Work grows like N^3 per step.
 */
ks_status ks_smooth_var(ks_ctx *ctx, int64_t k, const int32_t *nd, const int32_t *l,
                        const int32_t *m, const double *F, const double *H, const double *c,
                        const double *K, const double *G, const double *o, const double *C,
                        double *u_out, ks_handle *keep, int64_t *info);

/* Covariances cov(u_hat_i) (n_i x n_i each, packed [sum n_i^2]) of a factorization kept by
 * ks_smooth_var (Section 4, Algorithm 2 on the padded factor; the padding components are
 * uncorrelated with the real ones and are dropped).  KS_ERR_ARG for a handle of ks_smooth. */
ks_status ks_covariances_var(ks_ctx *ctx, ks_handle h, double *cov_out);

/*
 * Nonlinear smoothing (Section 2: with nonlinear evolution maps f_i and observation maps g_i the
 * minimiser is found by a Gauss-Newton-type iteration, each step a LINEAR smoothing problem with
 * the Jacobians at the current iterate, possibly concatenated with a diagonal matrix; only the
 * states of those problems are needed).  Model: u_{i+1} = f_i(u_i) + eps_i (cov K_i, H_i = I),
 * o_i = g_i(u_i) + delta_i (cov C_i, m rows at every step).
 *
 * ks_linearize_fn fills, for the iterate u (device, [k][n]), the device arrays
 *   J [k-1][n][n] = df_i/du (u_i),   e [k-1][n] = f_i(u_i) - u_{i+1},
 *   Gj [k][m][n] = dg_i/du (u_i),    r [k][m]   = o_i - g_i(u_i),
 * with work ordered on `stream` (a cudaStream_t); it returns 0 on success.
 */
typedef int (*ks_linearize_fn)(void *user, int64_t k, int n, int m, const double *u, double *J,
                               double *e, double *Gj, double *r, void *stream);

typedef struct {
    int max_iter;    /* most iterations (default 50) */
    double lambda0;  /* initial Levenberg-Marquardt damping, > 0 (default 1e-3) */
    double ftol;     /* stop after an accepted step that lowers the objective by <= ftol times
                        its value (default 1e-12) */
    double xtol;     /* stop when ||d|| <= xtol (||u|| + xtol) (default 1e-10) */
} ks_gn_options;

typedef struct {
    int iterations, accepted, converged;  /* converged: stopped by ftol or xtol */
    double objective0, objective;         /* Phi at the initial guess and at the result */
    double lambda;                        /* final damping */
} ks_gn_report;

void ks_gn_default_options(ks_gn_options *opt);

/*
 * Levenberg-Marquardt from the initial guess in u (device [k][n]; overwritten by the result).
 * Every iteration: damped observation blocks G'_i = [Gj_i ; I], o'_i = [r_i ; 0],
 * C'_i = diag(C_i, I / lambda); the linear smoother (ks_smooth, the ctx's precision) for the
 * correction d; the trial u + d is accepted if Phi = sum ||L_K,i^{-1} e_i||^2 +
 * sum ||L_C,i^{-1} r_i||^2 decreases (lambda / 3), else rejected (4 lambda).  K [k-1][n][n] and
 * C [k][m][m] are device arrays; 1 <= n <= 16, 0 <= m <= 16, k >= 2.  rep may be NULL.
 * Returns the status of the first failing linear solve or callback, else KS_OK (also when
 * max_iter ran out; see rep->converged).
 */
ks_status ks_gauss_newton(ks_ctx *ctx, int64_t k, int n, int m, ks_linearize_fn fn, void *user,
                          const double *K, const double *C, double *u, const ks_gn_options *opt,
                          ks_gn_report *rep);

/* Built-in model for ks_gauss_newton: a pendulum, u = (theta, w), one symplectic Euler step
 * w' = w - gravity sin(theta) dt, theta' = theta + w' dt; observation sin(theta) (n = 2,
 * m = 1).  `user` points to a ks_pendulum whose o is the device array of the k observations. */
typedef struct {
    double dt, gravity;
    const double *o;
} ks_pendulum;
int ks_pendulum_linearize(void *user, int64_t k, int n, int m, const double *u, double *J,
                          double *e, double *Gj, double *r, void *stream);

/* Bits of ks_problem.time_invariant: the array holds ONE matrix used at every step (a
 * time-invariant model) instead of one per step.  G and C may be time invariant only if every
 * m_i is the same. */
enum { KS_TI_F = 1, KS_TI_H = 2, KS_TI_K = 4, KS_TI_G = 8, KS_TI_C = 16 };

/* One problem of a batch: the arguments of ks_smooth plus its outputs. */
typedef struct {
    int64_t k;
    int n;
    const int32_t *m;                     /* host [k] */
    const double *F, *H, *c, *K, *G, *o, *C;
    double *u_out;                        /* [k][n] */
    double *cov_out;                      /* [k][n][n], or NULL for states only */
    unsigned time_invariant;              /* KS_TI_* bits (0 = every array per step) */
} ks_problem;

/*
 * Smooths nprob independent problems of any lengths and state sizes together (the batched form;
 * the paper treats one problem at a time).  Problems are grouped by state dimension; for every
 * group each recursion level of the odd-even factorization is ONE launch over the tiles of all
 * its problems (persistent thread blocks walking a device work list), and likewise for the
 * whitening, back substitution, refinement and SelInv levels.  The launch sequence is captured
 * once as a CUDA graph per batch shape (state dimensions, deepest level per group, precision,
 * covariances or not) and replayed for later batches of that shape, whatever their lengths;
 * the persistent grid of the heaviest launches is chosen by timing candidates at the first
 * batch of each group (see ks_options.tune_cache).
 * status / info: NULL, or [nprob] per-problem status and first failing index.  Returns KS_OK
 * if every problem succeeded, else the status of the first failing problem.
 */
ks_status ks_smooth_batch(ks_ctx *ctx, int nprob, const ks_problem *probs, int *status,
                          int64_t *info);

/*
 * Synthetic time-invariant problem generated on the device (input generation for tests and
 * serving benchmarks; none of the smoother's arithmetic).  Fills F, H, K (n x n), G (m x n),
 * C (m x m) -- one matrix each, to be passed with time_invariant = all KS_TI_* bits -- and
 * o ([k][m] per step), all device pointers, from a counter-based generator keyed by `seed`:
 * F = f_scale * (product of three random Householder reflections), H = I, K and C = L L^T
 * (L lower triangular, diagonal U[0.5, 1.5], off-diagonal N(0, 0.01)), G ~ N(0, 1/n),
 * o ~ N(0, 1).
 */
ks_status ks_generate(ks_ctx *ctx, int64_t k, int n, int m, uint64_t seed, double f_scale,
                      double *F, double *H, double *K, double *G, double *C, double *o);

/*
 * The same recipe with independent draws for every step (input generation for benchmarks; none of
 * the smoother's arithmetic): F [k-1][n][n] = f_scale * Q (Q as in ks_generate, one draw per
 * problem stored for every step), H [k-1][n][n] = I, and for every step K_i ([k-1][n][n]),
 * C_i ([k][m][m]) = L L^T with their own L, G_i ([k][m][n]) ~ N(0, 1/n), o ([k][m]) ~ N(0, 1).
 * Device pointers; the arrays are per step (time_invariant = 0).
 */
ks_status ks_generate_steps(ks_ctx *ctx, int64_t k, int n, int m, uint64_t seed, double f_scale,
                            double *F, double *H, double *K, double *G, double *C, double *o);

/*
 * Serving loop (continuous batching; the paper has no counterpart).  A server owns a scheduler
 * thread and a stream of the ctx's device.  Requests are admitted in arrival order as device
 * memory (mem_budget) and slots (max_active) allow; every scheduler tick advances each admitted
 * request by one stage of the method (whitening, one recursion level, the base, one level of
 * back substitution, one refinement step, one SelInv level), and the requests at the same kind
 * of stage share ONE launch per state-dimension group even when they are at different recursion
 * depths, so work of requests that arrived at different times overlaps on the device.  A
 * finished request's factor can be kept for later covariance queries.
 */
typedef struct ks_server ks_server;

typedef struct {
    size_t mem_budget;  /* device bytes for requests' work memory; 0 = 3/4 of the free memory */
    int max_active;     /* most admitted requests at a time; 0 = 4096 */
    int keep_factors;   /* 1 = keep every finished request's factor for ks_server_covariances */
} ks_server_options;

typedef struct {
    int done;           /* 1 once the request finished (its outputs are written) */
    int status;         /* ks_status of the request */
    int64_t info;       /* failing index, -1 if none */
    double queue_ms;    /* submission -> admission */
    double latency_ms;  /* submission -> completion */
    int64_t k;
    int n;
} ks_request_info;

typedef struct {
    int64_t submitted, admitted, completed, active, queued;
    int64_t ticks, launches;
    size_t bytes_in_use, bytes_budget;
    int64_t shared_launches;          /* launches that carried the work of two or more requests */
    int64_t max_requests_per_launch;  /* most requests that one launch carried */
} ks_server_counters;

ks_status ks_server_create(ks_ctx *ctx, const ks_server_options *opt, ks_server **out);
/* Enqueues one problem (arrays as in ks_smooth_batch; they must stay valid until the request is
 * done).  Never blocks on the GPU.  *id receives the request id. */
ks_status ks_server_submit(ks_server *srv, const ks_problem *prob, int64_t *id);
/* Enqueues a synthetic problem generated on the device at admission (see ks_generate, f_scale
 * 0.99); its outputs stay in server memory (fetch with ks_server_result). */
ks_status ks_server_submit_synthetic(ks_server *srv, int64_t k, int n, int m, uint64_t seed,
                                     int want_cov, int64_t *id);
/* Covariance follow-up on a finished request whose factor was kept: enqueues the SelInv levels
 * on that factor; cov_out (device or host, [k][n][n]) or NULL (keep them in server memory). */
ks_status ks_server_covariances(ks_server *srv, int64_t id, double *cov_out, int64_t *follow_id);
/* Waits up to timeout_ms (< 0: forever) for request id; fills *out (may be NULL). */
ks_status ks_server_wait(ks_server *srv, int64_t id, double timeout_ms, ks_request_info *out);
/* Copies a finished request's states / covariances kept in server memory (either may be NULL). */
ks_status ks_server_result(ks_server *srv, int64_t id, double *u_out, double *cov_out);
/* Frees a finished request's kept memory (factor, outputs). */
ks_status ks_server_release(ks_server *srv, int64_t id);
ks_status ks_server_stats(ks_server *srv, ks_server_counters *out);
/* Finishes every admitted and queued request, then frees the server. */
ks_status ks_server_destroy(ks_server *srv);

/*
 * Covariances of the smoothed states, cov(u_hat_i) = [(R^T R)^{-1}]_{ii}, by the odd-even
 * block SelInv (Section 4, Algorithm 2) on the factorization held by `h`.
 * cov_out: [k][n][n] FP64 (host or device).  cross_out: NULL, or [k-1][n][n] FP64 receiving
 * the lag-one blocks cov(u_hat_i, u_hat_{i+1}), which Algorithm 2 computes along the way.
 */
ks_status ks_covariances(ks_ctx *ctx, ks_handle h, double *cov_out, double *cross_out);

/* Minimal value of the objective (the squared norm of the rows that the factorization
 * discards), FP64, for the factorization held by `h`.  Written to *out (host). */
ks_status ks_residual(ks_ctx *ctx, ks_handle h, double *out);

/* Frees a handle's device memory.  NULL is a no-op. */
ks_status ks_release(ks_ctx *ctx, ks_handle h);

/* Waits for the ctx's stream and reports the first device-detected error since the last
 * report (for sync = 0). */
ks_status ks_sync(ks_ctx *ctx, int64_t *info);

/* Frees every handle and buffer of the context.  NULL is a no-op. */
ks_status ks_destroy(ks_ctx *ctx);

/* Message of the last failure on ctx (never NULL; "" if none). */
const char *ks_last_error(const ks_ctx *ctx);

/* Counters of the ctx since its creation or the last reset (reset != 0 zeroes them after the
 * read).  Waits for the ctx's stream so that the phase times are complete. */
ks_status ks_profile_read(ks_ctx *ctx, ks_profile *out, int reset);

/* Size of the work array that ks_smooth_static uses instead of allocating (16 MiB). */
#define KS_STATIC_SCRATCH_BYTES (16u << 20)

/*
 * Smoothing for callers that cannot allocate device memory.  (The paper has no counterpart;
 * this is a property of the library, not of the method.)
 *
 * Some callers are not allowed, or cannot afford, to allocate on the device: a plugin inside a
 * host application that owns the whole device-memory budget, or a real-time loop that must
 * never wait on the allocator (cudaMalloc can block, cudaFree synchronizes the device).  This
 * entry point needs no ks_ctx and calls no allocating routine.  The caller passes the inputs and
 * outputs; all other work memory comes from one array of KS_STATIC_SCRATCH_BYTES bytes built
 * into libks.so, which every GPU that loads the library keeps until the process exits.
 *
 * Same arguments and layouts as ks_smooth, restricted to: FP64; 1 <= n <= 8; the same
 * observation count m (0 <= m <= n) at every step; every array a DEVICE pointer of `device`;
 * (k, n, covariances or not) small enough for the array -- otherwise KS_ERR_ARG and a message
 * in err.  cov_out (NULL = states only) receives [k][n][n] covariances.  err / err_len: a
 * caller buffer for the message of a failure (may be NULL).  Runs on `stream` (a
 * cudaStream_t, NULL = the legacy default stream), waits for its work, reports device-detected
 * errors like ks_smooth, and leaves the caller's current device unchanged.
 *
 * The first call on each device looks up that device's address of the built-in array and keeps
 * it; make that first call before any stream capture.  All calls share the one array and each
 * call overwrites what the previous one left there: calls that overlap on the GPU (other
 * streams, other host threads) race, so the caller must serialize them.
 */
ks_status ks_smooth_static(int device, void *stream, int64_t k, int n, int m,
                           const double *F, const double *H, const double *c, const double *K,
                           const double *G, const double *o, const double *C,
                           double *u_out, double *cov_out, int64_t *info,
                           char *err, size_t err_len);

/* Measures the FMA rate of `device` in TFLOP/s (an FMA is two flops): FP64 for KS_FP64, FP32 for
 * KS_FP32_REFINE.  A measurement aid for rooflines (the paper has no counterpart): the
 * arithmetic-bound kernels are compared against this rate.  Runs two short kernels (about 30 ms)
 * on a private stream and allocates 16 bytes.  Returns KS_OK, KS_ERR_ARG or KS_ERR_CUDA. */
ks_status ks_measure_fma_rate(int device, int precision, double *tflops);

/* Largest state dimension n this ctx's precision supports on its device (128 on GB300: up to
 * 48 (FP64) / 64 (FP32) with shared-memory tiles, above that with the large-state kernels, which
 * work on the records in device memory and require every m_i <= n). */
int ks_max_n(const ks_ctx *ctx);

/* Largest per-step observation count m_i supported for state dimension n. */
int ks_max_m(const ks_ctx *ctx, int n);

#ifdef __cplusplus
}
#endif
#endif /* KS_H */

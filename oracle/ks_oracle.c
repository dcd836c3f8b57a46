/*
 * ks_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, sequential FP64 CPU implementation of the linear Kalman smoother of
 * Gargir & Toledo, "Parallel-in-Time Kalman Smoothing Using Orthogonal Transformations"
 * (IPDPS 2025).  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs may load it.  It shares no code, header, helper or constant with the
 * CUDA path, and nothing here is blocked, fused or reordered for speed.
 *
 * What it computes (Section 2, the generalized least-squares form of smoothing):
 *     u_hat = argmin_u  sum_i || V_i (H_i u_{i+1} - F_i u_i - c_i) ||^2
 *                     + sum_i || W_i (o_i - G_i u_i) ||^2 ,
 * with V_i^T V_i = K_i^{-1} and W_i^T W_i = C_i^{-1} (the paper's L_i is our observation
 * covariance C_i), no prior on u_0, and the covariances cov(u_hat_i), the diagonal blocks
 * of (R^T R)^{-1} where U A = Q R (Section 4).
 *
 * Indexing: k states u_0..u_{k-1}; evolution equation i (0 <= i < k-1) links u_i to u_{i+1}
 * (it is the paper's equation i+1); observation i has m_i rows (m_i may be 0).
 *
 * How (the sequential algorithms the paper builds on, not its odd-even method):
 *   1. Whitening (Section 2): V_i is taken as the upper-triangular factor with
 *      V_i^T V_i = K_i^{-1}, obtained from an explicit inverse of K_i.  This is a different
 *      factor from the one the CUDA path uses; the objective does not depend on the choice.
 *   2. Paige-Saunders block QR of U A (Section 2.2 and Section 3): block columns are
 *      eliminated left to right with Householder QR of [carry ; -B_{i+1}], the carry being
 *      the rows that live in column i only.
 *   3. Back substitution, block row by block row, bottom up.
 *   4. Algorithm 1 (block SelInv for (R^T R)^{-1}) with I = {j+1}, which also yields the
 *      lag-one blocks S_{j,j+1} = cov(u_hat_j, u_hat_{j+1}).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_SPD 2
#define ORC_SINGULAR 3
#define ORC_ARG 1
#define ORC_OOM 4

/* Cholesky A = L L^T in place (row-major n x n, lower triangle used).  Returns 0 or j+1. */
static int chol_lower(int n, double *A) {
    for (int j = 0; j < n; j++) {
        double d = A[j * n + j];
        for (int p = 0; p < j; p++) d -= A[j * n + p] * A[j * n + p];
        if (!(d > 0.0)) return j + 1;
        d = sqrt(d);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double s = A[i * n + j];
            for (int p = 0; p < j; p++) s -= A[i * n + p] * A[j * n + p];
            A[i * n + j] = s / d;
        }
        for (int i = 0; i < j; i++) A[i * n + j] = 0.0;
    }
    return 0;
}

/* Inverse of an SPD matrix through its Cholesky factor: A^{-1} = L^{-T} L^{-1}. */
static int inv_spd(int n, const double *A, double *Ainv, double *work /* 2 n*n */) {
    double *L = work, *Li = work + n * n;
    memcpy(L, A, sizeof(double) * n * n);
    int e = chol_lower(n, L);
    if (e) return e;
    /* Li = L^{-1}, lower triangular, by forward substitution on the identity. */
    for (int c = 0; c < n; c++) {
        for (int i = 0; i < n; i++) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int p = 0; p < i; p++) s -= L[i * n + p] * Li[p * n + c];
            Li[i * n + c] = s / L[i * n + i];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int p = 0; p < n; p++) s += Li[p * n + i] * Li[p * n + j];
            Ainv[i * n + j] = s;
        }
    return 0;
}

/* Whitening factor: V upper triangular with V^T V = Cov^{-1}.  Cov^{-1} = Lam Lam^T with Lam
 * lower (its Cholesky factor), so V = Lam^T.  Output V row-major d x d. */
static int whitening_factor(int d, const double *Cov, double *V, double *work /* 3 d*d */) {
    double *Ci = work;
    int e = inv_spd(d, Cov, Ci, work + d * d);
    if (e) return e;
    e = chol_lower(d, Ci);
    if (e) return e;
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) V[i * d + j] = Ci[j * d + i];
    return 0;
}

/* out (r x c) = V (r x r) * X (r x c), all row-major. */
static void matmul_sq(int r, int c, const double *V, const double *X, double *out) {
    for (int i = 0; i < r; i++)
        for (int j = 0; j < c; j++) {
            double s = 0.0;
            for (int p = 0; p < r; p++) s += V[i * r + p] * X[p * c + j];
            out[i * c + j] = s;
        }
}

/* Householder QR of the first nf columns of the rows x cols row-major matrix A, with every
 * reflector also applied to columns nf..cols-1.  Reflector for column j:
 * beta = -sign(alpha) ||x||, sign(0) = +1, H = I - tau v v^T with v_0 = 1; a zero tail gives
 * H = I.  On return the upper triangle of the first min(rows, nf) rows holds R and the
 * entries below the diagonal of the first nf columns are set to zero. */
static void householder(int rows, int cols, int nf, double *A) {
    int steps = nf < rows ? nf : rows;
    for (int j = 0; j < steps; j++) {
        double alpha = A[j * cols + j], sigma = 0.0;
        for (int i = j + 1; i < rows; i++) sigma += A[i * cols + j] * A[i * cols + j];
        if (sigma == 0.0) continue; /* H = I */
        double nrm = sqrt(alpha * alpha + sigma);
        double beta = alpha >= 0.0 ? -nrm : nrm;
        double tau = (beta - alpha) / beta;
        double scale = 1.0 / (alpha - beta);
        for (int i = j + 1; i < rows; i++) A[i * cols + j] *= scale; /* v below the 1 */
        for (int c = j + 1; c < cols; c++) {
            double s = A[j * cols + c];
            for (int i = j + 1; i < rows; i++) s += A[i * cols + j] * A[i * cols + c];
            s *= tau;
            A[j * cols + c] -= s;
            for (int i = j + 1; i < rows; i++) A[i * cols + c] -= s * A[i * cols + j];
        }
        A[j * cols + j] = beta;
        for (int i = j + 1; i < rows; i++) A[i * cols + j] = 0.0;
    }
}

/* Solve R x = b in place (R upper triangular n x n, row-major).  Returns 0 or 1 if singular. */
static int upper_solve_vec(int n, const double *R, double *x) {
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int p = i + 1; p < n; p++) s -= R[i * n + p] * x[p];
        if (R[i * n + i] == 0.0 || !isfinite(R[i * n + i])) return 1;
        x[i] = s / R[i * n + i];
    }
    return 0;
}

/* X = R^{-1} B for B n x c (row-major); R upper triangular. */
static int upper_solve_mat(int n, int c, const double *R, double *X) {
    for (int j = 0; j < c; j++)
        for (int i = n - 1; i >= 0; i--) {
            double s = X[i * c + j];
            for (int p = i + 1; p < n; p++) s -= R[i * n + p] * X[p * c + j];
            if (R[i * n + i] == 0.0 || !isfinite(R[i * n + i])) return 1;
            X[i * c + j] = s / R[i * n + i];
        }
    return 0;
}

/* R^{-1} R^{-T} for upper triangular R. */
static int rinv_rinvt(int n, const double *R, double *out, double *work /* n*n */) {
    double *Ri = work;
    for (int i = 0; i < n * n; i++) Ri[i] = 0.0;
    for (int i = 0; i < n; i++) Ri[i * n + i] = 1.0;
    if (upper_solve_mat(n, n, R, Ri)) return 1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int p = 0; p < n; p++) s += Ri[i * n + p] * Ri[j * n + p];
            out[i * n + j] = s;
        }
    return 0;
}

/* Appends the whitened observation block [W_i G_i | W_i o_i] of step i below the `rows` rows
 * of `carry` (row stride n+1).  Returns 0 or ORC_NOT_SPD. */
static int append_observation(int n, int mi, const double *Gi, const double *oi, const double *Ci,
                              double *carry, int *rows, double *V, double *work, double *tmp) {
    if (mi == 0) return 0;
    if (whitening_factor(mi, Ci, V, work)) return ORC_NOT_SPD;
    for (int r = 0; r < mi; r++) {
        for (int cc = 0; cc < n; cc++) tmp[r * (n + 1) + cc] = Gi[r * n + cc];
        tmp[r * (n + 1) + n] = oi[r];
    }
    matmul_sq(mi, n + 1, V, tmp, carry + (size_t)(*rows) * (n + 1));
    *rows += mi;
    return 0;
}

/* Replaces a carry of more than n rows by its R factor (n rows).  The rhs entries of the
 * dropped rows are the part of the residual that no choice of u can reduce. */
static void compress_carry(int n, double *carry, int *rows, double *res) {
    if (*rows <= n) return;
    householder(*rows, n + 1, n, carry);
    for (int r = n; r < *rows; r++) *res += carry[r * (n + 1) + n] * carry[r * (n + 1) + n];
    *rows = n;
}

/*
 * oracle_smooth: see the file header.  Arrays are row-major FP64:
 *   F, H, K : [k-1][n][n];  c : [k-1][n] or NULL (zero);
 *   G : packed, observation i occupies m_i*n entries in step order;  o : packed sum m_i;
 *   C : packed, observation i occupies m_i*m_i entries.
 * Outputs: u [k][n]; cov [k][n][n] or NULL; cross [k-1][n][n] (cov(u_i, u_{i+1})) or NULL;
 * resid2 (minimal objective value) or NULL; info (failing step / column) or NULL.
 * Returns 0, ORC_NOT_SPD, ORC_SINGULAR, ORC_ARG or ORC_OOM.
 */
int oracle_smooth(int64_t k, int n, const int32_t *m, const double *F, const double *H,
                  const double *c, const double *K, const double *G, const double *o,
                  const double *C, double *u, double *cov, double *cross, double *resid2,
                  int64_t *info) {
    if (k < 1 || n < 1 || !m || !u || (k > 1 && (!F || !H || !K))) return ORC_ARG;
    int mmax = 0;
    for (int64_t i = 0; i < k; i++) {
        if (m[i] < 0) return ORC_ARG;
        if (m[i] > mmax) mmax = m[i];
    }
    if (mmax > 0 && (!G || !o || !C)) return ORC_ARG;
    int d = n > mmax ? n : mmax;
    size_t tmpsz = (size_t)mmax * (n + 1);
    if (tmpsz < (size_t)n * (2 * n + 1)) tmpsz = (size_t)n * (2 * n + 1);
    int cols = 2 * n + 1;
    double *Rdiag = malloc(sizeof(double) * (size_t)k * n * n);
    double *Roff = malloc(sizeof(double) * (size_t)k * n * n); /* R_{i,i+1} */
    double *y = malloc(sizeof(double) * (size_t)k * n);
    double *V = malloc(sizeof(double) * d * d);
    double *work = malloc(sizeof(double) * 4 * d * d);
    double *S = malloc(sizeof(double) * (size_t)(2 * n) * cols);
    double *carry = malloc(sizeof(double) * (size_t)(n + mmax) * (n + 1)); /* [block | rhs] */
    double *tmp = malloc(sizeof(double) * tmpsz);
    double *Snext = malloc(sizeof(double) * n * n), *Scur = malloc(sizeof(double) * n * n);
    double *T = malloc(sizeof(double) * n * n), *Sx = malloc(sizeof(double) * n * n);
    int status = ORC_OK;
    int64_t where = -1;
    double res = 0.0;
    if (!Rdiag || !Roff || !y || !V || !work || !S || !carry || !tmp || !Snext || !Scur || !T || !Sx) {
        status = ORC_OOM;
        goto done;
    }
    int64_t goff = 0, coff = 0; /* packed offsets of observation i in G/o and in C */

    /* Block column 0 starts with the rows of the whitened observation of u_0. */
    int cr = 0;
    if (append_observation(n, m[0], G + goff * n, o + goff, C + coff, carry, &cr, V, work, tmp)) {
        status = ORC_NOT_SPD; where = 0; goto done;
    }
    goff += m[0]; coff += (int64_t)m[0] * m[0];
    compress_carry(n, carry, &cr, &res);

    for (int64_t i = 0; i + 1 < k; i++) {
        /* Whitened evolution equation i: V (H_i u_{i+1} - F_i u_i) = V c_i. */
        if (whitening_factor(n, K + (size_t)i * n * n, V, work)) {
            status = ORC_NOT_SPD; where = i; goto done;
        }
        int rows = cr + n;
        for (int r = 0; r < cr; r++) {
            for (int cc = 0; cc < n; cc++) S[r * cols + cc] = carry[r * (n + 1) + cc];
            for (int cc = 0; cc < n; cc++) S[r * cols + n + cc] = 0.0;
            S[r * cols + 2 * n] = carry[r * (n + 1) + n];
        }
        for (int r = 0; r < n; r++) {
            for (int cc = 0; cc < n; cc++) {
                tmp[r * cols + cc] = -F[(size_t)i * n * n + r * n + cc];
                tmp[r * cols + n + cc] = H[(size_t)i * n * n + r * n + cc];
            }
            tmp[r * cols + 2 * n] = c ? c[(size_t)i * n + r] : 0.0;
        }
        matmul_sq(n, cols, V, tmp, S + (size_t)cr * cols);
        /* QR of [carry ; -B] on block column i, applied to [0 ; D] and the rhs. */
        householder(rows, cols, n, S);
        /* The top n rows are block row i of R: R_ii, R_{i,i+1}, y_i. */
        for (int r = 0; r < n; r++) {
            for (int cc = 0; cc < n; cc++) {
                Rdiag[(size_t)i * n * n + r * n + cc] = S[r * cols + cc];
                Roff[(size_t)i * n * n + r * n + cc] = S[r * cols + n + cc];
            }
            y[(size_t)i * n + r] = S[r * cols + 2 * n];
        }
        /* The remaining rows live in block column i+1 only: they start its carry. */
        int nc = 0;
        for (int r = n; r < rows; r++, nc++) {
            for (int cc = 0; cc < n; cc++) carry[nc * (n + 1) + cc] = S[r * cols + n + cc];
            carry[nc * (n + 1) + n] = S[r * cols + 2 * n];
        }
        int mi = m[i + 1];
        if (append_observation(n, mi, G + goff * n, o + goff, C + coff, carry, &nc, V, work, tmp)) {
            status = ORC_NOT_SPD; where = i + 1; goto done;
        }
        goff += mi; coff += (int64_t)mi * mi;
        compress_carry(n, carry, &nc, &res);
        cr = nc;
    }
    /* Last block column: R_{k-1,k-1} is the R factor of the carry. */
    {
        int64_t i = k - 1;
        if (cr < n) { status = ORC_SINGULAR; where = i; goto done; }
        householder(cr, n + 1, n, carry);
        for (int r = 0; r < n; r++) {
            for (int cc = 0; cc < n; cc++) Rdiag[(size_t)i * n * n + r * n + cc] = carry[r * (n + 1) + cc];
            y[(size_t)i * n + r] = carry[r * (n + 1) + n];
        }
    }

    /* Back substitution: R_ii u_i = y_i - R_{i,i+1} u_{i+1}, bottom block row first. */
    for (int64_t i = k - 1; i >= 0; i--) {
        for (int r = 0; r < n; r++) {
            double s = y[(size_t)i * n + r];
            if (i + 1 < k)
                for (int cc = 0; cc < n; cc++)
                    s -= Roff[(size_t)i * n * n + r * n + cc] * u[(size_t)(i + 1) * n + cc];
            u[(size_t)i * n + r] = s;
        }
        if (upper_solve_vec(n, Rdiag + (size_t)i * n * n, u + (size_t)i * n)) {
            status = ORC_SINGULAR; where = i; goto done;
        }
    }

    /* Algorithm 1 with I = {j+1}:
     *   S_{k-1,k-1} = R^{-1} R^{-T};
     *   T = R_jj^{-1} R_{j,j+1};  S_{j,j+1} = -T S_{j+1,j+1};
     *   S_jj = R_jj^{-1} R_jj^{-T} - S_{j,j+1} T^T.                                       */
    if (cov || cross) {
        int64_t j = k - 1;
        if (rinv_rinvt(n, Rdiag + (size_t)j * n * n, Snext, work)) {
            status = ORC_SINGULAR; where = j; goto done;
        }
        if (cov) memcpy(cov + (size_t)j * n * n, Snext, sizeof(double) * n * n);
        for (j = k - 2; j >= 0; j--) {
            memcpy(T, Roff + (size_t)j * n * n, sizeof(double) * n * n);
            if (upper_solve_mat(n, n, Rdiag + (size_t)j * n * n, T)) {
                status = ORC_SINGULAR; where = j; goto done;
            }
            for (int r = 0; r < n; r++)
                for (int cc = 0; cc < n; cc++) {
                    double s = 0.0;
                    for (int p = 0; p < n; p++) s += T[r * n + p] * Snext[p * n + cc];
                    Sx[r * n + cc] = -s;
                }
            rinv_rinvt(n, Rdiag + (size_t)j * n * n, Scur, work);
            for (int r = 0; r < n; r++)
                for (int cc = 0; cc < n; cc++) {
                    double s = 0.0;
                    for (int p = 0; p < n; p++) s += Sx[r * n + p] * T[cc * n + p];
                    Scur[r * n + cc] -= s;
                }
            if (cov) memcpy(cov + (size_t)j * n * n, Scur, sizeof(double) * n * n);
            if (cross) memcpy(cross + (size_t)j * n * n, Sx, sizeof(double) * n * n);
            memcpy(Snext, Scur, sizeof(double) * n * n);
        }
    }
done:
    if (resid2) *resid2 = res;
    if (info) *info = where;
    free(Rdiag); free(Roff); free(y); free(V); free(work); free(S); free(carry); free(tmp);
    free(Snext); free(Scur); free(T); free(Sx);
    return status;
}

/*
 * oracle_smooth_var: the same smoother when the state dimension varies from step to step and
 * H_i is rectangular (Section 2: u_i has n_i entries; evolution equation i has l_i rows, with
 * H_i of size l_i x n_{i+1} and F_i of size l_i x n_i; "the dimensions of block rows and block
 * columns can vary", Section 3).  Written directly for ragged blocks -- no padding -- as the
 * same left-to-right Paige-Saunders elimination, back substitution and Algorithm 1 (I = {j+1})
 * as oracle_smooth.
 *
 * Packed row-major FP64 inputs, in step order:
 *   nd [k] state dimensions; l [k-1] evolution rows; m [k] observation rows (host int32);
 *   F : evolution i occupies l_i*n_i values;  H : l_i*n_{i+1};  c : l_i (or NULL = 0);
 *   K : l_i*l_i;  G : m_i*n_i;  o : m_i;  C : m_i*m_i.
 * Outputs: u packed sum n_i; cov packed sum n_i^2 (or NULL); resid2; info.
 */
int oracle_smooth_var(int64_t k, const int32_t *nd, const int32_t *l, const int32_t *m,
                      const double *F, const double *H, const double *c, const double *K,
                      const double *G, const double *o, const double *C, double *u, double *cov,
                      double *resid2, int64_t *info) {
    if (k < 1 || !nd || !m || !u || (k > 1 && (!l || !F || !H || !K))) return ORC_ARG;
    int nmax = 0, lmax = 0, mmax = 0;
    for (int64_t i = 0; i < k; i++) {
        if (nd[i] < 1 || m[i] < 0) return ORC_ARG;
        if (nd[i] > nmax) nmax = nd[i];
        if (m[i] > mmax) mmax = m[i];
        if (i + 1 < k) {
            if (l[i] < 0) return ORC_ARG;
            if (l[i] > lmax) lmax = l[i];
        }
    }
    if (mmax > 0 && (!G || !o || !C)) return ORC_ARG;
    /* Offsets of every block in the packed arrays and in the outputs. */
    int64_t *uo = malloc(sizeof(int64_t) * (size_t)(k + 1));   /* u, and R rows */
    int64_t *so = malloc(sizeof(int64_t) * (size_t)(k + 1));   /* n_i^2 blocks */
    int64_t *ro = malloc(sizeof(int64_t) * (size_t)(k + 1));   /* R_{i,i+1}: n_i x n_{i+1} */
    int d = nmax > lmax ? nmax : lmax;
    if (mmax > d) d = mmax;
    int cw = 2 * nmax + 1;                         /* widest [col i | col i+1 | rhs] */
    int maxrows = nmax + mmax + lmax + 1;
    double *Rdiag = NULL, *Roff = NULL, *y = NULL;
    double *V = malloc(sizeof(double) * d * d);
    double *work = malloc(sizeof(double) * 4 * d * d);
    double *S = malloc(sizeof(double) * (size_t)maxrows * cw);
    double *carry = malloc(sizeof(double) * (size_t)maxrows * (nmax + 1));
    double *tmp = malloc(sizeof(double) * (size_t)(d + 1) * cw);
    double *Snext = malloc(sizeof(double) * nmax * nmax), *Scur = malloc(sizeof(double) * nmax * nmax);
    double *T = malloc(sizeof(double) * nmax * nmax), *Sx = malloc(sizeof(double) * nmax * nmax);
    int status = ORC_OK;
    int64_t where = -1;
    double res = 0.0;
    if (!uo || !so || !ro || !V || !work || !S || !carry || !tmp || !Snext || !Scur || !T || !Sx) {
        status = ORC_OOM;
        goto done;
    }
    uo[0] = so[0] = ro[0] = 0;
    for (int64_t i = 0; i < k; i++) {
        uo[i + 1] = uo[i] + nd[i];
        so[i + 1] = so[i] + (int64_t)nd[i] * nd[i];
        ro[i + 1] = ro[i] + (i + 1 < k ? (int64_t)nd[i] * nd[i + 1] : 0);
    }
    Rdiag = malloc(sizeof(double) * (size_t)so[k]);
    Roff = malloc(sizeof(double) * (size_t)(ro[k] > 0 ? ro[k] : 1));
    y = malloc(sizeof(double) * (size_t)uo[k]);
    if (!Rdiag || !Roff || !y) { status = ORC_OOM; goto done; }

    int64_t go = 0, gv = 0, co = 0;   /* offsets of observation i: rows (o), values (G), C */
    int64_t fo = 0, ho = 0, eo = 0, ko = 0;   /* offsets of evolution i in F, H, c, K */
    /* Column 0 starts with the whitened observation of u_0 (n_0 + 1 wide: block | rhs). */
    int n0 = nd[0], cr = 0;
    if (append_observation(n0, m[0], G + gv, o + go, C + co, carry, &cr, V, work, tmp)) {
        status = ORC_NOT_SPD; where = 0; goto done;
    }
    go += m[0]; gv += (int64_t)m[0] * n0; co += (int64_t)m[0] * m[0];
    compress_carry(n0, carry, &cr, &res);

    for (int64_t i = 0; i + 1 < k; i++) {
        const int ni = nd[i], nj = nd[i + 1], li = l[i];
        const int w = ni + nj + 1;   /* [col i | col i+1 | rhs] */
        const int rows = cr + li;
        for (int r = 0; r < cr; r++) {
            for (int q = 0; q < ni; q++) S[r * w + q] = carry[r * (ni + 1) + q];
            for (int q = 0; q < nj; q++) S[r * w + ni + q] = 0.0;
            S[r * w + ni + nj] = carry[r * (ni + 1) + ni];
        }
        if (li > 0) {
            if (whitening_factor(li, K + ko, V, work)) { status = ORC_NOT_SPD; where = i; goto done; }
            /* Whitened evolution equation i: V (H_i u_{i+1} - F_i u_i) = V c_i. */
            for (int r = 0; r < li; r++) {
                for (int q = 0; q < ni; q++) tmp[r * w + q] = -F[fo + (int64_t)r * ni + q];
                for (int q = 0; q < nj; q++) tmp[r * w + ni + q] = H[ho + (int64_t)r * nj + q];
                tmp[r * w + ni + nj] = c ? c[eo + r] : 0.0;
            }
            matmul_sq(li, w, V, tmp, S + (size_t)cr * w);
        }
        fo += (int64_t)li * ni; ho += (int64_t)li * nj; eo += li; ko += (int64_t)li * li;
        if (rows < ni) { status = ORC_SINGULAR; where = i; goto done; }
        householder(rows, w, ni, S);
        for (int r = 0; r < ni; r++) {
            for (int q = 0; q < ni; q++) Rdiag[so[i] + (int64_t)r * ni + q] = S[r * w + q];
            for (int q = 0; q < nj; q++) Roff[ro[i] + (int64_t)r * nj + q] = S[r * w + ni + q];
            y[uo[i] + r] = S[r * w + ni + nj];
        }
        /* Rows below the first n_i live in column i+1 only: they start its carry. */
        int nc = 0;
        for (int r = ni; r < rows; r++, nc++) {
            for (int q = 0; q < nj; q++) carry[nc * (nj + 1) + q] = S[r * w + ni + q];
            carry[nc * (nj + 1) + nj] = S[r * w + ni + nj];
        }
        const int mi = m[i + 1];
        if (append_observation(nj, mi, G + gv, o + go, C + co, carry, &nc, V, work, tmp)) {
            status = ORC_NOT_SPD; where = i + 1; goto done;
        }
        go += mi; gv += (int64_t)mi * nj; co += (int64_t)mi * mi;
        compress_carry(nj, carry, &nc, &res);
        cr = nc;
    }
    {
        const int64_t i = k - 1;
        const int ni = nd[i];
        if (cr < ni) { status = ORC_SINGULAR; where = i; goto done; }
        householder(cr, ni + 1, ni, carry);
        for (int r = 0; r < ni; r++) {
            for (int q = 0; q < ni; q++) Rdiag[so[i] + (int64_t)r * ni + q] = carry[r * (ni + 1) + q];
            y[uo[i] + r] = carry[r * (ni + 1) + ni];
        }
    }
    /* Back substitution: R_ii u_i = y_i - R_{i,i+1} u_{i+1}. */
    for (int64_t i = k - 1; i >= 0; i--) {
        const int ni = nd[i];
        for (int r = 0; r < ni; r++) {
            double s = y[uo[i] + r];
            if (i + 1 < k)
                for (int q = 0; q < nd[i + 1]; q++)
                    s -= Roff[ro[i] + (int64_t)r * nd[i + 1] + q] * u[uo[i + 1] + q];
            u[uo[i] + r] = s;
        }
        if (upper_solve_vec(ni, Rdiag + so[i], u + uo[i])) { status = ORC_SINGULAR; where = i; goto done; }
    }
    /* Algorithm 1 with I = {j+1} on ragged blocks: T = R_jj^{-1} R_{j,j+1} (n_j x n_{j+1}),
     * S_{j,j+1} = -T S_{j+1,j+1}, S_jj = R_jj^{-1} R_jj^{-T} - S_{j,j+1} T^T. */
    if (cov) {
        int64_t j = k - 1;
        int nb = nd[j];
        if (rinv_rinvt(nb, Rdiag + so[j], Snext, work)) { status = ORC_SINGULAR; where = j; goto done; }
        memcpy(cov + so[j], Snext, sizeof(double) * nb * nb);
        for (j = k - 2; j >= 0; j--) {
            const int na = nd[j];
            memcpy(T, Roff + ro[j], sizeof(double) * na * nb);
            if (upper_solve_mat(na, nb, Rdiag + so[j], T)) { status = ORC_SINGULAR; where = j; goto done; }
            for (int r = 0; r < na; r++)
                for (int q = 0; q < nb; q++) {
                    double s = 0.0;
                    for (int p = 0; p < nb; p++) s += T[r * nb + p] * Snext[p * nb + q];
                    Sx[r * nb + q] = -s;
                }
            rinv_rinvt(na, Rdiag + so[j], Scur, work);
            for (int r = 0; r < na; r++)
                for (int q = 0; q < na; q++) {
                    double s = 0.0;
                    for (int p = 0; p < nb; p++) s += Sx[r * nb + p] * T[q * nb + p];
                    Scur[r * na + q] -= s;
                }
            memcpy(cov + so[j], Scur, sizeof(double) * na * na);
            memcpy(Snext, Scur, sizeof(double) * na * na);
            nb = na;
        }
    }
done:
    if (resid2) *resid2 = res;
    if (info) *info = where;
    free(uo); free(so); free(ro); free(Rdiag); free(Roff); free(y); free(V); free(work); free(S);
    free(carry); free(tmp); free(Snext); free(Scur); free(T); free(Sx);
    return status;
}

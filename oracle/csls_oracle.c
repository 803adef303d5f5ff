/*
 * csls_oracle.c -- plain, slow, obviously correct CPU reference for the
 * count-sketch preconditioned LSQR method (CSQRP-LSQR / CSSVDP-LSQR).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link or call this
 * file; it exists so the CUDA path can be checked against an independent
 * implementation. It shares no code, header or table with the CUDA library.
 *
 * Everything is scalar IEEE binary64 (binary32 only where a function says so),
 * compiled with -O2 -ffp-contract=off so no fused multiply-add changes rounding.
 * Matrices are column-major with an explicit leading dimension.
 *
 * Threads: the one OpenMP loop is the Householder QR's loop over trailing
 * columns. Each column's dot product and update are computed by one thread in
 * the same order as the serial loop, so the result is bit-identical for any
 * thread count (tested); threads only let the bench-size factorisations finish
 * on a multi-core host.
 *
 * Parity status: every function here is pinned by a CPU test (worked example,
 * closed form, library special case, brute force or invariant); none is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of threads of the QR's column loop (no effect in a build without OpenMP);
 * returns the count in force. */
int orc_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Count-sketch hash (Definition 2.3). The paper only asks that h(i) be uniform
 * on [s] and d(i) = +-1 with equal probability, independently per row. This
 * reading draws both from the SplitMix64 sequence seeded with `seed`
 * (Steele, Lea and Flood 2014): output i is mix(seed + (i+1) * 0x9E3779B97F4A7C15).
 * The bucket is Lemire's multiply-shift of the high 32 bits, the sign the low bit. */
uint64_t orc_splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_output(uint64_t seed, uint64_t i) {
    return orc_splitmix64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

void orc_hash(int64_t m, int64_t s, uint64_t seed, int32_t* h, int8_t* d) {
    for (int64_t i = 0; i < m; ++i) {
        uint64_t z = orc_splitmix64_output(seed, (uint64_t)i);
        uint64_t hi = z >> 32;
        h[i] = (int32_t)((hi * (uint64_t)s) >> 32);
        d[i] = (z & 1ULL) ? (int8_t)-1 : (int8_t)1;
    }
}

/* ------------------------------------------------------------------------ */
/* Sketched matrix SA = Phi D A (Definition 2.3, Algorithm 1 step 2): row i of A,
 * times d(i), is added to row h(i) of SA. S is never formed. Rows are visited in
 * ascending i, so each entry of SA is the sum of its contributions in ascending
 * row order, starting from +0.0. SA is s x n column-major with leading dim ld. */
void orc_sketch(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                const double* val, int64_t s, const int32_t* h, const int8_t* d,
                double* SA, int64_t ld) {
    for (int64_t j = 0; j < n; ++j)
        for (int64_t k = 0; k < s; ++k) SA[k + j * ld] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t k = h[i];
        double sign = (double)d[i];
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            SA[k + (int64_t)col[p] * ld] += sign * val[p];
    }
}

/* Binary32 sketch: each value is rounded to binary32 first and the sums are
 * binary32, in the same ascending-row order. */
void orc_sketch_f32(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                    const double* val, int64_t s, const int32_t* h, const int8_t* d,
                    float* SA, int64_t ld) {
    for (int64_t j = 0; j < n; ++j)
        for (int64_t k = 0; k < s; ++k) SA[k + j * ld] = 0.0f;
    for (int64_t i = 0; i < m; ++i) {
        int64_t k = h[i];
        float sign = (float)d[i];
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            SA[k + (int64_t)col[p] * ld] += sign * (float)val[p];
    }
}

/* ------------------------------------------------------------------------ */
/* Householder QR (Algorithm 1 step 3), unblocked, column by column as in
 * Golub and Van Loan's Householder QR: for column j the reflector
 * H_j = I - tau_j v_j v_j^T with v_j(0) = 1 maps A(j:s, j) onto beta_j e_1,
 * beta_j = -sign(alpha) ||A(j:s, j)||, and is applied to A(j:s, j+1:n).
 * On exit the upper triangle holds R and the strict lower part the v_j tails.
 * A column that is already zero below the diagonal gets tau_j = 0. */
void orc_householder_qr(int64_t s, int64_t n, double* A, int64_t lda, double* tau) {
    int64_t kmax = s < n ? s : n;
    for (int64_t j = 0; j < kmax; ++j) {
        double* x = A + j + j * lda;
        int64_t len = s - j;
        double alpha = x[0];
        double sigma = 0.0;
        for (int64_t i = 1; i < len; ++i) sigma += x[i] * x[i];
        if (sigma == 0.0) { tau[j] = 0.0; continue; }
        double norm = sqrt(alpha * alpha + sigma);
        double beta = alpha >= 0.0 ? -norm : norm;
        tau[j] = (beta - alpha) / beta;
        double scal = 1.0 / (alpha - beta);
        for (int64_t i = 1; i < len; ++i) x[i] *= scal;
        x[0] = beta;
        /* columns are independent: one thread per column, same arithmetic as serially */
#pragma omp parallel for schedule(static) if ((n - j) * len > 262144)
        for (int64_t c = j + 1; c < n; ++c) {
            double* y = A + j + c * lda;
            double w = y[0];
            for (int64_t i = 1; i < len; ++i) w += x[i] * y[i];
            w *= tau[j];
            y[0] -= w;
            for (int64_t i = 1; i < len; ++i) y[i] -= w * x[i];
        }
    }
}

void orc_householder_qr_f32(int64_t s, int64_t n, float* A, int64_t lda, float* tau) {
    int64_t kmax = s < n ? s : n;
    for (int64_t j = 0; j < kmax; ++j) {
        float* x = A + j + j * lda;
        int64_t len = s - j;
        float alpha = x[0];
        float sigma = 0.0f;
        for (int64_t i = 1; i < len; ++i) sigma += x[i] * x[i];
        if (sigma == 0.0f) { tau[j] = 0.0f; continue; }
        float norm = sqrtf(alpha * alpha + sigma);
        float beta = alpha >= 0.0f ? -norm : norm;
        tau[j] = (beta - alpha) / beta;
        float scal = 1.0f / (alpha - beta);
        for (int64_t i = 1; i < len; ++i) x[i] *= scal;
        x[0] = beta;
        for (int64_t c = j + 1; c < n; ++c) {
            float* y = A + j + c * lda;
            float w = y[0];
            for (int64_t i = 1; i < len; ++i) w += x[i] * y[i];
            w *= tau[j];
            y[0] -= w;
            for (int64_t i = 1; i < len; ++i) y[i] -= w * x[i];
        }
    }
}

/* Copy the n x n upper triangle of a factored matrix into R (zero below the
 * diagonal) and flip the sign of every row whose diagonal is negative, so that
 * R has a non-negative diagonal (the R factor is unique up to row signs). */
void orc_extract_r(int64_t n, const double* QR, int64_t lda, double* R, int64_t ldr) {
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = (i <= j) ? QR[i + j * lda] : 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (R[i + i * ldr] < 0.0)
            for (int64_t j = i; j < n; ++j) R[i + j * ldr] = -R[i + j * ldr];
}

/* ------------------------------------------------------------------------ */
/* Triangular solves with the n x n upper-triangular R (Algorithm 1 steps 4 and
 * 6 applied to a vector): back substitution for R z = v, forward substitution
 * for R^T z = v. Both overwrite x. */
void orc_trsv_upper(int64_t n, const double* R, int64_t ldr, double* x) {
    for (int64_t i = n - 1; i >= 0; --i) {
        double acc = x[i];
        for (int64_t j = i + 1; j < n; ++j) acc -= R[i + j * ldr] * x[j];
        x[i] = acc / R[i + i * ldr];
    }
}

void orc_trsv_upper_trans(int64_t n, const double* R, int64_t ldr, double* x) {
    for (int64_t i = 0; i < n; ++i) {
        double acc = x[i];
        for (int64_t j = 0; j < i; ++j) acc -= R[j + i * ldr] * x[j];
        x[i] = acc / R[i + i * ldr];
    }
}

/* y = A x and y = A^T x for CSR A. */
void orc_spmv(int64_t m, const int64_t* row_ptr, const int32_t* col, const double* val,
              const double* x, double* y) {
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) acc += val[p] * x[col[p]];
        y[i] = acc;
    }
}

void orc_spmv_trans(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                    const double* val, const double* x, double* y) {
    for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) y[col[p]] += val[p] * x[i];
}

/* ------------------------------------------------------------------------ */
/* The right preconditioner M of the implicit form (the Remark after
 * Algorithm 2): M = R^{-1} for the QR variant, M = P = V Sigma^{-1} (n x r) for
 * the SVD variant. apply: z = M y; apply_t: y = M^T g. */
typedef struct {
    int kind;          /* 0: R^{-1}; 1: P */
    int64_t n, r;
    const double* F;   /* R (n x n, ld) or P (n x r, ld) */
    int64_t ld;
} orc_prec;

static void prec_apply(const orc_prec* M, const double* y, double* z) {
    if (M->kind == 0) {
        memcpy(z, y, sizeof(double) * (size_t)M->n);
        orc_trsv_upper(M->n, M->F, M->ld, z);
    } else {
        for (int64_t i = 0; i < M->n; ++i) {
            double acc = 0.0;
            for (int64_t k = 0; k < M->r; ++k) acc += M->F[i + k * M->ld] * y[k];
            z[i] = acc;
        }
    }
}

static void prec_apply_t(const orc_prec* M, const double* g, double* y) {
    if (M->kind == 0) {
        memcpy(y, g, sizeof(double) * (size_t)M->n);
        orc_trsv_upper_trans(M->n, M->F, M->ld, y);
    } else {
        for (int64_t k = 0; k < M->r; ++k) {
            double acc = 0.0;
            for (int64_t i = 0; i < M->n; ++i) acc += M->F[i + k * M->ld] * g[i];
            y[k] = acc;
        }
    }
}

static double nrm2(int64_t n, const double* x) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += x[i] * x[i];
    return sqrt(acc);
}

/* LSQR (Paige and Saunders, ACM TOMS 8(1), 1982), the Krylov solver of
 * Algorithm 1 step 5, run on B = A M with y^(0) = 0 (Section 4.1), followed by
 * x = M y (Algorithm 1 step 6). Stopping: if fixed_iters > 0 exactly that many
 * iterations run with no test; otherwise Paige and Saunders' rules
 *   S1: ||r|| <= btol ||b|| + atol ||B|| ||y||
 *   S2: ||B^T r|| <= atol ||B|| ||r||
 * with ||B|| the running Frobenius estimate, or maxit iterations.
 * out[0..5] = iterations, istop (0 maxit/fixed, 1 S1, 2 S2, 3 exact zero
 * alpha or beta), ||r|| estimate, ||B^T r|| estimate, ||B|| estimate, ||y||.
 * rhist (may be NULL) receives ||r_k|| estimates for k = 0..iterations. */
/* x0 (n, may be NULL): initial guess. LSQR then runs on the residual r0 = b - A x0
 * (the preconditioned correction starts at y = 0) and returns x = x0 + M y; the
 * stopping rule S1 keeps ||b|| of the original right-hand side, as LSQR with an
 * initial point does (Remark 3.1 uses x0 = R^-1 Q^T S b). */
void orc_lsqr(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
              const double* val, const double* b, int prec_kind, const double* F,
              int64_t ldf, int64_t r, double atol, double btol, int64_t maxit,
              int64_t fixed_iters, const double* x0, double* x, double* out, double* rhist) {
    orc_prec M = {prec_kind, n, prec_kind == 0 ? n : r, F, ldf};
    int64_t nr = M.r;
    double* u = (double*)calloc((size_t)m, sizeof(double));
    double* v = (double*)calloc((size_t)nr, sizeof(double));
    double* w = (double*)calloc((size_t)nr, sizeof(double));
    double* y = (double*)calloc((size_t)nr, sizeof(double));
    double* z = (double*)calloc((size_t)n, sizeof(double));
    double* g = (double*)calloc((size_t)n, sizeof(double));
    double* t = (double*)calloc((size_t)m, sizeof(double));

    /* beta_1 u_1 = b - A x0, alpha_1 v_1 = B^T u_1 */
    memcpy(u, b, sizeof(double) * (size_t)m);
    double bnorm = nrm2(m, u);
    if (x0) {
        orc_spmv(m, row_ptr, col, val, x0, t);
        for (int64_t i = 0; i < m; ++i) u[i] -= t[i];
    }
    double beta = nrm2(m, u);
    int64_t it = 0;
    int istop = 0;
    double alpha = 0.0, rnorm = beta, arnorm = 0.0, anorm2 = 0.0, ynorm = 0.0;
    if (rhist) rhist[0] = beta;
    if (beta > 0.0) {
        for (int64_t i = 0; i < m; ++i) u[i] /= beta;
        orc_spmv_trans(m, n, row_ptr, col, val, u, g);
        prec_apply_t(&M, g, v);
        alpha = nrm2(nr, v);
    }
    if (beta == 0.0 || alpha == 0.0) {
        istop = 3;
    } else {
        for (int64_t k = 0; k < nr; ++k) { v[k] /= alpha; w[k] = v[k]; }
        double phibar = beta, rhobar = alpha;
        int64_t limit = fixed_iters > 0 ? fixed_iters : maxit;
        while (it < limit) {
            ++it;
            /* beta_{i+1} u_{i+1} = B v_i - alpha_i u_i */
            prec_apply(&M, v, z);
            orc_spmv(m, row_ptr, col, val, z, t);
            for (int64_t i = 0; i < m; ++i) u[i] = t[i] - alpha * u[i];
            beta = nrm2(m, u);
            anorm2 += alpha * alpha + beta * beta;
            if (beta > 0.0) {
                for (int64_t i = 0; i < m; ++i) u[i] /= beta;
                /* alpha_{i+1} v_{i+1} = B^T u_{i+1} - beta_{i+1} v_i */
                orc_spmv_trans(m, n, row_ptr, col, val, u, g);
                double* bt = (double*)malloc(sizeof(double) * (size_t)nr);
                prec_apply_t(&M, g, bt);
                for (int64_t k = 0; k < nr; ++k) v[k] = bt[k] - beta * v[k];
                free(bt);
                alpha = nrm2(nr, v);
                if (alpha > 0.0)
                    for (int64_t k = 0; k < nr; ++k) v[k] /= alpha;
            } else {
                alpha = 0.0;
            }
            /* plane rotation eliminating beta_{i+1} */
            double rho = sqrt(rhobar * rhobar + beta * beta);
            double c = rhobar / rho, sn = beta / rho;
            double theta = sn * alpha;
            rhobar = -c * alpha;
            double phi = c * phibar;
            phibar = sn * phibar;
            /* y_i = y_{i-1} + (phi/rho) w_i ; w_{i+1} = v_{i+1} - (theta/rho) w_i */
            for (int64_t k = 0; k < nr; ++k) {
                y[k] += (phi / rho) * w[k];
                w[k] = v[k] - (theta / rho) * w[k];
            }
            rnorm = phibar;
            arnorm = phibar * alpha * fabs(c);
            ynorm = nrm2(nr, y);
            if (rhist) rhist[it] = rnorm;
            if (fixed_iters > 0) continue;
            if (beta == 0.0 || alpha == 0.0) { istop = 3; break; }
            double anorm = sqrt(anorm2);
            if (rnorm <= btol * bnorm + atol * anorm * ynorm) { istop = 1; break; }
            if (arnorm <= atol * anorm * rnorm) { istop = 2; break; }
        }
    }
    prec_apply(&M, y, x);
    if (x0)
        for (int64_t k = 0; k < n; ++k) x[k] += x0[k];
    out[0] = (double)it; out[1] = (double)istop; out[2] = rnorm; out[3] = arnorm;
    out[4] = sqrt(anorm2); out[5] = ynorm;
    free(u); free(v); free(w); free(y); free(z); free(g); free(t);
}

/* ------------------------------------------------------------------------ */
/* Dense Householder least-squares solve (the HHQR direct method of Section
 * 4.1): QR of a copy of the m x n dense A, c = Q^T b, back substitution on the
 * leading n rows. Used as the independent reference x_* = argmin ||Ax - b||.
 * R_out (n x n, may be NULL) receives the sign-normalised R of A. */
void orc_hhqr_solve(int64_t m, int64_t n, const double* A, int64_t lda, const double* b,
                    double* x, double* R_out) {
    double* Q = (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* tau = (double*)malloc(sizeof(double) * (size_t)n);
    double* c = (double*)malloc(sizeof(double) * (size_t)m);
    for (int64_t j = 0; j < n; ++j) memcpy(Q + j * m, A + j * lda, sizeof(double) * (size_t)m);
    memcpy(c, b, sizeof(double) * (size_t)m);
    orc_householder_qr(m, n, Q, m, tau);
    for (int64_t j = 0; j < n; ++j) {
        double w = c[j];
        for (int64_t i = j + 1; i < m; ++i) w += Q[i + j * m] * c[i];
        w *= tau[j];
        c[j] -= w;
        for (int64_t i = j + 1; i < m; ++i) c[i] -= w * Q[i + j * m];
    }
    /* R x = c(0:n) with R the upper triangle of Q (signs as factored) */
    for (int64_t i = n - 1; i >= 0; --i) {
        double acc = c[i];
        for (int64_t j = i + 1; j < n; ++j) acc -= Q[i + j * m] * x[j];
        x[i] = acc / Q[i + i * m];
    }
    if (R_out) orc_extract_r(n, Q, m, R_out, n);
    free(Q); free(tau); free(c);
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes; Demmel and Veselic 1992) of the n x n R,
 * the factor of Algorithm 2 step 3: since SA = QR, SA and R share Sigma and V.
 * Column pairs of G = R are rotated until mutually orthogonal; V accumulates the
 * rotations; sigma_j = ||G_j||. Output sorted by decreasing sigma.
 * Returns the number of sweeps used. */
int orc_jacobi_svd(int64_t n, const double* R, int64_t ldr, double* sigma, double* V, int64_t ldv,
                   int max_sweeps) {
    double* G = (double*)malloc(sizeof(double) * (size_t)(n * n));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) G[i + j * n] = R[i + j * ldr];
    double* W = (double*)calloc((size_t)(n * n), sizeof(double));
    for (int64_t i = 0; i < n; ++i) W[i + i * n] = 1.0;
    const double tol = 1e-15;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                double a = 0.0, bb = 0.0, g = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    a += G[i + p * n] * G[i + p * n];
                    bb += G[i + q * n] * G[i + q * n];
                    g += G[i + p * n] * G[i + q * n];
                }
                if (fabs(g) <= tol * sqrt(a * bb) || g == 0.0) continue;
                rotated = 1;
                double zeta = (bb - a) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int64_t i = 0; i < n; ++i) {
                    double gp = G[i + p * n], gq = G[i + q * n];
                    G[i + p * n] = cs * gp - sn * gq;
                    G[i + q * n] = sn * gp + cs * gq;
                    double wp = W[i + p * n], wq = W[i + q * n];
                    W[i + p * n] = cs * wp - sn * wq;
                    W[i + q * n] = sn * wp + cs * wq;
                }
            }
        }
        if (!rotated) break;
    }
    double* sv = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) { sv[j] = nrm2(n, G + j * n); order[j] = j; }
    for (int64_t a = 1; a < n; ++a) {  /* insertion sort, descending */
        int64_t key = order[a];
        int64_t b2 = a - 1;
        while (b2 >= 0 && sv[order[b2]] < sv[key]) { order[b2 + 1] = order[b2]; --b2; }
        order[b2 + 1] = key;
    }
    for (int64_t j = 0; j < n; ++j) {
        sigma[j] = sv[order[j]];
        for (int64_t i = 0; i < n; ++i) V[i + j * ldv] = W[i + order[j] * n];
    }
    free(G); free(W); free(sv); free(order);
    return sweep;
}

/* Truncated preconditioner of Algorithm 2: keep sigma_j > rcond * sigma_1
 * (the RCOND convention described before Algorithm 2), P = V_r Sigma_r^{-1}.
 * Returns r. */
int64_t orc_svd_precond(int64_t n, const double* sigma, const double* V, int64_t ldv,
                        double rcond, double* P, int64_t ldp) {
    int64_t r = 0;
    while (r < n && sigma[r] > rcond * sigma[0]) ++r;
    for (int64_t k = 0; k < r; ++k)
        for (int64_t i = 0; i < n; ++i) P[i + k * ldp] = V[i + k * ldv] / sigma[k];
    return r;
}

/* ------------------------------------------------------------------------ */
/* Gradients of a loss L(x_*) through the least-squares solution (implicit
 * differentiation; the paper has no backward pass). With g = dL/dx,
 * lambda = (A^T A)^{-1} g, r = b - A x:
 *   dL/db = A lambda,   dL/dA_ij = r_i lambda_j - (A lambda)_i x_j  (on the pattern).
 * lambda is computed densely as R_A^{-1} R_A^{-T} g from the R of A. */
void orc_adjoint(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                 const double* val, const double* b, const double* x, const double* RA,
                 int64_t ldr, const double* g, double* lambda, double* grad_b, double* grad_val) {
    memcpy(lambda, g, sizeof(double) * (size_t)n);
    orc_trsv_upper_trans(n, RA, ldr, lambda);
    orc_trsv_upper(n, RA, ldr, lambda);
    double* al = (double*)malloc(sizeof(double) * (size_t)m);
    orc_spmv(m, row_ptr, col, val, lambda, al);
    for (int64_t i = 0; i < m; ++i) grad_b[i] = al[i];
    for (int64_t i = 0; i < m; ++i) {
        double ax = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) ax += val[p] * x[col[p]];
        double ri = b[i] - ax;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            grad_val[p] = ri * lambda[col[p]] - al[i] * x[col[p]];
    }
    free(al);
}

/*
 * csls.h -- C ABI of the GB300 count-sketch preconditioned LSQR library.
 *
 * The library solves the overdetermined sparse least-squares problem
 *     min_x || A x - b ||_2,   A in R^{m x n}, m >= n,          (Section 1, eq. (1.1))
 * by the paper's CSQRP-LSQR / CSSVDP-LSQR method (Algorithms 1 and 2): a count
 * sketch SA with s = gamma n rows (Definition 2.3), a QR (or truncated SVD) of
 * the s x n sketch giving a right preconditioner, and LSQR on the
 * preconditioned operator. The preconditioner is applied per step (triangular
 * solves with R, the form of the Remark after Algorithm 2), so A R^{-1} is never
 * formed.
 *
 * Conventions for every entry point
 *  - All array pointers are DEVICE pointers unless a comment says "host".
 *    Arrays are owned by the caller; the library never frees them.
 *  - Dense matrices are column-major with an explicit leading dimension.
 *  - Integers are int64_t except CSR column indices (int32_t).
 *  - The library never calls cudaMalloc/cudaFree. Every call that needs
 *    scratch memory has a *_workspace query returning the byte counts; the
 *    caller allocates (any device memory, 256-byte aligned) and passes it in.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream). Calls that return a report synchronise `stream` before returning.
 *  - Every entry point returns a csls_status (0 = CSLS_OK). No call traps,
 *    aborts or exits; device-side waits are bounded and report
 *    CSLS_ERR_TIMEOUT instead of hanging.
 */
#ifndef CSLS_H
#define CSLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* csls_stream_t;

/* ---------------------------------------------------------------- status */
typedef enum {
    CSLS_OK = 0,
    CSLS_ERR_ARG = 1,            /* invalid argument, size, layout or CSR structure */
    CSLS_ERR_RANK_DEFICIENT = 2, /* R has a zero or non-finite diagonal entry (QR variant; cf. Theorem 3.1) */
    CSLS_ERR_NOT_CONVERGED = 3,  /* LSQR hit maxit before a stopping rule held */
    CSLS_ERR_BREAKDOWN = 4,      /* alpha or beta became zero with a nonzero residual estimate */
    CSLS_ERR_NONFINITE = 5,      /* NaN/Inf in A's values, in b or produced during the solve */
    CSLS_ERR_PRECOND_GUARD = 6,  /* binary32 factor rejected: estimated cond(A R^{-1}) >= opts.guard_cond */
    CSLS_ERR_TIMEOUT = 7,        /* a bounded device wait gave up (opts.spin_limit) */
    CSLS_ERR_CUDA = 8,           /* a CUDA runtime call failed */
    CSLS_ERR_WORKSPACE = 9       /* workspace pointer NULL/misaligned or smaller than the query */
} csls_status;

/* Human-readable name of a status code (static storage, never NULL). */
const char* csls_status_string(int status);

/* After a call returned CSLS_ERR_CUDA: the CUDA runtime's name and message for the error and the
 * library source location that saw it (per host thread; empty before any error; no paper
 * counterpart, a diagnostic). The string lives until the thread's next failing call. */
const char* csls_last_cuda_error(void);

/* ---------------------------------------------------------------- types */
enum { CSLS_VARIANT_QR = 0, CSLS_VARIANT_SVD = 1 };   /* Algorithm 1 / Algorithm 2 */
/* Arithmetic of the sketch and its factorisation:
 *   CSLS_PREC_F64      binary64 throughout (trailing updates on the FP64 MMA pipe);
 *   CSLS_PREC_F32      binary32 sketch and QR (accepted only under the cond guard);
 *   CSLS_PREC_F64_EMU  binary64 sketch and panels; the trailing-update products are computed
 *                      exactly from 8-bit digit pieces on the bf16 tensor cores and the trailing
 *                      matrix is kept in 62-bit fixed point per column: each product carries a
 *                      relative error of about 2^-38 of (sum |v| |c|), far below what the
 *                      preconditioner needs; R is stored in binary64. */
enum { CSLS_PREC_F64 = 0, CSLS_PREC_F32 = 1, CSLS_PREC_F64_EMU = 2 };

/* Sparse A in CSR form. Device pointers, caller-owned. Rows are zero-based;
 * column indices in [0, n), strictly ascending within each row. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t* row_ptr;   /* m + 1 entries, row_ptr[0] = 0, row_ptr[m] = nnz */
    const int32_t* col;       /* nnz entries */
    const double* val;        /* nnz entries */
} csls_csr;

typedef struct {
    double gamma;         /* oversampling factor: s = round(gamma n) when s <= 0 (Algorithm 1 step 1) */
    int64_t s;            /* sketch rows; clamped to m */
    uint64_t seed;        /* count-sketch hash seed */
    int variant;          /* CSLS_VARIANT_QR or CSLS_VARIANT_SVD */
    int factor_prec;      /* CSLS_PREC_F64, CSLS_PREC_F32 or CSLS_PREC_F64_EMU */
    double rcond;         /* SVD truncation sigma_i > rcond sigma_1; <= 0 means max(s, n) * 2^-53
                             (max(s, n) * 2^-38 with CSLS_PREC_F64_EMU) */
    double atol, btol;    /* Paige-Saunders stopping tolerances */
    int64_t maxit;        /* <= 0 means n (Section 4.1) */
    int64_t fixed_iters;  /* > 0: run exactly this many LSQR iterations, no stopping test */
    double guard_cond;    /* binary32 factor accepted only if estimated cond(A M) < guard_cond */
    int64_t spin_limit;   /* iteration bound for every device spin-wait */
    int64_t check_every;  /* host polls the convergence flag every this many iterations */
    int64_t time_kernels; /* nonzero: csls_factor brackets each launch of its three QR kernel
                             families with CUDA events and fills the kern_* report fields */
    int64_t warm_start;   /* nonzero: csls_solve starts LSQR from the x passed in (one right-hand
                             side): it solves for the correction from r0 = b - A x, keeps ||b|| in
                             the stopping rule, and returns x + correction. Use with the x0 of
                             csls_factor_warm (Remark 3.1) or any other initial guess. */
    int64_t refine;       /* restarts after the solve (single right-hand-side path): LSQR is run again
                             from the x just found, on the correction from r = b - A x, recomputed in
                             binary64 (the warm start above with x0 = the previous solution). With
                             per-step triangular solves the first solve's attainable accuracy in the
                             A-norm is limited by rounding in the preconditioner applications, relative
                             to the size of the iterates; the restart solves for a small correction, so
                             one restart brings x to the accuracy of the residual computation. 0 = none. */
} csls_opts;

/* Defaults: gamma 4, s 0, seed 1, QR, F64, rcond 0, atol = btol = 1e-12,
 * maxit 0 (= n), fixed_iters 0, guard_cond 10, spin_limit 2e7, check_every 16, time_kernels 0,
 * warm_start 0, refine 0. */
void csls_opts_default(csls_opts* opts);

/* Host-side report, filled by csls_factor / csls_solve / csls_solve_backward. */
typedef struct {
    int status;
    int istop;            /* 0 maxit or fixed, 1 rule S1, 2 rule S2, 3 exact (alpha or beta = 0) */
    int64_t iterations;
    int64_t s, r;         /* sketch rows used; preconditioner rank (n for QR) */
    double bnorm;         /* ||b|| */
    double rnorm;         /* LSQR estimate of ||b - A x|| */
    double arnorm;        /* LSQR estimate of ||(A M)^T r|| */
    double anorm;         /* running Frobenius estimate of ||A M|| */
    double ynorm;         /* ||y|| of the preconditioned problem */
    double cond_est;      /* cond(A M) from the Golub-Kahan bidiagonal of the last solve (0 if none) */
    double rdiag_min, rdiag_max;  /* min / max |R_jj| (QR variant) */
    double ms_sketch, ms_factor, ms_solve;  /* device time per phase (CUDA events) */
    int64_t launches;     /* kernels launched by the call */
    /* csls_factor with opts->time_kernels: per QR kernel family (0 Householder panel,
     * 1 W = V^T C product, 2 trailing update C -= V W) the summed CUDA-event time of its
     * launches, the launch count, and the algorithmic binary64 flops of the products
     * (2 L n' b per launch for an L x n' trailing matrix and a b-wide panel; 0 for panels). */
    double kern_ms[3];
    int64_t kern_launches[3];
    double kern_flop[3];
    int64_t iterations_refine;   /* csls_solve with opts->refine: iterations of the restarts (included in
                                    `iterations`) */
} csls_report;

typedef struct csls_factor_s csls_factor_t;

/* ---------------------------------------------------------------- sketch */
/* Count-sketch product SA = Phi D A (Definition 2.3; Algorithm 1 step 2).
 * Row i of A, times d(i) = +-1, is added to row h(i) of SA, where h(i) and d(i)
 * come from the SplitMix64 output stream of `seed` (output i = mix(seed + (i+1)
 * 0x9E3779B97F4A7C15); h = (hi32 * s) >> 32, d = -1 iff the low bit is set).
 * Each entry of SA is the sum of its contributions in ascending row order,
 * starting from +0.0, with plain (unfused) additions, so the result is
 * bit-reproducible. prec = CSLS_PREC_F64 writes double SA; CSLS_PREC_F32 rounds
 * each value to float first and writes float SA with float sums.
 *   SA: s x n column-major, leading dimension ld >= s, caller-owned; fully overwritten.
 * Workspace: csls_sketch_workspace(A, s, &bytes). */
int csls_sketch_workspace(const csls_csr* A, int64_t s, size_t* bytes);
int csls_sketch(const csls_csr* A, int64_t s, uint64_t seed, int prec, void* SA, int64_t ld,
                void* work, size_t work_bytes, csls_stream_t stream);

/* Same result as csls_sketch, for callers that cannot call cudaMalloc
 * themselves -- for example code whose device memory is entirely owned by
 * another framework's pool allocator, or a plug-in that the host application
 * forbids to allocate device memory after start-up. (The paper has no
 * counterpart; this is a library convenience.) Like csls_sketch, every call
 * first validates the CSR arrays and reads the result back to the host, so it
 * synchronises `stream` before it returns.
 * Instead of a caller workspace it uses a fixed 16 MiB scratch array that the
 * library keeps in device memory: every GPU that loads the library holds those
 * 16 MiB until the process exits. The call allocates nothing. Sizes whose
 * scratch needs exceed 16 MiB (roughly 4 m + 16 s bytes) are rejected with
 * CSLS_ERR_WORKSPACE before any device work; use csls_sketch for those.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress with that device current). All calls share the one
 * array and each call starts by
 * clearing what must start at zero, so calls that overlap on the GPU (different
 * streams, or different host threads on the same device) race and must be
 * serialised by the caller. Arguments, layout and results are those of
 * csls_sketch. */
int csls_sketch_noalloc(const csls_csr* A, int64_t s, uint64_t seed, int prec, void* SA, int64_t ld,
                        csls_stream_t stream);

/* ---------------------------------------------------------------- factor */
/* Algorithm 1 steps 1-3 (QR variant) or Algorithm 2 steps 1-3 (SVD variant):
 * sketch, blocked Householder QR of the s x n sketch, R with non-negative
 * diagonal; for the SVD variant also the one-sided Jacobi SVD R = U Sigma V^T
 * and P = V_r Sigma_r^{-1} with r = #{sigma_i > rcond sigma_1}. Also builds the
 * transposed CSR of A used for A^T u.
 * Two workspaces: `persist` holds the factor (R or P, block inverses, A^T, and for
 * a binary64 QR factor the per-step operand packs of the triangular solves,
 * 2 x ceil(n/64) x 160 KB) and must outlive the handle; `temp` (the dense sketch and QR scratch) may be
 * released once the call has returned. The handle itself is small host memory
 * owned by the library: release it with csls_factor_destroy (which frees no
 * device memory). rep may be NULL. */
int csls_factor_workspace(const csls_csr* A, const csls_opts* opts, size_t* persist_bytes,
                          size_t* temp_bytes);
int csls_factor(const csls_csr* A, const csls_opts* opts, void* persist, size_t persist_bytes,
                void* temp, size_t temp_bytes, csls_factor_t** factor, csls_report* rep,
                csls_stream_t stream);
/* csls_factor plus the warm start of Remark 3.1 (QR variant): b (m, device) is sketched with A,
 * the QR runs on the augmented sketch [SA, Sb], whose last column then holds Q^T S b, and
 * x0 (n, device, caller-owned) receives R^-1 (Q^T S b)(0:n) = argmin ||S (A x - b)||, the
 * sketch-and-solve point. The factor is the same as csls_factor's; the workspace sizes are
 * those of csls_factor_workspace (which always leaves room for the extra column). Pass x0 to
 * csls_solve with opts->warm_start set. Errors: CSLS_ERR_ARG for the SVD variant, NULL b or
 * x0, or s < n + 1; CSLS_ERR_NONFINITE for NaN/Inf in b. */
int csls_factor_warm(const csls_csr* A, const double* b, const csls_opts* opts, void* persist,
                     size_t persist_bytes, void* temp, size_t temp_bytes, csls_factor_t** factor,
                     double* x0, csls_report* rep, csls_stream_t stream);

int csls_factor_destroy(csls_factor_t* factor);

/* Read-only view of a factor for inspection. *R points to the n x n upper
 * triangle (ld n; double for CSLS_PREC_F64, float for CSLS_PREC_F32) or NULL;
 * *P to the n x r matrix P (double, ld n) or NULL. Any output may be NULL. */
int csls_factor_view(const csls_factor_t* factor, int64_t* n, int64_t* s, int64_t* r, int* variant,
                     int* prec, const void** R, const double** P);

/* ---------------------------------------------------------------- building blocks */
/* z = M v (trans = 0) or z = M^T v (trans = 1) for the factor's right
 * preconditioner M = R^{-1} (QR) or M = P (SVD): the per-step application of
 * Algorithm 1 step 4 in the implicit form. v and z are distinct device vectors
 * (length n, or r for the y-space side of P). */
int csls_precond_apply(const csls_factor_t* factor, int trans, const double* v, double* z,
                       void* work, size_t work_bytes, csls_stream_t stream);
/* y = A x (trans = 0, x length n, y length m) or y = A^T x (trans = 1), using
 * the factor's transposed copy of A for the latter. */
int csls_spmv(const csls_factor_t* factor, const csls_csr* A, int trans, const double* x, double* y,
              csls_stream_t stream);
int csls_apply_workspace(const csls_factor_t* factor, size_t* bytes);

/* ---------------------------------------------------------------- measurement */
/* Streaming-read probe (no paper counterpart): the HBM read ceiling that the
 * read-dominated SpMV pair is compared with. Reads `count` 8-byte words at `buf`
 * (device, 16-byte aligned, caller-owned) once, with ctas_per_sm CTAs of 512 threads
 * per SM, each thread keeping `unroll` independent 16-byte evict-first loads in
 * flight (bytes in flight = SMs x ctas_per_sm x 512 x unroll x 16), and folds them
 * into 64-bit wrap-around integer sums: partials (device, SMs x ctas_per_sm words)
 * receives one per CTA; their wrap-around sum is the sum of the words. Asynchronous
 * on `stream`. Errors: CSLS_ERR_ARG for a NULL partials (or a NULL buf with
 * count > 0), a misaligned buf, count < 0, ctas_per_sm outside 1..4, or unroll
 * other than 1, 2, 4 or 8. */
int csls_read_probe(const void* buf, int64_t count, int ctas_per_sm, int unroll, unsigned long long* partials,
                    csls_stream_t stream);

/* ---------------------------------------------------------------- solve */
/* Algorithm 1 steps 4-6 (Algorithm 2 steps 4-6): LSQR (Paige and Saunders 1982)
 * on min || A M y - b || from y = 0, returning x = M y. nrhs right-hand sides
 * are solved as independent LSQR recurrences that share each pass over A and
 * R (block form). b: m x nrhs (ld ldb >= m); x: n x nrhs (ld ldx >= n), both
 * caller-owned device memory. A must be the matrix the factor was built from.
 * rep (host, may be NULL) is filled after a stream synchronisation; for nrhs > 1
 * it reports the first column and the maximum iteration count.
 * With opts->refine > 0 each right-hand side (also in the block form) is
 * restarted that many times: LSQR on the correction from r = b - A x, added to x.
 * With a binary64 QR factor the triangular solves run as one cluster of 8 CTAs
 * plus worker CTAs that must become resident as earlier ones finish: a GPU kept
 * full by other work delays them, and a wait longer than 4 s ends the solve
 * with CSLS_ERR_TIMEOUT.
 * Status: CSLS_ERR_NOT_CONVERGED if maxit was reached before S1/S2 held (x is
 * still the last iterate); CSLS_ERR_PRECOND_GUARD for a binary32 factor whose
 * cond estimate is >= guard_cond (x still written). */
int csls_solve_workspace(const csls_factor_t* factor, int64_t nrhs, size_t* bytes);
int csls_solve(const csls_factor_t* factor, const csls_csr* A, const double* b, int64_t nrhs,
               int64_t ldb, double* x, int64_t ldx, const csls_opts* opts, void* work,
               size_t work_bytes, csls_report* rep, csls_stream_t stream);

/* ---------------------------------------------------------------- backward */
/* Gradients of a scalar loss L(x) through x = argmin ||A x - b|| (the paper
 * has no backward pass; implicit differentiation of the normal equations).
 * With g = dL/dx, lambda = (A^T A)^{-1} g and r = b - A x:
 *     dL/db = A lambda,    dL/dA_ij = r_i lambda_j - (A lambda)_i x_j  (on A's pattern).
 * lambda = R^{-1} mu with (B^T B) mu = R^{-T} g, B = A R^{-1}, solved by conjugate
 * gradients on the well-conditioned B^T B, reusing the forward factor.
 * grad_b (m) and grad_val (nnz) are device outputs; either may be NULL.
 * Single right-hand side. */
int csls_backward_workspace(const csls_factor_t* factor, size_t* bytes);
int csls_solve_backward(const csls_factor_t* factor, const csls_csr* A, const double* b,
                        const double* x, const double* grad_x, double* grad_b, double* grad_val,
                        const csls_opts* opts, void* work, size_t work_bytes, csls_report* rep,
                        csls_stream_t stream);

/* ---------------------------------------------------------------- RFM assembly */
/* One row of a random-feature-method system for the Poisson problem (Section 2.1):
 * kind 0 = -Laplace u at the local point t of `box`, 1 = the value u (boundary row),
 * 2 = C0 jump u(box) - u(nbox) and 3 = C1 jump of d u / d x_axis across the `axis` face
 * where box's local point is t (t[axis] = +1) and nbox's is t with t[axis] = -1.
 * Unused fields are ignored (t[2] in 2D; nbox, axis for kinds 0-1). */
typedef struct {
    int32_t kind, box, nbox, axis;
    double t[3];
} csls_rfm_row;

/* The CSR matrix of an RFM system on the device: box i carries J features
 * tanh(k_ij . l_i(x) + c_ij) with l_i the affine map of the box onto [-1, 1]^dim of
 * half-widths r_half (host, dim entries); k (device, boxes x J x dim, feature-major) and
 * c (device, boxes x J). rows (device, nrows descriptors) fix the row order. Output (device,
 * caller-owned): row_ptr (nrows + 1), col and val (sum of the widths: J per row of kinds
 * 0-1, 2 J for 2-3; columns box-major, ascending within each row). Scratch: the
 * csls_rfm_assemble_workspace bytes. Errors: CSLS_ERR_ARG (dim not 2 or 3, J outside 1..65536,
 * non-positive half-widths, NULL pointers). */
int csls_rfm_assemble_workspace(int64_t nrows, size_t* bytes);
/* The number of nonzeros csls_rfm_assemble will write for these rows (host output *nnz), so
 * that the caller can size col and val: the widths summed on the device (rows and work as for
 * csls_rfm_assemble); synchronises `stream` before it returns. Errors: CSLS_ERR_ARG (J outside
 * 1..65536, nrows <= 0, NULL pointers), CSLS_ERR_WORKSPACE. */
int csls_rfm_nnz(int64_t nrows, const csls_rfm_row* rows, int64_t J, void* work, size_t work_bytes,
                 int64_t* nnz, csls_stream_t stream);
int csls_rfm_assemble(int dim, const double* r_half, int64_t J, const double* k, const double* c,
                      int64_t nrows, const csls_rfm_row* rows, int64_t* row_ptr, int32_t* col,
                      double* val, void* work, size_t work_bytes, csls_stream_t stream);

/* ---------------------------------------------------------------- explicit form */
/* The paper's explicit form (Algorithm 1 / 2 steps 4-6): B = A R^-1 (QR variant) or B = A P
 * (SVD variant) formed as a dense m x r matrix, LSQR on B, x = R^-1 y or P y. It costs
 * m n^2 flops to form B (a right-side triangular solve on the densified A) and a dense
 * m x r pass per product, against the per-step triangular solves of csls_solve; it is
 * there to compare the two forms.
 * csls_form_b: B (device, column-major, ld ldb >= m, r columns; caller-owned, fully
 * written). QR variant needs a binary64 R (CSLS_ERR_ARG for a binary32 factor).
 * csls_solve_explicit: one right-hand side b (m) -> x (n); opts as for csls_solve
 * (warm_start ignored); rep as for csls_solve. */
int csls_form_b_workspace(const csls_factor_t* factor, size_t* bytes);
int csls_form_b(const csls_factor_t* factor, const csls_csr* A, double* B, int64_t ldb, void* work,
                size_t work_bytes, csls_stream_t stream);
int csls_solve_explicit_workspace(const csls_factor_t* factor, size_t* bytes);
int csls_solve_explicit(const csls_factor_t* factor, const double* B, int64_t ldb, const double* b,
                        double* x, const csls_opts* opts, void* work, size_t work_bytes,
                        csls_report* rep, csls_stream_t stream);

/* ---------------------------------------------------------------- batches */
/* Many independent problems of uneven size, each with its own factor (built by
 * csls_factor): all LSQR recurrences advance together in batched kernels whose
 * grids cover every instance, and the whole iteration runs as ONE CUDA-graph
 * launch -- a WHILE conditional node repeats one batched iteration until every
 * instance has met its stopping rule or limit (the loop condition is set on the
 * device). Each instance computes the same recurrence as csls_solve (single
 * right-hand side, QR variant). A[i], b[i] (m_i) and x[i] (n_i) are device arrays;
 * reps (host, count entries, may be NULL) is filled after a stream sync; each
 * report's status is that instance's, the return value the first non-OK one.
 * Binary32 factors get the cond guard per instance (CSLS_ERR_PRECOND_GUARD), also
 * early, after 32 and 128 iterations. opts->warm_start is not supported here
 * (CSLS_ERR_ARG). The call creates and destroys one capture stream and one graph
 * per call. */
int csls_batch_solve_workspace(int64_t count, const csls_factor_t* const* factors, size_t* bytes);
int csls_batch_solve(int64_t count, const csls_factor_t* const* factors, const csls_csr* A,
                     const double* const* b, double* const* x, const csls_opts* opts, void* work,
                     size_t work_bytes, csls_report* reps, csls_stream_t stream);

/* Autotuner for the SpMV pair: times A x and A^T u with 4, 8, 16 and 32 threads
 * per row (CUDA events, 5 runs each) on this matrix and stores the fastest
 * choices in the factor (used by csls_batch_solve). Workspace: 16 (m + n) + 1024
 * bytes. group, group_t and ms[2] (best times) may be NULL. */
int csls_autotune_spmv(csls_factor_t* factor, const csls_csr* A, void* work, size_t work_bytes, int* group,
                       int* group_t, float* ms, csls_stream_t stream);
/* Set the SpMV threads-per-row choices directly (4, 8, 16 or 32), e.g. from a
 * persisted autotuning cache. */
int csls_factor_set_spmv_groups(csls_factor_t* factor, int group, int group_t);

#ifdef __cplusplus
}
#endif

#endif /* CSLS_H */

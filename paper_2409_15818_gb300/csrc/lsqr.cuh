// Device-side LSQR state and the fused step helpers shared by the triangular
// solve, SpMV and dense-preconditioner kernels.
//
// Vector conventions (single right-hand side), following Paige and Saunders:
//   ut  = beta_{i} u_i       (u kept unnormalised; 1/beta folded into A^T u)
//   vt  = alpha_i v_i        (v kept unnormalised; 1/alpha folded into M v)
//   z   = M v_i              (M = R^{-1} or P)
//   wx  = M w_i              (search direction mapped to x-space)
//   x   = M y_i              (tracked directly)
#pragma once

#include "csls_internal.cuh"

namespace csls {

struct TrsvCtl {
    unsigned epoch;    // completed launches; flags of the current launch are set to epoch + 1
    unsigned ticket;   // block-row tickets handed out by the current launch
    unsigned done;     // CTAs finished in the current launch
    unsigned pad;
};

struct LsqrState {
    // recurrence (Paige-Saunders names)
    double alpha, beta;        // alpha_i and beta_{i+1} (beta_i before the SpMV of iteration i)
    double rhobar, phibar;
    double cx, cw;             // x += cx wx ; wx = z - cw wx   (applied in the next M-apply)
    double anorm2, bnorm, rnorm, arnorm, ynorm;
    double cs2, sn2, zz, xxnorm;   // ||y|| estimate (Paige-Saunders xnorm recurrence)
    double inv_beta;
    double atol, btol;
    double bnorm_ref;          // > 0: ||b|| of the original right-hand side (warm start), kept in rule S1
    long long iter, maxit, fixed, hist_cap;
    int done, istop, first, err;
    unsigned spmv_cnt, apply_cnt;
    TrsvCtl up, lo;
};

// Last-CTA detection: every CTA calls this after publishing its partial.
__device__ __forceinline__ bool last_cta(unsigned* counter, unsigned nblocks) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

// Fixed-order sum of nb partials (called by one thread).
__device__ __forceinline__ double sum_partials(const double* p, int nb) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += __ldcg(p + i);
    return t;
}

// Epilogue of M v_i for element k of the x-space vectors.
__device__ __forceinline__ void xw_update(LsqrState* st, int first, double cx, double cw, double zk, double* wx,
                                          double* x, int64_t k) {
    if (first) {
        wx[k] = zk;
    } else {
        const double w = wx[k];
        x[k] += cx * w;
        wx[k] = zk - cw * w;
    }
}

// Partial dot product of one CSR row with x for lane `sub` of a G-lane group (lane
// sub takes nonzeros sub, sub + G, ...; x is gathered through the read-only path).
__device__ __forceinline__ double row_dot(const int32_t* __restrict__ col, const double* __restrict__ val,
                                          const double* __restrict__ x, int64_t pb, int64_t pe, int sub, int G) {
    double acc = 0.0;
    for (int64_t p = pb + sub; p < pe; p += G) acc = fma(val[p], __ldg(x + col[p]), acc);
    return acc;
}

// The same for long rows with 16-byte loads: after an odd leading nonzero (taken by
// lane 0), lane sub takes the aligned pairs starting at 2 sub, 2 sub + 2G, ... and keeps
// four partial sums, combined in a fixed order. val and col must be 16- and 8-byte
// aligned at index 0 (allocation alignment).
__device__ __forceinline__ double row_dot_pairs(const int32_t* __restrict__ col, const double* __restrict__ val,
                                                const double* __restrict__ x, int64_t pb, int64_t pe, int sub,
                                                int G) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if ((pb & 1) && pb < pe) {
        if (sub == 0) a0 = val[pb] * __ldg(x + col[pb]);
        ++pb;
    }
    for (int64_t p = pb + 2 * sub; p < pe; p += 4 * (int64_t)G) {
        const int64_t q = p + 2 * (int64_t)G;
        double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0);
        int2 c0 = make_int2(-1, -1), c1 = make_int2(-1, -1);
        if (p + 1 < pe) {
            v0 = __ldcs(reinterpret_cast<const double2*>(val + p));
            c0 = __ldcs(reinterpret_cast<const int2*>(col + p));
        } else if (p < pe) {
            v0.x = val[p];
            c0.x = col[p];
        }
        if (q + 1 < pe) {
            v1 = __ldcs(reinterpret_cast<const double2*>(val + q));
            c1 = __ldcs(reinterpret_cast<const int2*>(col + q));
        } else if (q < pe) {
            v1.x = val[q];
            c1.x = col[q];
        }
        if (c0.x >= 0) a0 = fma(v0.x, __ldg(x + c0.x), a0);
        if (c0.y >= 0) a1 = fma(v0.y, __ldg(x + c0.y), a1);
        if (c1.x >= 0) a2 = fma(v1.x, __ldg(x + c1.x), a2);
        if (c1.y >= 0) a3 = fma(v1.y, __ldg(x + c1.y), a3);
    }
    return (a0 + a1) + (a2 + a3);
}

// One scalar step of LSQR after alpha_{i+1} is known (run by a single thread).
__device__ __forceinline__ void lsqr_scalar_step(LsqrState* st, double alpha_new, double* hist) {
    const double beta = st->beta;
    const double alpha_old = st->alpha;
    st->anorm2 += alpha_old * alpha_old + beta * beta;
    const double rhobar = st->rhobar, phibar = st->phibar;
    const double rho = sqrt(rhobar * rhobar + beta * beta);
    const double c = rhobar / rho, sn = beta / rho;
    const double theta = sn * alpha_new;
    const double phi = c * phibar;
    st->rhobar = -c * alpha_new;
    st->phibar = sn * phibar;
    // ||y|| estimate
    const double delta = st->sn2 * rho, gambar = -st->cs2 * rho;
    const double rhs = phi - delta * st->zz;
    const double zbar = rhs / gambar;
    st->ynorm = sqrt(st->xxnorm + zbar * zbar);
    const double gamma = sqrt(gambar * gambar + theta * theta);
    st->cs2 = gambar / gamma;
    st->sn2 = theta / gamma;
    st->zz = rhs / gamma;
    st->xxnorm += st->zz * st->zz;
    st->cx = phi / rho;
    st->cw = theta / rho;
    st->alpha = alpha_new;
    st->rnorm = st->phibar;
    st->arnorm = st->phibar * alpha_new * fabs(c);
    st->iter += 1;
    if (hist && st->iter <= st->hist_cap) {
        hist[2 * st->iter] = alpha_new;
        hist[2 * st->iter + 1] = beta;
    }
    const double anorm = sqrt(st->anorm2);
    int stop = 0, istop = 0;
    if (!isfinite(rho) || !isfinite(alpha_new) || !isfinite(st->phibar)) {
        stop = 1;
        set_error(&st->err, CSLS_ERR_NONFINITE);
    } else if (alpha_new == 0.0 || beta == 0.0) {
        stop = 1; istop = 3;
    } else if (st->fixed > 0) {
        stop = st->iter >= st->fixed;
    } else {
        if (st->rnorm <= st->btol * st->bnorm + st->atol * anorm * st->ynorm) { stop = 1; istop = 1; }
        else if (st->arnorm <= st->atol * anorm * st->rnorm) { stop = 1; istop = 2; }
        else if (st->iter >= st->maxit) { stop = 1; istop = 0; }
    }
    st->istop = istop;
    if (stop) st->done = 1;
}

// Condition number of the (k+1) x k lower bidiagonal B_k of the Golub-Kahan process
// (alpha_1..alpha_k on the diagonal, beta_2..beta_{k+1} below), read from the LSQR
// history (hist[2i] = alpha_{i+1}, hist[2i+3] = beta_{i+2}), by Sturm bisection on the
// tridiagonal B_k^T B_k. The singular values of B_k lie inside those of the
// preconditioned operator, so the value is a lower bound on cond(A M) that rises
// toward it with k.
__host__ __device__ inline double bidiag_cond_hist(const double* hist, long long k) {
    if (k <= 0) return 0.0;
    auto al = [&](long long i) { return hist[2 * i]; };
    auto be = [&](long long i) { return hist[2 * (i + 1) + 1]; };
    auto dg = [&](long long i) { return al(i) * al(i) + be(i) * be(i); };
    auto of = [&](long long i) { return al(i + 1) * be(i); };   // (i, i+1) entry of B^T B
    double hi = 0.0;
    for (long long i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(of(i - 1)) : 0.0) + (i + 1 < k ? fabs(of(i)) : 0.0);
        hi = fmax(hi, dg(i) + r);
    }
    auto count_below = [&](double x) {
        long long cnt = 0;
        double q = dg(0) - x;
        if (q < 0) ++cnt;
        for (long long i = 1; i < k; ++i) {
            const double qq = q != 0.0 ? q : 1e-300;
            const double e = of(i - 1);
            q = dg(i) - x - e * e / qq;
            if (q < 0) ++cnt;
        }
        return cnt;
    };
    auto kth = [&](long long idx) {
        double a = 0.0, b = hi;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (a + b);
            if (count_below(mid) > idx) b = mid; else a = mid;
            if (b - a <= 1e-15 * b) break;
        }
        return 0.5 * (a + b);
    };
    const double lmin = kth(0), lmax = kth(k - 1);
    if (!(lmin > 0.0)) return INFINITY;
    return sqrt(lmax / lmin);
}

// Iterations after which a binary32 factor's cond guard is evaluated early (the bound
// above already exceeds the guard when the factor has lost the preconditioner).
__host__ __device__ inline bool guard_checkpoint(long long it) { return it == 32 || it == 128; }

// ------------------------------------------------------------------ launchers (solve building blocks)

struct TrsvArgs {
    const void* R;          // n x n upper (ld n), double or float
    int rprec;              // CSLS_PREC_*
    const double* Dinv;
    int64_t n;
    int nb;                 // ceil(n / 64)
    const double* pack_up = nullptr;   // per-step operand packs of the cluster-chain solves (binary64 R)
    const double* pack_lo = nullptr;
};

// Synchronisation words of one solve direction, all zeroed before a solve's first launch: nb flag
// words (the one-CTA-per-block kernel), then, 16-byte aligned, two arrays of n + 64 tagged 16-byte
// words (the cluster-chain kernel: the chain's solutions for its workers, the workers' far sums).
inline int64_t trsv_flag_ints(int64_t nb, int64_t n) { return ((nb + 3) & ~(int64_t)3) + 8 * (n + 64); }
inline int64_t trsv_flag_count(int64_t nb, int64_t n) { return trsv_flag_ints(nb, n); }
inline ulonglong2* trsv_tagged(int* flags, int64_t nb) {
    return reinterpret_cast<ulonglong2*>(flags + ((nb + 3) & ~(int64_t)3));
}
// doubles of one direction's operand pack (ceil(n / 64) x 8 ranks x the per-step slot)
int64_t trsv_pack_doubles(int64_t n);
int trsv_build_packs(const double* R, int64_t n, const double* Dinv, double* pack_up, double* pack_lo,
                     cudaStream_t s);
// whether this device can keep the chain cluster and a worker cluster resident together
bool trsv_cluster_usable();
int launch_trsv_cl_upper(const TrsvArgs& a, int mode, const double* v, double* z, int* flags, TrsvCtl* ctl,
                         LsqrState* st, double* wx, double* x, long long spin, int* err, cudaStream_t s);
int launch_trsv_cl_lower(const TrsvArgs& a, int mode, double* g, double* vt, double* out, int* flags, TrsvCtl* ctl,
                         LsqrState* st, double* hist, long long spin, int* err, cudaStream_t s);

// mode 0: z = R^{-1} v. mode 1: LSQR step (v scaled by 1/alpha, x / wx epilogue).
int launch_trsv_upper(const TrsvArgs& a, int mode, const double* v, double* z, int* flags, TrsvCtl* ctl,
                      LsqrState* st, double* wx, double* x, long long spin, int* err, cudaStream_t s);
// mode 0: z = R^{-T} g (in place allowed: z == g). mode 1: LSQR step vt = R^{-T} g - (beta/alpha) vt,
// alpha update and scalar step. mode 2: LSQR start vt = R^{-T} g, alpha_1.
int launch_trsv_lower(const TrsvArgs& a, int mode, double* g, double* vt, double* out, int* flags, TrsvCtl* ctl,
                      LsqrState* st, double* partials, double* hist, long long spin, int* err, cudaStream_t s);

// mode 0: y = A x. mode 1: ut = A z - (alpha/beta) ut, beta update. mode 2: ut = b copy, beta_1.
int launch_spmv(const csls_csr* A, int mode, const double* x, double* y, LsqrState* st, double* partials,
                int grid, cudaStream_t s);
// y = A^T x * scale (scale = 1 for mode 0, st->inv_beta for mode 1).
// y = b - A x (row-parallel), the initial residual of a warm-started solve.
int launch_residual(const csls_csr* A, const double* x, const double* b, double* y, cudaStream_t s);
int launch_spmv_t(const Transpose& AT, int64_t n, int64_t m, int64_t nnz, int mode, const double* x, double* y,
                  LsqrState* st, cudaStream_t s);
int spmv_grid(const csls_csr* A);

// Dense preconditioner P (n x r, ld n) for the SVD variant.
// mode 0: z = P v. mode 1: LSQR step z = P (vt / alpha) with x / wx epilogue.
int launch_pgemv(const double* P, int64_t n, int64_t r, int mode, const double* v, double* z, LsqrState* st,
                 double* wx, double* x, cudaStream_t s);
// mode 0: y = P^T g. mode 1: vt = P^T g - (beta/alpha) vt + alpha update + scalar step. mode 2: start.
int launch_pgemv_t(const double* P, int64_t n, int64_t r, int mode, const double* g, double* vt, double* out,
                   LsqrState* st, double* partials, double* hist, cudaStream_t s);
// streaming-read probe: 64-bit checksum of `count` 8-byte words, one partial per CTA
int launch_read_probe(const void* buf, int64_t count, int ctas_per_sm, int unroll, unsigned long long* partials,
                      cudaStream_t s);

}  // namespace csls

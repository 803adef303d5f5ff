// The explicit form of the method (Algorithm 1 steps 4-6, Algorithm 2 steps 4-6): the
// preconditioned matrix B = A R^-1 (QR variant) or B = A P (SVD variant) is formed as a dense
// m x r matrix, LSQR runs on B with dense matrix-vector products, and x = R^-1 y (or P y).
//
// Forming B = A R^-1 is a right-side triangular solve X R = A on the densified A, done by
// 64-column blocks from left to right: block b is A(:, b) - X(:, <b) R(<b, b), then times the
// block's diagonal inverse. It costs m n^2 flops (binary64 FMA), against the implicit form's
// two triangular solves per iteration; the path exists to compare the two forms' accuracy.
//
// The LSQR recurrence is the one of the implicit solve (unnormalised u and v folded into
// the next kernel, fixed-order reductions finished by the last CTA, the scalar step in the
// last CTA of the v update); the preconditioner applications become the identity.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lsqr.cuh"

namespace csls {

constexpr int kXt = 64;    // rows and columns of a TRSM tile (= the diagonal block size)
constexpr int kXk = 16;    // K chunk of the tile product
constexpr int kExT = 256;  // threads per CTA of the LSQR kernels

static int ex_grid(int64_t work) {
    int64_t g = ceil_div(work, kExT);
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ forming B

__global__ void k_zero_dense(double* B, int64_t ld, int64_t m, int64_t ncols) {
    for (int64_t j = blockIdx.y; j < ncols; j += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
            B[i + j * ld] = 0.0;
}

// B(i, col) = A(i, col) for every stored entry (a warp per row).
__global__ void k_scatter_csr(const int64_t* rp, const int32_t* col, const double* val, int64_t m, double* B,
                              int64_t ld) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nw)
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) B[i + (int64_t)col[p] * ld] = val[p];
}

// Column block b of X R = Y, in place in B: rows [64 blockIdx.x, +64) of
// X(:, b) = (Y(:, b) - X(:, <b) R(<b, b)) inv(R_bb).
__global__ void __launch_bounds__(256) k_trsm_right(double* B, int64_t ld, int64_t m, int64_t n, const double* R,
                                                    const double* Dinv, int b) {
    __shared__ double Xs[kXk][kXt + 1];
    __shared__ double Rs[kXk][kXt + 1];
    __shared__ double Ys[kXt][kXt + 1];
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;   // outputs rows 4 tr.., cols 4 tc..
    const int64_t r0 = (int64_t)blockIdx.x * kXt, c0 = (int64_t)b * kXt;
    const int bs = (int)(n - c0 < kXt ? n - c0 : kXt);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t r = r0 + 4 * tr + i;
            const int c = 4 * tc + j;
            acc[i][j] = (r < m && c < bs) ? B[r + (c0 + c) * ld] : 0.0;
        }
    for (int64_t k0 = 0; k0 < c0; k0 += kXk) {
        for (int e = tid; e < kXk * kXt; e += 256) {
            const int rr = e % kXt, kk = e / kXt;
            const int64_t r = r0 + rr;
            Xs[kk][rr] = r < m ? B[r + (k0 + kk) * ld] : 0.0;
        }
        for (int e = tid; e < kXk * kXt; e += 256) {
            const int kk = e % kXk, cc = e / kXk;
            Rs[kk][cc] = cc < bs ? R[(k0 + kk) + (c0 + cc) * n] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kXk; ++kk) {
            double xv[4], rv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][4 * tr + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) rv[j] = Rs[kk][4 * tc + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(-xv[i], rv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Ys[4 * tr + i][4 * tc + j] = acc[i][j];
    __syncthreads();
    const double* D = Dinv + (int64_t)b * kXt * kXt;   // inv(R_bb), column-major
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * tc + j;
            double t = 0.0;
            for (int k = 0; k <= c; ++k) t += Ys[4 * tr + i][k] * __ldg(D + k + c * kXt);
            acc[i][j] = t;
        }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t r = r0 + 4 * tr + i;
            const int c = 4 * tc + j;
            if (r < m && c < bs) B[r + (c0 + c) * ld] = acc[i][j];
        }
}

// Pt = P^T (r x n, column-major), so that a row of A times P reads rows of P contiguously.
__global__ void k_transpose(const double* P, int64_t n, int64_t r, double* Pt) {
    for (int64_t k = blockIdx.y; k < n; k += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < r; j += (int64_t)gridDim.x * blockDim.x)
            Pt[j + k * r] = P[k + j * n];
}

// B(i, :) = sum_p A(i, col_p) P(col_p, :)  (one CTA per row, threads along the columns).
__global__ void k_rows_times_p(const int64_t* rp, const int32_t* col, const double* val, int64_t m, const double* Pt,
                               int64_t r, double* B, int64_t ld) {
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
        for (int64_t j = threadIdx.x; j < r; j += blockDim.x) {
            double t = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) t = fma(val[p], Pt[j + (int64_t)col[p] * r], t);
            B[i + j * ld] = t;
        }
}

// ------------------------------------------------------------------ LSQR on B

// LSQR start: ut = b, beta_1 = ||b||.
__global__ void __launch_bounds__(kExT) k_ex_start(const double* b, int64_t m, double* ut, LsqrState* st,
                                                   double* partials) {
    __shared__ double red[kExT / 32];
    double sq = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kExT + threadIdx.x; i < m; i += (int64_t)gridDim.x * kExT) {
        const double v = b[i];
        ut[i] = v;
        sq += v * v;
    }
    const double t = block_sum<kExT>(sq, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (last_cta(&st->spmv_cnt, gridDim.x) && threadIdx.x == 0) {
        const double beta = sqrt(sum_partials(partials, gridDim.x));
        st->beta = beta;
        st->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        st->bnorm = beta;
        st->phibar = beta;
        st->rnorm = beta;
        if (!isfinite(beta)) { set_error(&st->err, CSLS_ERR_NONFINITE); st->done = 1; }
        if (beta == 0.0) { st->done = 1; st->istop = 3; }
        st->spmv_cnt = 0;
    }
}

// z = vt / alpha and the y / wy epilogue (the identity in place of R^-1).
__global__ void __launch_bounds__(kExT) k_ex_apply(const double* vt, double* z, int64_t r, LsqrState* st, double* wy,
                                                   double* y) {
    __shared__ double coef[4];
    if (*(volatile int*)&st->done) return;
    if (threadIdx.x == 0) {
        coef[0] = 1.0 / st->alpha;
        coef[1] = st->cx;
        coef[2] = st->cw;
        coef[3] = (double)st->first;
    }
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)kExT + threadIdx.x; k < r; k += (int64_t)gridDim.x * kExT) {
        const double zk = vt[k] * coef[0];
        z[k] = zk;
        xw_update(st, coef[3] != 0.0, coef[1], coef[2], zk, wy, y, k);
    }
    if (last_cta(&st->apply_cnt, gridDim.x) && threadIdx.x == 0) {
        st->first = 0;
        st->apply_cnt = 0;
    }
}

// ut = B z - (alpha / beta) ut, beta_{i+1} = ||ut||: a thread per row, 8 columns in flight.
__global__ void __launch_bounds__(kExT) k_ex_gemv(const double* __restrict__ B, int64_t ld, int64_t m, int64_t r,
                                                  const double* __restrict__ z, double* ut, LsqrState* st,
                                                  double* partials) {
    __shared__ double red[kExT / 32];
    __shared__ double zs[1024];
    __shared__ double coef_s;
    if (*(volatile int*)&st->done) return;
    if (threadIdx.x == 0) coef_s = st->alpha / st->beta;
    const int64_t nrb = (m + kExT - 1) / kExT;
    double sq = 0.0;
    for (int64_t rb = blockIdx.x; rb < nrb; rb += gridDim.x) {
        const int64_t i = rb * kExT + threadIdx.x;
        double acc = 0.0;
        for (int64_t j0 = 0; j0 < r; j0 += 1024) {
            const int jn = (int)(r - j0 < 1024 ? r - j0 : 1024);
            __syncthreads();
            for (int t = threadIdx.x; t < jn; t += kExT) zs[t] = z[j0 + t];
            __syncthreads();
            if (i < m) {
                const double* bp = B + i + j0 * ld;
                int j = 0;
                double a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = 0.0;
                for (; j + 8 <= jn; j += 8) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) a[u] = fma(__ldcs(bp + (int64_t)(j + u) * ld), zs[j + u], a[u]);
                }
                for (; j < jn; ++j) a[0] = fma(__ldcs(bp + (int64_t)j * ld), zs[j], a[0]);
                acc += ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
            }
        }
        if (i < m) {
            const double un = acc - coef_s * ut[i];
            ut[i] = un;
            sq += un * un;
        }
    }
    const double t = block_sum<kExT>(sq, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (last_cta(&st->spmv_cnt, gridDim.x) && threadIdx.x == 0) {
        const double beta = sqrt(sum_partials(partials, gridDim.x));
        st->beta = beta;
        st->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(beta)) { set_error(&st->err, CSLS_ERR_NONFINITE); st->done = 1; }
        st->spmv_cnt = 0;
    }
}

// g = B^T ut / beta: a warp per column.
__global__ void __launch_bounds__(kExT) k_ex_gemv_t(const double* __restrict__ B, int64_t ld, int64_t m, int64_t r,
                                                    const double* __restrict__ ut, double* g, const LsqrState* st,
                                                    int mode) {
    if (mode == 1 && *(volatile const int*)&st->done) return;
    const double scale = st->inv_beta;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * kExT) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * kExT + threadIdx.x) >> 5; j < r; j += nw) {
        const double* bp = B + j * ld;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t i = lane;
        for (; i + 96 < m; i += 128) {
            a0 = fma(__ldcs(bp + i), __ldg(ut + i), a0);
            a1 = fma(__ldcs(bp + i + 32), __ldg(ut + i + 32), a1);
            a2 = fma(__ldcs(bp + i + 64), __ldg(ut + i + 64), a2);
            a3 = fma(__ldcs(bp + i + 96), __ldg(ut + i + 96), a3);
        }
        for (; i < m; i += 32) a0 = fma(__ldcs(bp + i), __ldg(ut + i), a0);
        double acc = (a0 + a1) + (a2 + a3);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) g[j] = acc * scale;
    }
}

// MODE 1: vt = g - (beta / alpha) vt, alpha and the scalar step. MODE 2: vt = g, alpha_1.
template <int MODE>
__global__ void __launch_bounds__(kExT) k_ex_vupdate(const double* g, double* vt, int64_t r, LsqrState* st,
                                                     double* partials, double* hist) {
    __shared__ double red[kExT / 32];
    __shared__ double coef_s;
    if (MODE == 1 && *(volatile int*)&st->done) return;
    if (threadIdx.x == 0) coef_s = MODE == 1 ? st->beta / st->alpha : 0.0;
    __syncthreads();
    double sq = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)kExT + threadIdx.x; k < r; k += (int64_t)gridDim.x * kExT) {
        const double vn = MODE == 1 ? g[k] - coef_s * vt[k] : g[k];
        vt[k] = vn;
        sq += vn * vn;
    }
    const double t = block_sum<kExT>(sq, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (last_cta(&st->apply_cnt, gridDim.x) && threadIdx.x == 0) {
        st->apply_cnt = 0;
        const double alpha_new = sqrt(sum_partials(partials, gridDim.x));
        if (MODE == 1) {
            lsqr_scalar_step(st, alpha_new, hist);
        } else {
            st->alpha = alpha_new;
            st->rhobar = alpha_new;
            if (hist) hist[0] = alpha_new;
            if (alpha_new == 0.0 || !isfinite(alpha_new)) {
                st->done = 1;
                st->istop = 3;
                if (!isfinite(alpha_new)) set_error(&st->err, CSLS_ERR_NONFINITE);
            }
        }
    }
}

__global__ void k_ex_final(double* y, const double* wy, int64_t r, const LsqrState* st) {
    const double cx = st->cx;
    if (st->iter <= 0) return;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < r; k += (int64_t)gridDim.x * blockDim.x)
        y[k] += cx * wy[k];
}

__global__ void k_ex_check_finite(const double* v, int64_t len, int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) set_error(err, CSLS_ERR_NONFINITE);
}

struct ExWs {
    LsqrState* st;
    double *ut, *vt, *z, *g, *wy, *y, *part, *hist;
    TrsvCtl* ctl;
    int* flags;
    int64_t hist_cap;
};

static ExWs ex_carve(Carve& c, const csls_factor_t* F) {
    ExWs w;
    const int64_t m = F->m, r = F->r;
    w.st = c.take<LsqrState>(1);
    w.ut = c.take<double>((size_t)m);
    w.vt = c.take<double>((size_t)r);
    w.z = c.take<double>((size_t)r);
    w.g = c.take<double>((size_t)r);
    w.wy = c.take<double>((size_t)r);
    w.y = c.take<double>((size_t)r);
    w.part = c.take<double>((size_t)device_sm_count() * 8 + 64);
    w.hist_cap = r + 4;
    w.hist = c.take<double>((size_t)(2 * (r + 6)));
    w.ctl = c.take<TrsvCtl>(1);
    w.flags = c.take<int>((size_t)trsv_flag_ints(F->nblocks, F->n));
    return w;
}

}  // namespace csls

using namespace csls;

static bool ex_aligned(const void* p) { return ((uintptr_t)p & 255) == 0; }

int csls_form_b_workspace(const csls_factor_t* F, size_t* bytes) {
    if (!F || !bytes) return CSLS_ERR_ARG;
    *bytes = F->variant == CSLS_VARIANT_SVD ? (size_t)round_up((int64_t)(F->n * F->r * 8), 256) : 256;
    return CSLS_OK;
}

int csls_form_b(const csls_factor_t* F, const csls_csr* A, double* B, int64_t ldb, void* work, size_t work_bytes,
                csls_stream_t stream) {
    if (!F || !A || !B || A->m != F->m || A->n != F->n || A->nnz != F->nnz || ldb < F->m) return CSLS_ERR_ARG;
    if (F->variant == CSLS_VARIANT_QR && F->prec != CSLS_PREC_F64) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_form_b_workspace(F, &need));
    if (!work || work_bytes < need || !ex_aligned(work)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t m = F->m, n = F->n;
    if (F->variant == CSLS_VARIANT_QR) {
        dim3 zg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 256), 64)),
                (unsigned)std::min<int64_t>(n, 65535));
        k_zero_dense<<<zg, 256, 0, st>>>(B, ldb, m, n);
        CSLS_CUDA(cudaGetLastError());
        k_scatter_csr<<<ex_grid(m * 32), kExT, 0, st>>>(A->row_ptr, A->col, A->val, m, B, ldb);
        CSLS_CUDA(cudaGetLastError());
        const unsigned rt = (unsigned)ceil_div(m, (int64_t)kXt);
        for (int b = 0; b < (int)F->nblocks; ++b) {
            k_trsm_right<<<rt, 256, 0, st>>>(B, ldb, m, n, (const double*)F->R, F->Dinv, b);
            CSLS_CUDA(cudaGetLastError());
        }
    } else {
        const int64_t r = F->r;
        double* Pt = (double*)work;
        dim3 tg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(r, 256), 64)),
                (unsigned)std::min<int64_t>(n, 65535));
        k_transpose<<<tg, 256, 0, st>>>(F->P, n, r, Pt);
        CSLS_CUDA(cudaGetLastError());
        k_rows_times_p<<<(unsigned)std::min<int64_t>(m, (int64_t)device_sm_count() * 64), 256, 0, st>>>(
            A->row_ptr, A->col, A->val, m, Pt, r, B, ldb);
        CSLS_CUDA(cudaGetLastError());
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? CSLS_OK : CSLS_ERR_CUDA;
}

int csls_solve_explicit_workspace(const csls_factor_t* F, size_t* bytes) {
    if (!F || !bytes) return CSLS_ERR_ARG;
    Carve c{nullptr, 0, 0, true};
    ex_carve(c, F);
    *bytes = c.off;
    return CSLS_OK;
}

int csls_solve_explicit(const csls_factor_t* F, const double* B, int64_t ldb, const double* b, double* x,
                        const csls_opts* o, void* work, size_t work_bytes, csls_report* rep, csls_stream_t stream) {
    if (!F || !B || !b || !x || !o || ldb < F->m) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_solve_explicit_workspace(F, &need));
    if (!work || work_bytes < need || !ex_aligned(work)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Carve c{(char*)work, 0, work_bytes, false};
    ExWs w = ex_carve(c, F);
    const int64_t m = F->m, n = F->n, r = F->r;
    if (rep) std::memset(rep, 0, sizeof(*rep));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    LsqrState h{};
    h.atol = o->atol;
    h.btol = o->btol;
    h.maxit = o->maxit > 0 ? o->maxit : n;
    h.fixed = o->fixed_iters;
    h.hist_cap = w.hist_cap;
    h.cs2 = -1.0;
    h.first = 1;
    CSLS_CUDA(cudaMemcpyAsync(w.st, &h, sizeof(LsqrState), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemsetAsync(w.y, 0, sizeof(double) * (size_t)r, st));
    CSLS_CUDA(cudaMemsetAsync(w.wy, 0, sizeof(double) * (size_t)r, st));
    CSLS_CUDA(cudaMemsetAsync(w.hist, 0, sizeof(double) * (size_t)(2 * (r + 6)), st));
    k_ex_check_finite<<<ex_grid(m), 256, 0, st>>>(b, m, &w.st->err);
    CSLS_CUDA(cudaGetLastError());
    const int gm = ex_grid(m), gr = ex_grid(r), gt = ex_grid(r * 32);
    int64_t launches = 1;
    // start: beta_1 u_1 = b ; alpha_1 v_1 = B^T u_1
    k_ex_start<<<gm, kExT, 0, st>>>(b, m, w.ut, w.st, w.part);
    k_ex_gemv_t<<<gt, kExT, 0, st>>>(B, ldb, m, r, w.ut, w.g, w.st, 0);
    k_ex_vupdate<2><<<gr, kExT, 0, st>>>(w.g, w.vt, r, w.st, w.part, w.hist);
    CSLS_CUDA(cudaGetLastError());
    launches += 3;
    const int64_t limit = o->fixed_iters > 0 ? o->fixed_iters : h.maxit;
    const int64_t chunk = o->check_every > 0 ? o->check_every : 16;
    const int gv = (int)std::min<int64_t>(ceil_div(m, (int64_t)kExT), (int64_t)device_sm_count() * 8);
    for (int64_t it = 0; it < limit; it += chunk) {
        for (int64_t k = 0; k < chunk && it + k < limit; ++k) {
            k_ex_apply<<<gr, kExT, 0, st>>>(w.vt, w.z, r, w.st, w.wy, w.y);
            k_ex_gemv<<<gv, kExT, 0, st>>>(B, ldb, m, r, w.z, w.ut, w.st, w.part);
            k_ex_gemv_t<<<gt, kExT, 0, st>>>(B, ldb, m, r, w.ut, w.g, w.st, 1);
            k_ex_vupdate<1><<<gr, kExT, 0, st>>>(w.g, w.vt, r, w.st, w.part, w.hist);
            CSLS_CUDA(cudaGetLastError());
            launches += 4;
        }
        int done = 0;
        CSLS_CUDA(cudaMemcpyAsync(&done, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CSLS_CUDA(cudaStreamSynchronize(st));
        if (done) break;
    }
    k_ex_final<<<gr, 256, 0, st>>>(w.y, w.wy, r, w.st);
    CSLS_CUDA(cudaGetLastError());
    // x = R^-1 y  or  P y
    if (F->variant == CSLS_VARIANT_QR) {
        TrsvArgs ta{F->R, F->prec, F->Dinv, n, (int)F->nblocks, F->pack_up, F->pack_lo};
        CSLS_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(TrsvCtl), st));
        CSLS_CUDA(cudaMemsetAsync(w.flags, 0, sizeof(int) * (size_t)trsv_flag_count(F->nblocks, F->n), st));
        CSLS_TRY(launch_trsv_upper(ta, 0, w.y, x, w.flags, w.ctl, nullptr, nullptr, nullptr, o->spin_limit,
                                   &w.st->err, st));
    } else {
        CSLS_TRY(launch_pgemv(F->P, n, r, 0, w.y, x, nullptr, nullptr, nullptr, st));
    }
    launches += 2;
    cudaEventRecord(e1, st);
    LsqrState out{};
    CSLS_CUDA(cudaMemcpyAsync(&out, w.st, sizeof(LsqrState), cudaMemcpyDeviceToHost, st));
    const int64_t kk = std::min<int64_t>(out.iter, w.hist_cap);
    std::vector<double> hh((size_t)(2 * (kk + 1) + 2));
    CSLS_CUDA(cudaMemcpyAsync(hh.data(), w.hist, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double cond = bidiag_cond_hist(hh.data(), kk);
    if (rep) {
        rep->istop = out.istop;
        rep->iterations = out.iter;
        rep->s = F->s;
        rep->r = r;
        rep->bnorm = out.bnorm;
        rep->rnorm = out.rnorm;
        rep->arnorm = out.arnorm;
        rep->anorm = std::sqrt(out.anorm2);
        rep->ynorm = out.ynorm;
        rep->cond_est = cond;
        rep->ms_solve = ms;
        rep->launches = launches;
    }
    int status = out.err;
    if (status == CSLS_OK && o->fixed_iters <= 0 && out.istop == 0) status = CSLS_ERR_NOT_CONVERGED;
    if (rep) rep->status = status;
    return status;
}

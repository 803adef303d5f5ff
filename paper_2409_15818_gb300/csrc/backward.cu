// Adjoint of the least-squares solve (implicit differentiation; the paper has
// no backward pass). With g = dL/dx, lambda = (A^T A)^{-1} g is computed as
// lambda = R^{-1} mu, (B^T B) mu = R^{-T} g, B = A R^{-1}, by conjugate gradients
// on the well-conditioned B^T B (cond(B)^2 = O(1) by Theorem 3.2) reusing the
// forward factor. lambda is accumulated directly: lambda += a_k R^{-1} p_k.
// Then dL/db = A lambda and dL/dA_ij = r_i lambda_j - (A lambda)_i x_j.
#include <algorithm>
#include <cstring>

#include "lsqr.cuh"

namespace csls {

struct CgState {
    double rr, rr0, pq, alpha, beta;
    long long iter, maxit;
    double tol;
    int done;
    unsigned cnt;
};

constexpr int kCgThreads = 256;

__device__ __forceinline__ void block_partial(double v, double* partials) {
    __shared__ double red[kCgThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kCgThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// r = p = h ; rr = ||h||^2 ; lambda = 0
__global__ void __launch_bounds__(kCgThreads) k_cg_init(const double* h, double* r, double* p, double* lam, int64_t n,
                                                        CgState* cs, double* partials) {
    double sq = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = h[i];
        r[i] = v; p[i] = v; lam[i] = 0.0;
        sq += v * v;
    }
    block_partial(sq, partials);
    if (last_cta(&cs->cnt, gridDim.x) && threadIdx.x == 0) {
        cs->rr = sum_partials(partials, gridDim.x);
        cs->rr0 = cs->rr;
        cs->iter = 0;
        cs->done = !(cs->rr > 0.0);
        cs->cnt = 0;
    }
}

// pq = ||w||^2 (w = B p = A t) ; alpha = rr / pq
__global__ void __launch_bounds__(kCgThreads) k_cg_pq(const double* w, int64_t m, CgState* cs, double* partials) {
    if (*(volatile int*)&cs->done) return;
    double sq = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        sq += w[i] * w[i];
    block_partial(sq, partials);
    if (last_cta(&cs->cnt, gridDim.x) && threadIdx.x == 0) {
        cs->pq = sum_partials(partials, gridDim.x);
        cs->alpha = cs->pq > 0.0 ? cs->rr / cs->pq : 0.0;
        cs->cnt = 0;
    }
}

// lambda += alpha t ; r -= alpha q ; rr_new ; beta ; p = r + beta p (after the reduction, separate kernel)
__global__ void __launch_bounds__(kCgThreads) k_cg_update(const double* t, const double* q, double* lam, double* r,
                                                          int64_t n, CgState* cs, double* partials) {
    if (*(volatile int*)&cs->done) return;
    const double a = cs->alpha;
    double sq = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        lam[i] += a * t[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        sq += ri * ri;
    }
    block_partial(sq, partials);
    if (last_cta(&cs->cnt, gridDim.x) && threadIdx.x == 0) {
        const double rr_new = sum_partials(partials, gridDim.x);
        cs->beta = cs->rr > 0.0 ? rr_new / cs->rr : 0.0;
        cs->rr = rr_new;
        cs->iter += 1;
        if (!(rr_new > cs->tol * cs->tol * cs->rr0) || cs->iter >= cs->maxit || !isfinite(rr_new)) cs->done = 1;
        cs->cnt = 0;
    }
}

__global__ void k_cg_dir(const double* r, double* p, int64_t n, const CgState* cs) {
    if (*(volatile const int*)&cs->done) return;
    const double b = cs->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + b * p[i];
}

// Per row: ax = (A x)_i, al = (A lambda)_i ; grad_b = al ; grad_val = (b_i - ax) lambda_j - al x_j.
__global__ void __launch_bounds__(kCgThreads)
k_grad(const int64_t* rp, const int32_t* col, const double* val, int64_t m, const double* b, const double* x,
       const double* lam, double* grad_b, double* grad_val) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double ax = 0.0, al = 0.0;
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            const int32_t j = col[p];
            ax += val[p] * x[j];
            al += val[p] * lam[j];
        }
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            al += __shfl_xor_sync(0xffffffffu, al, o);
        }
        if (grad_b && lane == 0) grad_b[i] = al;
        if (grad_val) {
            const double ri = b[i] - ax;
            for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
                const int32_t j = col[p];
                grad_val[p] = ri * lam[j] - al * x[j];
            }
        }
    }
}

// ------------------------------------------------------------------ host driver

struct BackwardWs {
    CgState* cs;
    double *h, *r, *p, *t, *q, *w, *g2, *lam, *partials;
    int* flags_up;
    int* flags_lo;
    TrsvCtl* ctl;   // [2]
    int* err;
};

size_t backward_ws_bytes(int64_t m, int64_t n, int64_t nb);
BackwardWs backward_ws_carve(Carve& c, int64_t m, int64_t n, int64_t nb);

size_t backward_ws_bytes(int64_t m, int64_t n, int64_t nb) {
    Carve c{nullptr, 0, 0, true};
    backward_ws_carve(c, m, n, nb);
    return c.off;
}

BackwardWs backward_ws_carve(Carve& c, int64_t m, int64_t n, int64_t nb) {
    BackwardWs w;
    w.cs = c.take<CgState>(1);
    w.h = c.take<double>((size_t)n);
    w.r = c.take<double>((size_t)n);
    w.p = c.take<double>((size_t)n);
    w.t = c.take<double>((size_t)n);
    w.q = c.take<double>((size_t)n);
    w.g2 = c.take<double>((size_t)n);
    w.lam = c.take<double>((size_t)n);
    w.w = c.take<double>((size_t)m);
    w.partials = c.take<double>((size_t)device_sm_count() * 8 + 64);
    w.flags_up = c.take<int>((size_t)trsv_flag_ints(nb, n));
    w.flags_lo = c.take<int>((size_t)trsv_flag_ints(nb, n));
    w.ctl = c.take<TrsvCtl>(2);
    w.err = c.take<int>(1);
    return w;
}

int backward_run(const csls_factor_t* F, const csls_csr* A, const double* b, const double* x, const double* grad_x,
                 double* grad_b, double* grad_val, const csls_opts* o, const BackwardWs& w, csls_report* rep,
                 cudaStream_t st) {
    const int64_t n = F->n, m = F->m;
    if (F->variant != CSLS_VARIANT_QR) return CSLS_ERR_ARG;
    TrsvArgs ta{F->R, F->prec, F->Dinv, n, (int)F->nblocks, F->pack_up, F->pack_lo};
    const long long spin = o->spin_limit;
    CSLS_CUDA(cudaMemsetAsync(w.flags_up, 0, sizeof(int) * (size_t)trsv_flag_count(F->nblocks, F->n), st));
    CSLS_CUDA(cudaMemsetAsync(w.flags_lo, 0, sizeof(int) * (size_t)trsv_flag_count(F->nblocks, F->n), st));
    CSLS_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(TrsvCtl) * 2, st));
    CSLS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    CgState hc{};
    hc.tol = o->atol > 0 ? o->atol : 1e-12;
    hc.maxit = o->maxit > 0 ? o->maxit : n;
    CSLS_CUDA(cudaMemcpyAsync(w.cs, &hc, sizeof(CgState), cudaMemcpyHostToDevice, st));
    // h = R^{-T} g
    CSLS_CUDA(cudaMemcpyAsync(w.h, grad_x, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    CSLS_TRY(launch_trsv_lower(ta, 0, w.h, nullptr, w.h, w.flags_lo, &w.ctl[1], nullptr, nullptr, nullptr, spin, w.err, st));
    const int gv = (int)std::min<int64_t>(ceil_div(n, kCgThreads), (int64_t)device_sm_count() * 8);
    const int gm = (int)std::min<int64_t>(ceil_div(m, kCgThreads), (int64_t)device_sm_count() * 8);
    k_cg_init<<<gv, kCgThreads, 0, st>>>(w.h, w.r, w.p, w.lam, n, w.cs, w.partials);
    CSLS_CUDA(cudaGetLastError());
    int64_t launches = 4;
    const int64_t chunk = o->check_every > 0 ? o->check_every : 16;
    for (int64_t it = 0; it < hc.maxit; it += chunk) {
        for (int64_t k = 0; k < chunk; ++k) {
            // t = R^{-1} p ; w = A t ; pq = ||w||^2 ; g2 = A^T w ; q = R^{-T} g2
            CSLS_TRY(launch_trsv_upper(ta, 0, w.p, w.t, w.flags_up, &w.ctl[0], nullptr, nullptr, nullptr, spin, w.err, st));
            CSLS_TRY(launch_spmv(A, 0, w.t, w.w, nullptr, nullptr, spmv_grid(A), st));
            k_cg_pq<<<gm, kCgThreads, 0, st>>>(w.w, m, w.cs, w.partials);
            CSLS_CUDA(cudaGetLastError());
            CSLS_TRY(launch_spmv_t(F->AT, n, m, F->nnz, 0, w.w, w.g2, nullptr, st));
            CSLS_TRY(launch_trsv_lower(ta, 0, w.g2, nullptr, w.q, w.flags_lo, &w.ctl[1], nullptr, nullptr, nullptr, spin, w.err, st));
            k_cg_update<<<gv, kCgThreads, 0, st>>>(w.t, w.q, w.lam, w.r, n, w.cs, w.partials);
            CSLS_CUDA(cudaGetLastError());
            k_cg_dir<<<gv, kCgThreads, 0, st>>>(w.r, w.p, n, w.cs);
            CSLS_CUDA(cudaGetLastError());
            launches += 7;
        }
        int done = 0;
        CSLS_CUDA(cudaMemcpyAsync(&done, &w.cs->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CSLS_CUDA(cudaStreamSynchronize(st));
        if (done) break;
    }
    const int gr = (int)std::min<int64_t>(ceil_div(m * 32, kCgThreads), (int64_t)device_sm_count() * 16);
    k_grad<<<gr, kCgThreads, 0, st>>>(A->row_ptr, A->col, A->val, m, b, x, w.lam, grad_b, grad_val);
    CSLS_CUDA(cudaGetLastError());
    ++launches;
    CgState out{};
    int err = 0;
    CSLS_CUDA(cudaMemcpyAsync(&out, w.cs, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    if (rep) {
        rep->iterations = out.iter;
        rep->rnorm = sqrt(out.rr);
        rep->bnorm = sqrt(out.rr0);
        rep->launches += launches;
    }
    if (err) return err;
    if (!isfinite(out.rr)) return CSLS_ERR_NONFINITE;
    if (!out.done) return CSLS_ERR_NOT_CONVERGED;
    if (out.iter >= out.maxit && out.rr > out.tol * out.tol * out.rr0) return CSLS_ERR_NOT_CONVERGED;
    return CSLS_OK;
}

}  // namespace csls

// ======================================================================= C ABI

extern "C" int csls_solve_backward(const csls_factor_t* F, const csls_csr* A, const double* b, const double* x,
                                   const double* grad_x, double* grad_b, double* grad_val, const csls_opts* o,
                                   void* work, size_t work_bytes, csls_report* rep, csls_stream_t stream) {
    using namespace csls;
    if (!F || !A || !o || !b || !x || !grad_x) return CSLS_ERR_ARG;
    if (A->m != F->m || A->n != F->n || A->nnz != F->nnz || !A->row_ptr) return CSLS_ERR_ARG;
    size_t need = 0;
    if (csls_backward_workspace(F, &need) != CSLS_OK) return CSLS_ERR_ARG;
    if (!work || work_bytes < need || ((uintptr_t)work & 255)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Carve c{(char*)work, 0, work_bytes, false};
    BackwardWs w = backward_ws_carve(c, F->m, F->n, F->nblocks);
    if (rep) std::memset(rep, 0, sizeof(*rep));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    int rc = backward_run(F, A, b, x, grad_x, grad_b, grad_val, o, w, rep, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rep) {
        rep->ms_solve = ms;
        rep->status = rc;
        rep->s = F->s;
        rep->r = F->r;
    }
    return rc;
}

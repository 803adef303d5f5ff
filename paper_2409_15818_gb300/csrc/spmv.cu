// CSR SpMV with A (row-parallel, G lanes per row) and with A^T through the
// transposed copy built at factor time, with the LSQR vector update and the
// ||u||^2 reduction fused into the A z epilogue; also the dense P / P^T
// products of the SVD variant.
#include "lsqr.cuh"

namespace csls {

constexpr int kSpThreads = 256;

__device__ __forceinline__ double group_sum(double v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// MODE 0: y = A x. MODE 1: ut = A z - (alpha/beta) ut, beta_{i+1} = ||ut||.
// MODE 2: ut = b, beta_1 = ||b|| and the LSQR start values.
template <int G, int MODE>
__global__ void __launch_bounds__(kSpThreads)
k_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const double* __restrict__ val, int64_t m,
       const double* __restrict__ x, double* y, LsqrState* st, double* partials) {
    __shared__ double red[kSpThreads / 32];
    __shared__ double coef_s;
    const int tid = threadIdx.x, lane = tid & 31, sub = lane & (G - 1);
    if (MODE == 1 && *(volatile int*)&st->done) return;
    if (tid == 0) coef_s = MODE == 1 ? st->alpha / st->beta : 0.0;
    __syncthreads();
    const double coef = coef_s;
    const int rows_per_warp = 32 / G;
    const int64_t warp_g = ((int64_t)blockIdx.x * kSpThreads + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kSpThreads) >> 5;
    double sq = 0.0;
    const int64_t stride = nwarps * rows_per_warp;
    // the next row's bounds (and old u entry) are loaded before the current row's data
    int64_t i = warp_g * rows_per_warp + (lane / G);
    int64_t pb = 0, pe = 0;
    double yo = 0.0;
    if (i < m) {
        if (MODE != 2) { pb = rp[i]; pe = rp[i + 1]; }
        if (MODE == 1 && sub == 0) yo = y[i];
    }
    for (int64_t base = warp_g * rows_per_warp; base < m; base += stride) {
        const bool active = i < m;
        const int64_t inext = i + stride;
        int64_t nb = 0, ne = 0;
        double yn = 0.0;
        if (inext < m) {
            if (MODE != 2) { nb = rp[inext]; ne = rp[inext + 1]; }
            if (MODE == 1 && sub == 0) yn = y[inext];
        }
        double acc = 0.0;
        if (MODE != 2 && active) acc = row_dot(col, val, x, pb, pe, sub, G);
        if (MODE != 2) acc = group_sum(acc, G);
        if (active && sub == 0) {
            if (MODE == 0) {
                y[i] = acc;
            } else if (MODE == 1) {
                const double un = acc - coef * yo;
                y[i] = un;
                sq += un * un;
            } else {
                const double bi = x[i];
                y[i] = bi;
                sq += bi * bi;
            }
        }
        i = inext; pb = nb; pe = ne; yo = yn;
    }
    if constexpr (MODE == 0) {
        return;
    } else {
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kSpThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
    if (last_cta(&st->spmv_cnt, gridDim.x) && tid == 0) {
        const double beta = sqrt(sum_partials(partials, gridDim.x));
        st->beta = beta;
        st->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(beta)) {
            set_error(&st->err, CSLS_ERR_NONFINITE);
            st->done = 1;
        }
        if (MODE == 2) {
            st->bnorm = st->bnorm_ref > 0.0 ? st->bnorm_ref : beta;
            st->phibar = beta;
            st->rnorm = beta;
            if (beta == 0.0) { st->done = 1; st->istop = 3; }
        }
        st->spmv_cnt = 0;
    }
    }
}

// y = scale * A^T x with A^T in CSR (rows = columns of A). scale = 1 (MODE 0) or 1/beta (MODE 1).
template <int G, int MODE>
__global__ void __launch_bounds__(kSpThreads)
k_spmv_t(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const double* __restrict__ val, int64_t n,
         const double* __restrict__ x, double* y, const LsqrState* st) {
    __shared__ double scale_s;
    const int tid = threadIdx.x, lane = tid & 31, sub = lane & (G - 1);
    if (MODE == 1 && *(volatile const int*)&st->done) return;
    if (tid == 0) scale_s = MODE == 1 ? st->inv_beta : 1.0;
    __syncthreads();
    const double scale = scale_s;
    const int rows_per_warp = 32 / G;
    const int64_t warp_g = ((int64_t)blockIdx.x * kSpThreads + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kSpThreads) >> 5;
    const int64_t stride = nwarps * rows_per_warp;
    int64_t j = warp_g * rows_per_warp + (lane / G);
    int64_t pb = 0, pe = 0;
    if (j < n) { pb = rp[j]; pe = rp[j + 1]; }
    for (int64_t base = warp_g * rows_per_warp; base < n; base += stride) {
        const bool active = j < n;
        const int64_t jnext = j + stride;
        int64_t nb = 0, ne = 0;
        if (jnext < n) { nb = rp[jnext]; ne = rp[jnext + 1]; }
        double acc = 0.0;
        if (active) acc = G == 32 ? row_dot_pairs(col, val, x, pb, pe, sub, G) : row_dot(col, val, x, pb, pe, sub, G);
        acc = group_sum(acc, G);
        if (active && sub == 0) y[j] = acc * scale;
        j = jnext; pb = nb; pe = ne;
    }
}

// Lanes per row from the mean row length: two half-warp rows at a time up to ~500
// nonzeros (more rows in flight per warp), a whole warp with paired loads beyond.
__global__ void __launch_bounds__(kSpThreads)
k_residual(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const double* __restrict__ val,
           int64_t m, const double* __restrict__ x, const double* __restrict__ b, double* y) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * kSpThreads) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * kSpThreads + threadIdx.x) >> 5; i < m; i += nw) {
        double acc = group_sum(row_dot(col, val, x, rp[i], rp[i + 1], lane, 32), 32);
        if (lane == 0) y[i] = b[i] - acc;
    }
}

int launch_residual(const csls_csr* A, const double* x, const double* b, double* y, cudaStream_t s) {
    int64_t g = ceil_div(A->m * 32, kSpThreads);
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    k_residual<<<(int)(g < 1 ? 1 : g), kSpThreads, 0, s>>>(A->row_ptr, A->col, A->val, A->m, x, b, y);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

static int pick_group(int64_t nnz, int64_t rows) {
    const double avg = rows > 0 ? (double)nnz / (double)rows : 0.0;
    if (avg >= 512) return 32;
    if (avg >= 20) return 16;
    if (avg >= 8) return 8;
    return 4;
}

int spmv_grid(const csls_csr* A) {
    const int G = pick_group(A->nnz, A->m);
    int64_t g = ceil_div(A->m * (int64_t)G, kSpThreads);
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

int launch_spmv(const csls_csr* A, int mode, const double* x, double* y, LsqrState* st, double* partials, int grid,
                cudaStream_t s) {
    const int G = pick_group(A->nnz, A->m);
#define CSLS_SP(GG)                                                                                              \
    do {                                                                                                         \
        if (mode == 0) k_spmv<GG, 0><<<grid, kSpThreads, 0, s>>>(A->row_ptr, A->col, A->val, A->m, x, y, st, partials); \
        else if (mode == 1) k_spmv<GG, 1><<<grid, kSpThreads, 0, s>>>(A->row_ptr, A->col, A->val, A->m, x, y, st, partials); \
        else k_spmv<GG, 2><<<grid, kSpThreads, 0, s>>>(A->row_ptr, A->col, A->val, A->m, x, y, st, partials); \
    } while (0)
    switch (G) {
        case 32: CSLS_SP(32); break;
        case 16: CSLS_SP(16); break;
        case 8: CSLS_SP(8); break;
        default: CSLS_SP(4); break;
    }
#undef CSLS_SP
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

int launch_spmv_t(const Transpose& AT, int64_t n, int64_t m, int64_t nnz, int mode, const double* x, double* y,
                  LsqrState* st, cudaStream_t s) {
    (void)m;
    const int G = pick_group(nnz, n);
    int64_t g = ceil_div(n * (int64_t)G, kSpThreads);
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    const int grid = (int)(g < 1 ? 1 : g);
#define CSLS_SPT(GG)                                                                                        \
    do {                                                                                                    \
        if (mode == 0) k_spmv_t<GG, 0><<<grid, kSpThreads, 0, s>>>(AT.row_ptr, AT.col, AT.val, n, x, y, st); \
        else k_spmv_t<GG, 1><<<grid, kSpThreads, 0, s>>>(AT.row_ptr, AT.col, AT.val, n, x, y, st);           \
    } while (0)
    switch (G) {
        case 32: CSLS_SPT(32); break;
        case 16: CSLS_SPT(16); break;
        case 8: CSLS_SPT(8); break;
        default: CSLS_SPT(4); break;
    }
#undef CSLS_SPT
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

// ------------------------------------------------------------------ dense P (SVD variant)

// MODE 0: z = P v. MODE 1: z = P (vt / alpha), then the x / wx epilogue.
template <int MODE>
__global__ void __launch_bounds__(kSpThreads)
k_pgemv(const double* __restrict__ P, int64_t n, int64_t r, const double* v, double* z, LsqrState* st, double* wx,
        double* x) {
    __shared__ double coef[4];
    if (MODE == 1 && *(volatile int*)&st->done) return;
    if (threadIdx.x == 0) {
        coef[0] = MODE == 1 ? 1.0 / st->alpha : 1.0;
        if (MODE == 1) { coef[1] = st->cx; coef[2] = st->cw; coef[3] = (double)st->first; }
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t k = 0; k < r; ++k) acc += P[i + k * n] * v[k];
        acc *= coef[0];
        z[i] = acc;
        if (MODE == 1) xw_update(st, coef[3] != 0.0, coef[1], coef[2], acc, wx, x, i);
    }
    if (MODE == 1 && last_cta(&st->apply_cnt, gridDim.x) && threadIdx.x == 0) {
        st->first = 0;
        st->apply_cnt = 0;
    }
}

// MODE 0: y = P^T g. MODE 1: vt = P^T g - (beta/alpha) vt, alpha, scalar step. MODE 2: vt = P^T g, alpha_1.
template <int MODE>
__global__ void __launch_bounds__(kSpThreads)
k_pgemv_t(const double* __restrict__ P, int64_t n, int64_t r, const double* g, double* vt, double* out,
          LsqrState* st, double* partials, double* hist) {
    __shared__ double red[kSpThreads / 32];
    __shared__ double coef_s;
    const int tid = threadIdx.x, lane = tid & 31;
    if (MODE == 1 && *(volatile int*)&st->done) return;
    if (tid == 0) coef_s = MODE == 1 ? st->beta / st->alpha : 0.0;
    __syncthreads();
    double sq = 0.0;
    const int64_t warp_g = ((int64_t)blockIdx.x * kSpThreads + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kSpThreads) >> 5;
    for (int64_t k = warp_g; k < r; k += nwarps) {
        double acc = 0.0;
        for (int64_t i = lane; i < n; i += 32) acc += P[i + k * n] * g[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            if (MODE == 0) {
                out[k] = acc;
            } else {
                const double vn = MODE == 1 ? acc - coef_s * vt[k] : acc;
                vt[k] = vn;
                sq += vn * vn;
            }
        }
    }
    if (MODE == 0) return;
    if (lane == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kSpThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
    if (last_cta(&st->apply_cnt, gridDim.x) && tid == 0) {
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
        st->apply_cnt = 0;
    }
}

int launch_pgemv(const double* P, int64_t n, int64_t r, int mode, const double* v, double* z, LsqrState* st,
                 double* wx, double* x, cudaStream_t s) {
    int64_t g = ceil_div(n, kSpThreads);
    if (g < 1) g = 1;
    if (mode == 0) k_pgemv<0><<<(unsigned)g, kSpThreads, 0, s>>>(P, n, r, v, z, st, wx, x);
    else k_pgemv<1><<<(unsigned)g, kSpThreads, 0, s>>>(P, n, r, v, z, st, wx, x);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

int launch_pgemv_t(const double* P, int64_t n, int64_t r, int mode, const double* g, double* vt, double* out,
                   LsqrState* st, double* partials, double* hist, cudaStream_t s) {
    int64_t gr = ceil_div(r * 32, kSpThreads);
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (gr > cap) gr = cap;
    if (gr < 1) gr = 1;
    if (mode == 0) k_pgemv_t<0><<<(unsigned)gr, kSpThreads, 0, s>>>(P, n, r, g, vt, out, st, partials, hist);
    else if (mode == 1) k_pgemv_t<1><<<(unsigned)gr, kSpThreads, 0, s>>>(P, n, r, g, vt, out, st, partials, hist);
    else k_pgemv_t<2><<<(unsigned)gr, kSpThreads, 0, s>>>(P, n, r, g, vt, out, st, partials, hist);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

}  // namespace csls

// ------------------------------------------------------------------ streaming-read probe
//
// The HBM read ceiling that the SpMV pair (a read-dominated stream) is compared with. Each thread
// keeps U independent 16-byte loads in flight (evict-first) and folds them into a 64-bit integer
// checksum: an FP64 sum would itself be the limit on this part (two FP64 additions per 16 bytes
// per thread need more than the FP64 pipe's two operations per clock per SM at HBM rate).
namespace csls {

template <int U>
__global__ void __launch_bounds__(512) k_read_probe(const ulonglong2* __restrict__ p, int64_t n2,
                                                    const unsigned long long* __restrict__ tail, int has_tail,
                                                    unsigned long long* partials) {
    unsigned long long a0 = 0, a1 = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < n2; i += U * stride) {
        ulonglong2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldcs(p + i + u * stride);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a0 += v[u].x;
            a1 += v[u].y;
        }
    }
    for (; i < n2; i += stride) {
        const ulonglong2 v = __ldcs(p + i);
        a0 += v.x;
        a1 += v.y;
    }
    unsigned long long a = a0 + a1;
    if (has_tail && blockIdx.x == 0 && threadIdx.x == 0) a += *tail;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    __shared__ unsigned long long ws[16];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}

int launch_read_probe(const void* buf, int64_t count, int ctas_per_sm, int unroll, unsigned long long* partials,
                      cudaStream_t s) {
    const unsigned grid = (unsigned)(device_sm_count() * ctas_per_sm);
    const ulonglong2* p = (const ulonglong2*)buf;
    const int64_t n2 = count / 2;
    const unsigned long long* tail = (const unsigned long long*)buf + (count - 1);
    const int has_tail = (int)(count & 1);
    switch (unroll) {
        case 1: k_read_probe<1><<<grid, 512, 0, s>>>(p, n2, tail, has_tail, partials); break;
        case 2: k_read_probe<2><<<grid, 512, 0, s>>>(p, n2, tail, has_tail, partials); break;
        case 4: k_read_probe<4><<<grid, 512, 0, s>>>(p, n2, tail, has_tail, partials); break;
        default: k_read_probe<8><<<grid, 512, 0, s>>>(p, n2, tail, has_tail, partials); break;
    }
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

}  // namespace csls

// Batched LSQR over many independent problems of uneven size (one factor per
// instance), run as ONE CUDA-graph launch: the LSQR start is a few batched
// kernels, then a WHILE conditional node repeats one batched iteration
// (preconditioner solve, SpMV, transposed SpMV, transposed solve + scalar step)
// until every instance has converged or hit its limit; the loop condition is
// set on the device, so the host never polls between iterations.
//
// Each batched kernel covers all instances in one grid: a CTA finds its
// instance from a prefix table of per-instance CTA counts. Triangular solves keep
// their per-instance ticket and flag chains (a CTA only waits for CTAs of its own
// instance that started earlier) and SpMVs keep per-instance fixed-order reductions,
// so each instance is deterministic; its sums run in the order of its tuned SpMV
// thread group, so it matches the single-instance solve to rounding, not bit for bit.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lsqr.cuh"

namespace csls {

struct InstDesc {
    const int64_t* rp;
    const int32_t* col;
    const double* val;
    const int64_t* rpt;
    const int32_t* colt;
    const double* valt;
    const void* R;
    const double* Dinv;
    const double* b;
    double* x;
    double *ut, *vt, *z, *g, *wx, *sp_part, *lo_part, *hist;
    int *flags_up, *flags_lo;
    LsqrState* st;
    int64_t m, n;
    int nb, rprec, G, Gt;
};

struct BatchCtl {
    unsigned live;
    unsigned iter;
    unsigned limit;
    unsigned pad;
    double guard;       // cond guard for binary32 factors (0: off)
};

constexpr int kBatT = 256;

__device__ __forceinline__ int find_inst(const int* off, int count, int cta) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double group_sum_rt(double v, int G) {
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        if (o < G) v += w;
    }
    return v;
}

// MODE 2: ut = b, beta_1. MODE 1: ut = A z - (alpha/beta) ut, beta.
template <int MODE>
__global__ void __launch_bounds__(kBatT) k_bat_spmv(const InstDesc* inst, const int* off, int count) {
    __shared__ double red[kBatT / 32];
    __shared__ double coef_s;
    __shared__ int skip_s;
    const int ii = find_inst(off, count, blockIdx.x);
    const InstDesc& d = inst[ii];
    const int local = blockIdx.x - off[ii], ncta = off[ii + 1] - off[ii];
    LsqrState* st = d.st;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        skip_s = MODE == 1 && *(volatile int*)&st->done;
        coef_s = MODE == 1 ? st->alpha / st->beta : 0.0;
    }
    __syncthreads();
    if (skip_s) return;
    const int G = d.G, sub = lane & (G - 1), rows_per_warp = 32 / G;
    const int64_t warp_g = ((int64_t)local * kBatT + tid) >> 5;
    const int64_t nwarps = ((int64_t)ncta * kBatT) >> 5;
    double sq = 0.0;
    for (int64_t base = warp_g * rows_per_warp; base < d.m; base += nwarps * rows_per_warp) {
        const int64_t i = base + lane / G;
        const bool active = i < d.m;
        double acc = 0.0;
        if (MODE == 1 && active)
            acc = row_dot(d.col, d.val, d.z, d.rp[i], d.rp[i + 1], sub, G);
        if (MODE == 1) acc = group_sum_rt(acc, G);
        if (active && sub == 0) {
            const double un = MODE == 1 ? acc - coef_s * d.ut[i] : d.b[i];
            d.ut[i] = un;
            sq += un * un;
        }
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kBatT / 32; ++w) t += red[w];
        d.sp_part[local] = t;
    }
    if (last_cta(&st->spmv_cnt, (unsigned)ncta) && tid == 0) {
        const double beta = sqrt(sum_partials(d.sp_part, ncta));
        st->beta = beta;
        st->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(beta)) { set_error(&st->err, CSLS_ERR_NONFINITE); st->done = 1; }
        if (MODE == 2) {
            st->bnorm = beta;
            st->phibar = beta;
            st->rnorm = beta;
            if (beta == 0.0) { st->done = 1; st->istop = 3; }
        }
        st->spmv_cnt = 0;
    }
}

// g = A^T ut / beta
__global__ void __launch_bounds__(kBatT) k_bat_spmtv(const InstDesc* inst, const int* off, int count, int mode) {
    const int ii = find_inst(off, count, blockIdx.x);
    const InstDesc& d = inst[ii];
    const int local = blockIdx.x - off[ii], ncta = off[ii + 1] - off[ii];
    const LsqrState* st = d.st;
    if (mode == 1 && *(volatile const int*)&st->done) return;
    const double scale = st->inv_beta;
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = d.Gt, sub = lane & (G - 1), rows_per_warp = 32 / G;
    const int64_t warp_g = ((int64_t)local * kBatT + tid) >> 5;
    const int64_t nwarps = ((int64_t)ncta * kBatT) >> 5;
    for (int64_t base = warp_g * rows_per_warp; base < d.n; base += nwarps * rows_per_warp) {
        const int64_t j = base + lane / G;
        const bool active = j < d.n;
        double acc = 0.0;
        if (active)
            acc = row_dot(d.colt, d.valt, d.ut, d.rpt[j], d.rpt[j + 1], sub, G);
        acc = group_sum_rt(acc, G);
        if (active && sub == 0) d.g[j] = acc * scale;
    }
}

__device__ __forceinline__ void wait_flag_bat(const int* flag, int want, long long spin, int* err) {
    long long it = 0;
    while (ld_acquire(flag) != want) {
        if (++it > spin) { set_error(err, CSLS_ERR_TIMEOUT); return; }
        __nanosleep(32);
    }
}

template <class TR>
__device__ __forceinline__ double bat_upper_dot(const TR* R, int64_t n, int64_t row, int64_t c0, int q, int cs,
                                                const double* z) {
    double acc = 0.0;
    const TR* rp = R + row + (c0 + q * 16) * n;
    const double* zp = z + c0 + q * 16;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
        if (q * 16 + kk < cs) acc += (double)__ldg(rp + (int64_t)kk * n) * __ldcg(zp + kk);
    return acc;
}

template <class TR>
__device__ __forceinline__ double bat_lower_dot(const TR* R, int64_t n, int64_t colj, int64_t c0, int q,
                                                const double* g) {
    double acc = 0.0;
    const TR* rp = R + (c0 + q * 16) + colj * n;
    const double* gp = g + c0 + q * 16;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc += (double)__ldg(rp + kk) * __ldcg(gp + kk);
    return acc;
}

// z = R^{-1} (vt / alpha) with the x / wx epilogue, per instance.
__global__ void __launch_bounds__(kBatT) k_bat_trsv_upper(const InstDesc* inst, const int* off, int count,
                                                          long long spin, int* err) {
    __shared__ int sb_s, skip_s;
    __shared__ unsigned epoch_s;
    __shared__ double part[4][kTrsvBlock];
    __shared__ double rhs[kTrsvBlock];
    __shared__ double coef[4];
    const int ii = find_inst(off, count, blockIdx.x);
    const InstDesc& d = inst[ii];
    LsqrState* st = d.st;
    const int tid = threadIdx.x;
    if (tid == 0) {
        skip_s = *(volatile int*)&st->done;
        if (!skip_s) {
            epoch_s = *(volatile unsigned*)&st->up.epoch;
            sb_s = (int)atomicAdd(&st->up.ticket, 1u);
            coef[0] = 1.0 / st->alpha;
            coef[1] = st->cx;
            coef[2] = st->cw;
            coef[3] = (double)st->first;
        }
    }
    __syncthreads();
    if (skip_s) return;
    const int nb = d.nb, want = (int)(epoch_s + 1u);
    const int b = nb - 1 - sb_s;
    const int64_t n = d.n, r0 = (int64_t)b * kTrsvBlock;
    const int bs = (int)(n - r0 < kTrsvBlock ? n - r0 : kTrsvBlock);
    const int row = tid & (kTrsvBlock - 1), q = tid >> 6;
    double acc = 0.0;
    for (int c = nb - 1; c > b; --c) {
        const int64_t c0 = (int64_t)c * kTrsvBlock;
        const int cs = (int)(n - c0 < kTrsvBlock ? n - c0 : kTrsvBlock);
        if (tid == 0) wait_flag_bat(&d.flags_up[c], want, spin, err);
        __syncthreads();
        if (row < bs)
            acc += d.rprec == CSLS_PREC_F64 ? bat_upper_dot((const double*)d.R, n, r0 + row, c0, q, cs, d.z)
                                            : bat_upper_dot((const float*)d.R, n, r0 + row, c0, q, cs, d.z);
    }
    part[q][row] = acc;
    __syncthreads();
    if (tid < kTrsvBlock)
        rhs[tid] = tid < bs ? d.vt[r0 + tid] * coef[0] - (((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid])
                            : 0.0;
    __syncthreads();
    const double* D = d.Dinv + (int64_t)b * kTrsvBlock * kTrsvBlock;
    double a2 = 0.0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) a2 += D[row + (q * 16 + kk) * kTrsvBlock] * rhs[q * 16 + kk];
    part[q][row] = a2;
    __syncthreads();
    if (tid < bs) {
        const double zb = ((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid];
        d.z[r0 + tid] = zb;
        xw_update(st, coef[3] != 0.0, coef[1], coef[2], zb, d.wx, d.x, r0 + tid);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        st_release(&d.flags_up[b], want);
        if (atomicAdd(&st->up.done, 1u) == (unsigned)nb - 1) {
            st->up.ticket = 0;
            st->up.done = 0;
            st->first = 0;
            __threadfence();
            atomicAdd(&st->up.epoch, 1u);
        }
    }
}

// MODE 2: vt = R^{-T} g, alpha_1. MODE 1: vt = R^{-T} g - (beta/alpha) vt, alpha, scalar step.
template <int MODE>
__global__ void __launch_bounds__(kBatT) k_bat_trsv_lower(const InstDesc* inst, const int* off, int count,
                                                          BatchCtl* ctl, long long spin, int* err) {
    __shared__ int sb_s, skip_s;
    __shared__ unsigned epoch_s;
    __shared__ double part[4][kTrsvBlock];
    __shared__ double rhs[kTrsvBlock];
    __shared__ double coef_s;
    __shared__ double red[kBatT / 32];
    const int ii = find_inst(off, count, blockIdx.x);
    const InstDesc& d = inst[ii];
    LsqrState* st = d.st;
    const int tid = threadIdx.x;
    if (tid == 0) {
        skip_s = MODE == 1 && *(volatile int*)&st->done;
        if (!skip_s) {
            epoch_s = *(volatile unsigned*)&st->lo.epoch;
            sb_s = (int)atomicAdd(&st->lo.ticket, 1u);
            coef_s = MODE == 1 ? st->beta / st->alpha : 0.0;
        }
    }
    __syncthreads();
    if (skip_s) return;
    const int nb = d.nb, want = (int)(epoch_s + 1u);
    const int b = sb_s;
    const int64_t n = d.n, r0 = (int64_t)b * kTrsvBlock;
    const int bs = (int)(n - r0 < kTrsvBlock ? n - r0 : kTrsvBlock);
    const int colj = tid & (kTrsvBlock - 1), q = tid >> 6;
    double acc = 0.0;
    for (int c = 0; c < b; ++c) {
        const int64_t c0 = (int64_t)c * kTrsvBlock;
        if (tid == 0) wait_flag_bat(&d.flags_lo[c], want, spin, err);
        __syncthreads();
        if (colj < bs)
            acc += d.rprec == CSLS_PREC_F64 ? bat_lower_dot((const double*)d.R, n, r0 + colj, c0, q, d.g)
                                            : bat_lower_dot((const float*)d.R, n, r0 + colj, c0, q, d.g);
    }
    part[q][colj] = acc;
    __syncthreads();
    if (tid < kTrsvBlock)
        rhs[tid] = tid < bs ? d.g[r0 + tid] - (((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid]) : 0.0;
    __syncthreads();
    const double* D = d.Dinv + (int64_t)b * kTrsvBlock * kTrsvBlock;
    double a2 = 0.0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) a2 += D[(q * 16 + kk) + colj * kTrsvBlock] * rhs[q * 16 + kk];
    part[q][colj] = a2;
    __syncthreads();
    double sq = 0.0;
    if (tid < bs) {
        const double zb = ((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid];
        d.g[r0 + tid] = zb;
        const double vn = MODE == 1 ? zb - coef_s * d.vt[r0 + tid] : zb;
        d.vt[r0 + tid] = vn;
        sq = vn * vn;
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) red[tid >> 5] = sq;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kBatT / 32; ++w) t += red[w];
        d.lo_part[b] = t;
        __threadfence();
        st_release(&d.flags_lo[b], want);
        if (atomicAdd(&st->lo.done, 1u) == (unsigned)nb - 1) {
            __threadfence();
            const double alpha_new = sqrt(sum_partials(d.lo_part, nb));
            if (MODE == 1) {
                lsqr_scalar_step(st, alpha_new, d.hist);
            } else {
                st->alpha = alpha_new;
                st->rhobar = alpha_new;
                if (d.hist) d.hist[0] = alpha_new;
                if (alpha_new == 0.0 || !isfinite(alpha_new)) {
                    st->done = 1;
                    st->istop = 3;
                    if (!isfinite(alpha_new)) set_error(&st->err, CSLS_ERR_NONFINITE);
                }
            }
            st->lo.ticket = 0;
            st->lo.done = 0;
            __threadfence();
            atomicAdd(&st->lo.epoch, 1u);
        }
    }
}

// One CTA: count the iteration and the instances still running, apply the early cond
// guard to instances with a binary32 factor, and decide whether the WHILE node runs
// the body again.
__global__ void __launch_bounds__(kBatT) k_bat_cond(const InstDesc* inst, int count, BatchCtl* ctl,
                                                     cudaGraphConditionalHandle handle) {
    __shared__ unsigned live_s;
    if (threadIdx.x == 0) live_s = 0u;
    __syncthreads();
    const double guard = ctl->guard;
    unsigned live = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        LsqrState* st = inst[i].st;
        if (*(volatile int*)&st->done) continue;
        if (inst[i].rprec == CSLS_PREC_F32 && guard > 0.0 && st->fixed <= 0 && guard_checkpoint(st->iter) &&
            st->iter <= st->hist_cap && !(bidiag_cond_hist(inst[i].hist, st->iter) < guard)) {
            set_error(&st->err, CSLS_ERR_PRECOND_GUARD);
            st->done = 1;
            continue;
        }
        ++live;
    }
    atomicAdd(&live_s, live);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned it = ++ctl->iter;
        ctl->live = live_s;
        cudaGraphSetConditional(handle, (live_s > 0 && it < ctl->limit) ? 1u : 0u);
    }
}

__global__ void k_bat_finish(const InstDesc* inst, const int* off, int count) {
    const int ii = find_inst(off, count, blockIdx.x);
    const InstDesc& d = inst[ii];
    const int local = blockIdx.x - off[ii], ncta = off[ii + 1] - off[ii];
    if (d.st->iter <= 0) return;
    const double cx = d.st->cx;
    for (int64_t i = (int64_t)local * blockDim.x + threadIdx.x; i < d.n; i += (int64_t)ncta * blockDim.x)
        d.x[i] += cx * d.wx[i];
}

// ------------------------------------------------------------------ host side

struct BatchLayout {
    BatchCtl* ctl;
    InstDesc* desc;
    int *sp_off, *spt_off, *tr_off, *fin_off;
    int* err;
};

static void carve_inst(Carve& c, int64_t m, int64_t n, int64_t nb, int64_t ncta_sp, InstDesc& d) {
    d.st = c.take<LsqrState>(1);
    d.ut = c.take<double>((size_t)m);
    d.vt = c.take<double>((size_t)n);
    d.z = c.take<double>((size_t)n);
    d.g = c.take<double>((size_t)n);
    d.wx = c.take<double>((size_t)n);
    d.sp_part = c.take<double>((size_t)ncta_sp + 8);
    d.lo_part = c.take<double>((size_t)nb + 8);
    d.hist = c.take<double>((size_t)(2 * (n + 6)));
    d.flags_up = c.take<int>((size_t)nb);
    d.flags_lo = c.take<int>((size_t)nb);
}

static int spmv_ctas(int64_t rows, int G) {
    int64_t g = ceil_div(rows * (int64_t)G, kBatT);
    const int64_t cap = (int64_t)device_sm_count() * 2;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

static size_t batch_carve(Carve& c, int64_t count, const csls_factor_t* const* F, InstDesc* host_desc,
                          BatchLayout& L) {
    L.ctl = c.take<BatchCtl>(1);
    L.desc = c.take<InstDesc>((size_t)count);
    L.sp_off = c.take<int>((size_t)count + 1);
    L.spt_off = c.take<int>((size_t)count + 1);
    L.tr_off = c.take<int>((size_t)count + 1);
    L.fin_off = c.take<int>((size_t)count + 1);
    L.err = c.take<int>(1);
    for (int64_t i = 0; i < count; ++i) {
        InstDesc d{};
        const int G = F[i]->spmv_group > 0 ? F[i]->spmv_group : 8;
        carve_inst(c, F[i]->m, F[i]->n, F[i]->nblocks, spmv_ctas(F[i]->m, G), d);
        if (host_desc) host_desc[i] = d;
    }
    return c.off;
}

}  // namespace csls

using namespace csls;

extern "C" int csls_batch_solve_workspace(int64_t count, const csls_factor_t* const* factors, size_t* bytes) {
    if (count <= 0 || !factors || !bytes) return CSLS_ERR_ARG;
    for (int64_t i = 0; i < count; ++i)
        if (!factors[i] || factors[i]->variant != CSLS_VARIANT_QR) return CSLS_ERR_ARG;
    Carve c{nullptr, 0, 0, true};
    BatchLayout L;
    *bytes = batch_carve(c, count, factors, nullptr, L);
    return CSLS_OK;
}

extern "C" int csls_batch_solve(int64_t count, const csls_factor_t* const* F, const csls_csr* A,
                                const double* const* b, double* const* x, const csls_opts* o, void* work,
                                size_t work_bytes, csls_report* reps, csls_stream_t stream) {
    if (count <= 0 || !F || !A || !b || !x || !o || o->warm_start) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_batch_solve_workspace(count, F, &need));
    if (!work || work_bytes < need || ((uintptr_t)work & 255)) return CSLS_ERR_WORKSPACE;
    for (int64_t i = 0; i < count; ++i)
        if (A[i].m != F[i]->m || A[i].n != F[i]->n || A[i].nnz != F[i]->nnz || !b[i] || !x[i]) return CSLS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<InstDesc> desc((size_t)count);
    Carve c{(char*)work, 0, work_bytes, false};
    BatchLayout L;
    batch_carve(c, count, F, desc.data(), L);
    std::vector<int> sp_off((size_t)count + 1, 0), spt_off((size_t)count + 1, 0), tr_off((size_t)count + 1, 0),
        fin_off((size_t)count + 1, 0);
    int64_t maxit = 0;
    for (int64_t i = 0; i < count; ++i) {
        const csls_factor_t* f = F[i];
        InstDesc& d = desc[(size_t)i];
        d.rp = A[i].row_ptr; d.col = A[i].col; d.val = A[i].val;
        d.rpt = f->AT.row_ptr; d.colt = f->AT.col; d.valt = f->AT.val;
        d.R = f->R; d.Dinv = f->Dinv; d.rprec = f->prec; d.nb = (int)f->nblocks;
        d.b = b[i]; d.x = x[i]; d.m = f->m; d.n = f->n;
        d.G = f->spmv_group > 0 ? f->spmv_group : 8;
        d.Gt = f->spmv_group_t > 0 ? f->spmv_group_t : 32;
        sp_off[(size_t)i + 1] = sp_off[(size_t)i] + spmv_ctas(d.m, d.G);
        spt_off[(size_t)i + 1] = spt_off[(size_t)i] + spmv_ctas(d.n, d.Gt);
        tr_off[(size_t)i + 1] = tr_off[(size_t)i] + d.nb;
        fin_off[(size_t)i + 1] = fin_off[(size_t)i] + (int)std::min<int64_t>(ceil_div(d.n, 256), 64);
        maxit = std::max<int64_t>(maxit, o->fixed_iters > 0 ? o->fixed_iters : (o->maxit > 0 ? o->maxit : d.n));
        LsqrState h{};
        h.atol = o->atol;
        h.btol = o->btol;
        h.maxit = o->maxit > 0 ? o->maxit : d.n;
        h.fixed = o->fixed_iters;
        h.hist_cap = d.n + 4;
        h.cs2 = -1.0;
        h.first = 1;
        CSLS_CUDA(cudaMemcpyAsync(d.st, &h, sizeof(LsqrState), cudaMemcpyHostToDevice, st));
        CSLS_CUDA(cudaMemsetAsync(d.flags_up, 0, sizeof(int) * (size_t)d.nb, st));
        CSLS_CUDA(cudaMemsetAsync(d.flags_lo, 0, sizeof(int) * (size_t)d.nb, st));
        CSLS_CUDA(cudaMemsetAsync(d.x, 0, sizeof(double) * (size_t)d.n, st));
        CSLS_CUDA(cudaMemsetAsync(d.wx, 0, sizeof(double) * (size_t)d.n, st));
    }
    BatchCtl hc{0, 0, (unsigned)std::min<int64_t>(maxit, 0x7fffffff), 0, o->guard_cond};
    CSLS_CUDA(cudaMemcpyAsync(L.ctl, &hc, sizeof(BatchCtl), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemcpyAsync(L.desc, desc.data(), sizeof(InstDesc) * (size_t)count, cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemcpyAsync(L.sp_off, sp_off.data(), sizeof(int) * sp_off.size(), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemcpyAsync(L.spt_off, spt_off.data(), sizeof(int) * spt_off.size(), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemcpyAsync(L.tr_off, tr_off.data(), sizeof(int) * tr_off.size(), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemcpyAsync(L.fin_off, fin_off.data(), sizeof(int) * fin_off.size(), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int), st));
    const int n_inst = (int)count;
    const long long spin = o->spin_limit;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    // start: beta_1 u_1 = b, alpha_1 v_1 = R^{-T} A^T u_1
    k_bat_spmv<2><<<sp_off.back(), kBatT, 0, st>>>(L.desc, L.sp_off, n_inst);
    k_bat_spmtv<<<spt_off.back(), kBatT, 0, st>>>(L.desc, L.spt_off, n_inst, 0);
    k_bat_trsv_lower<2><<<tr_off.back(), kBatT, 0, st>>>(L.desc, L.tr_off, n_inst, L.ctl, spin, L.err);
    CSLS_CUDA(cudaGetLastError());
    // the iteration loop as one graph launch: a WHILE node over one batched iteration
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    int rc = CSLS_OK;
    do {
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) { rc = CSLS_ERR_CUDA; break; }
        cudaGraphConditionalHandle handle;
        if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            rc = CSLS_ERR_CUDA;
            break;
        }
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) { rc = CSLS_ERR_CUDA; break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { rc = CSLS_ERR_CUDA; break; }
        if (cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess) {
            rc = CSLS_ERR_CUDA;
            break;
        }
        k_bat_trsv_upper<<<tr_off.back(), kBatT, 0, cap>>>(L.desc, L.tr_off, n_inst, spin, L.err);
        k_bat_spmv<1><<<sp_off.back(), kBatT, 0, cap>>>(L.desc, L.sp_off, n_inst);
        k_bat_spmtv<<<spt_off.back(), kBatT, 0, cap>>>(L.desc, L.spt_off, n_inst, 1);
        k_bat_trsv_lower<1><<<tr_off.back(), kBatT, 0, cap>>>(L.desc, L.tr_off, n_inst, L.ctl, spin, L.err);
        k_bat_cond<<<1, kBatT, 0, cap>>>(L.desc, n_inst, L.ctl, handle);
        cudaGraph_t captured = nullptr;
        if (cudaStreamEndCapture(cap, &captured) != cudaSuccess) { rc = CSLS_ERR_CUDA; break; }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { rc = CSLS_ERR_CUDA; break; }
        if (cudaGraphLaunch(exec, st) != cudaSuccess) { rc = CSLS_ERR_CUDA; break; }
    } while (0);
    if (rc == CSLS_OK) {
        k_bat_finish<<<fin_off.back(), 256, 0, st>>>(L.desc, L.fin_off, n_inst);
        if (cudaGetLastError() != cudaSuccess) rc = CSLS_ERR_CUDA;
    }
    cudaEventRecord(e1, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == CSLS_OK) rc = CSLS_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (rc != CSLS_OK) return rc;
    int err = 0;
    BatchCtl out{};
    CSLS_CUDA(cudaMemcpy(&err, L.err, sizeof(int), cudaMemcpyDeviceToHost));
    CSLS_CUDA(cudaMemcpy(&out, L.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost));
    int status = err;
    for (int64_t i = 0; i < count; ++i) {
        LsqrState s{};
        CSLS_CUDA(cudaMemcpy(&s, desc[(size_t)i].st, sizeof(LsqrState), cudaMemcpyDeviceToHost));
        const long long kk = std::min<long long>(s.iter, s.hist_cap);
        std::vector<double> hh((size_t)(2 * (kk + 1) + 2));
        CSLS_CUDA(cudaMemcpy(hh.data(), desc[(size_t)i].hist, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost));
        const double cond = bidiag_cond_hist(hh.data(), kk);
        int inst_status = s.err;
        if (inst_status == CSLS_OK && F[i]->prec == CSLS_PREC_F32 && o->guard_cond > 0 && o->fixed_iters <= 0 &&
            kk > 0 && !(cond < o->guard_cond))
            inst_status = CSLS_ERR_PRECOND_GUARD;
        if (inst_status == CSLS_OK && o->fixed_iters <= 0 && s.istop == 0) inst_status = CSLS_ERR_NOT_CONVERGED;
        if (status == CSLS_OK) status = inst_status;
        if (reps) {
            csls_report& r = reps[i];
            std::memset(&r, 0, sizeof(r));
            r.status = inst_status;
            r.cond_est = cond;
            r.istop = s.istop;
            r.iterations = s.iter;
            r.s = F[i]->s;
            r.r = F[i]->r;
            r.bnorm = s.bnorm;
            r.rnorm = s.rnorm;
            r.arnorm = s.arnorm;
            r.anorm = std::sqrt(s.anorm2);
            r.ynorm = s.ynorm;
            r.ms_solve = ms;
            r.launches = 5 + 1;   // 4 start/finish kernels + one graph launch
        }
    }
    return status;
}

// ------------------------------------------------------------------ autotuner support

namespace csls {

template <int G>
__global__ void __launch_bounds__(kBatT) k_tune_spmv(const int64_t* rp, const int32_t* col, const double* val,
                                                     int64_t rows, const double* x, double* y) {
    const int lane = threadIdx.x & 31, sub = lane & (G - 1);
    const int64_t warp_g = ((int64_t)blockIdx.x * kBatT + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBatT) >> 5;
    for (int64_t base = warp_g * (32 / G); base < rows; base += nwarps * (32 / G)) {
        const int64_t i = base + lane / G;
        double acc = 0.0;
        if (i < rows)
            acc = row_dot(col, val, x, rp[i], rp[i + 1], sub, G);
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < rows && sub == 0) y[i] = acc;
    }
}

static int time_group(int G, const int64_t* rp, const int32_t* col, const double* val, int64_t rows, const double* x,
                      double* y, cudaStream_t st, float* ms_out) {
    const int grid = spmv_ctas(rows, G) * 4;
    auto launch = [&]() {
        switch (G) {
            case 4: k_tune_spmv<4><<<grid, kBatT, 0, st>>>(rp, col, val, rows, x, y); break;
            case 8: k_tune_spmv<8><<<grid, kBatT, 0, st>>>(rp, col, val, rows, x, y); break;
            case 16: k_tune_spmv<16><<<grid, kBatT, 0, st>>>(rp, col, val, rows, x, y); break;
            default: k_tune_spmv<32><<<grid, kBatT, 0, st>>>(rp, col, val, rows, x, y); break;
        }
    };
    cudaEvent_t a, b;
    CSLS_CUDA(cudaEventCreate(&a));
    CSLS_CUDA(cudaEventCreate(&b));
    launch();
    CSLS_CUDA(cudaEventRecord(a, st));
    for (int r = 0; r < 5; ++r) launch();
    CSLS_CUDA(cudaEventRecord(b, st));
    CSLS_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CSLS_CUDA(cudaGetLastError());
    *ms_out = ms / 5.f;
    return CSLS_OK;
}

}  // namespace csls

extern "C" int csls_autotune_spmv(csls_factor_t* F, const csls_csr* A, void* work, size_t work_bytes, int* group,
                                  int* group_t, float* ms, csls_stream_t stream) {
    if (!F || !A || A->m != F->m || A->n != F->n) return CSLS_ERR_ARG;
    const size_t need = sizeof(double) * (size_t)(2 * (F->m + F->n)) + 1024;
    if (!work || work_bytes < need || ((uintptr_t)work & 255)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    double* xm = (double*)work;                 // length m (input of A^T u)
    double* xn = xm + F->m;                     // length n (input of A z)
    double* ym = xn + F->n;
    double* yn = ym + F->m;
    CSLS_CUDA(cudaMemsetAsync(work, 0, need - 1024, st));
    const int cand[4] = {4, 8, 16, 32};
    float best = 1e30f, best_t = 1e30f;
    int bg = 8, bgt = 32;
    for (int G : cand) {
        float t = 0.f;
        CSLS_TRY(time_group(G, A->row_ptr, A->col, A->val, A->m, xn, ym, st, &t));
        if (t < best) { best = t; bg = G; }
        CSLS_TRY(time_group(G, F->AT.row_ptr, F->AT.col, F->AT.val, F->n, xm, yn, st, &t));
        if (t < best_t) { best_t = t; bgt = G; }
    }
    F->spmv_group = bg;
    F->spmv_group_t = bgt;
    if (group) *group = bg;
    if (group_t) *group_t = bgt;
    if (ms) { ms[0] = best; ms[1] = best_t; }
    return CSLS_OK;
}

extern "C" int csls_factor_set_spmv_groups(csls_factor_t* F, int group, int group_t) {
    auto ok = [](int g) { return g == 4 || g == 8 || g == 16 || g == 32; };
    if (!F || !ok(group) || !ok(group_t)) return CSLS_ERR_ARG;
    F->spmv_group = group;
    F->spmv_group_t = group_t;
    return CSLS_OK;
}

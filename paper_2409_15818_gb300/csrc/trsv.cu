// Blocked triangular solves with R (the per-step preconditioner of the implicit
// form, Remark after Algorithm 2), one kernel per solve.
//
// R is cut into 64 x 64 blocks. One CTA owns one block row (upper solve) or
// block column (transposed solve); CTAs take block indices from an atomic
// ticket in launch order, so a CTA only ever waits for blocks owned by CTAs that
// started before it and the chain always progresses. Finished blocks are
// published with a release store of the launch epoch into a per-block flag;
// consumers acquire it with a bounded spin. The diagonal blocks are applied
// through their precomputed inverses, so both the solve with R and the one with
// R^T apply the same fixed operator and its exact transpose.
#include "lsqr.cuh"

namespace csls {

constexpr int kTs = kTrsvBlock;   // 64
constexpr int kTsThreads = 256;   // 4 threads per row / column

// Polls a block flag (one lane per warp; the warp then reads the block's entries). The first polls
// do not sleep: a flag on the chain is usually set within a few microseconds.
__device__ __forceinline__ bool wait_flag(const int* flag, int want, long long spin, int* err) {
    long long it = 0;
    while (ld_acquire(flag) != want) {
        if (++it > spin) {
            set_error(err, CSLS_ERR_TIMEOUT);
            return false;
        }
        if (it > 512) __nanosleep(32);
    }
    return true;
}

template <class TR>
__device__ __forceinline__ double ldr(const TR* p) { return (double)__ldg(p); }

// z = R^{-1} v  (MODE 0)   |   z = R^{-1} (vt / alpha) with the x / wx epilogue (MODE 1)
template <class TR, int MODE>
__global__ void __launch_bounds__(kTsThreads)
k_trsv_upper(const TR* __restrict__ R, int64_t n, int nb, const double* __restrict__ Dinv, const double* v,
             double* z, int* flags, TrsvCtl* ctl, LsqrState* st, double* wx, double* x, long long spin, int* err) {
    __shared__ int sb_s;
    __shared__ unsigned epoch_s;
    __shared__ double part[4][kTs];
    __shared__ double rhs[kTs];
    __shared__ double coef[4];
    __shared__ double dsm[kTs * kTs];   // this block's diagonal inverse (32 KB)
    const int tid = threadIdx.x;
    if (MODE == 1 && *(volatile int*)&st->done) return;
    if (tid == 0) {
        epoch_s = *(volatile unsigned*)&ctl->epoch;
        sb_s = (int)atomicAdd(&ctl->ticket, 1u);
        if (MODE == 1) {
            coef[0] = 1.0 / st->alpha;
            coef[1] = st->cx;
            coef[2] = st->cw;
            coef[3] = (double)st->first;
        } else {
            coef[0] = 1.0;
        }
    }
    __syncthreads();
    const int want = (int)(epoch_s + 1u);
    const int b = nb - 1 - sb_s;
    const int64_t r0 = (int64_t)b * kTs;
    const int bs = (int)(n - r0 < kTs ? n - r0 : kTs);
    const int row = tid & (kTs - 1), q = tid >> 6;
    // The diagonal-block inverse and each off-diagonal block of R are loaded before the flag
    // that releases them is awaited: once block c's solution is published, only its 64 z
    // entries are still to be fetched, so the chain from block to block carries no R traffic.
    const double* D = Dinv + (int64_t)b * kTs * kTs;
    for (int i = tid; i < kTs * kTs; i += kTsThreads) dsm[i] = __ldg(D + i);
    const double vpre = (tid < bs) ? v[r0 + tid] * coef[0] : 0.0;   // this block's right-hand side
    double rv[16];
    auto load_block = [&](int c, double (&dst)[16]) {
        const int64_t c0 = (int64_t)c * kTs;
        const int cs = (int)(n - c0 < kTs ? n - c0 : kTs);
        const TR* rp = R + (r0 + row) + (c0 + q * 16) * n;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) dst[kk] = (row < bs && q * 16 + kk < cs) ? ldr(rp + (int64_t)kk * n) : 0.0;
    };
    if (b < nb - 1) load_block(nb - 1, rv);
    double acc = 0.0;
    for (int c = nb - 1; c > b; --c) {
        const int64_t c0 = (int64_t)c * kTs;
        const int cs = (int)(n - c0 < kTs ? n - c0 : kTs);
        if ((tid & 31) == 0) wait_flag(&flags[c], want, spin, err);
        __syncwarp();
        double zv[16];
        const double* zp = z + c0 + q * 16;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) zv[kk] = q * 16 + kk < cs ? __ldcg(zp + kk) : 0.0;
        double rn[16];
        if (c - 1 > b) load_block(c - 1, rn);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fma(rv[kk], zv[kk], acc);
        if (c - 1 > b) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) rv[kk] = rn[kk];
        }
    }
    part[q][row] = acc;
    __syncthreads();
    if (tid < kTs) {
        double r = 0.0;
        if (tid < bs) r = vpre - (((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid]);
        rhs[tid] = r;
    }
    __syncthreads();
    double a2 = 0.0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = q * 16 + kk;
        a2 += dsm[row + k * kTs] * rhs[k];
    }
    part[q][row] = a2;
    __syncthreads();
    if (tid >= 32) return;
    // warp 0 finishes the block: rows lane and lane + 32, then publishes it (one warp, so no
    // CTA-wide barrier sits between the last product and the flag)
    const int lane = tid;
    double zb[2] = {0.0, 0.0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < bs) {
            zb[h] = ((part[0][i] + part[1][i]) + part[2][i]) + part[3][i];
            z[r0 + i] = zb[h];
        }
    }
    __threadfence();
    __syncwarp();
    // publish this block first: the x / w epilogue below touches only this block's rows
    if (lane == 0) st_release(&flags[b], want);
    if (MODE == 1)
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < bs) xw_update(st, coef[3] != 0.0, coef[1], coef[2], zb[h], wx, x, r0 + lane + 32 * h);
    if (lane == 0) {
        unsigned prev = atomicAdd(&ctl->done, 1u);
        if (prev == (unsigned)nb - 1) {
            ctl->ticket = 0;
            ctl->done = 0;
            if (MODE == 1) st->first = 0;
            __threadfence();
            atomicAdd(&ctl->epoch, 1u);
        }
    }
}

// MODE 0: out = R^{-T} g.  MODE 1: vt = R^{-T} g - (beta/alpha) vt, then alpha and the scalar step.
// MODE 2: vt = R^{-T} g, alpha_1 and the LSQR start values.
// The solve runs in place in g (block b's entries of g are read only by block b before
// being replaced by the solution, which later blocks then read).
template <class TR, int MODE>
__global__ void __launch_bounds__(kTsThreads)
k_trsv_lower(const TR* __restrict__ R, int64_t n, int nb, const double* __restrict__ Dinv, double* g, double* vt,
             double* out, int* flags, TrsvCtl* ctl, LsqrState* st, double* partials, double* hist, long long spin,
             int* err) {
    __shared__ int sb_s;
    __shared__ unsigned epoch_s;
    __shared__ double part[4][kTs];
    __shared__ double rhs[kTs];
    __shared__ double coef[2];
    __shared__ double dsm[kTs * kTs];   // this block's diagonal inverse (32 KB)
    const int tid = threadIdx.x;
    if (MODE == 1 && *(volatile int*)&st->done) return;
    if (tid == 0) {
        epoch_s = *(volatile unsigned*)&ctl->epoch;
        sb_s = (int)atomicAdd(&ctl->ticket, 1u);
        coef[0] = MODE == 1 ? st->beta / st->alpha : 0.0;
    }
    __syncthreads();
    const int want = (int)(epoch_s + 1u);
    const int b = sb_s;
    const int64_t r0 = (int64_t)b * kTs;
    const int bs = (int)(n - r0 < kTs ? n - r0 : kTs);
    const int col = tid & (kTs - 1), q = tid >> 6;
    // as in the upper solve: the diagonal inverse and the next block of R are loaded ahead of
    // the flag that releases them
    const double* D = Dinv + (int64_t)b * kTs * kTs;
    for (int i = tid; i < kTs * kTs; i += kTsThreads) dsm[i] = __ldg(D + i);
    // this block's own entries of g and v: read only by this CTA, so they are loaded up front
    const double gpre = (tid < bs) ? g[r0 + tid] : 0.0;
    // warp 0 finishes the block (rows lane and lane + 32): their previous vt entries, read up front
    double vtp[2] = {0.0, 0.0};
    if (MODE == 1 && tid < 32) {
        if (tid < bs) vtp[0] = vt[r0 + tid];
        if (tid + 32 < bs) vtp[1] = vt[r0 + tid + 32];
    }
    double rv[16];
    auto load_block = [&](int c, double (&dst)[16]) {
        const int64_t c0 = (int64_t)c * kTs;
        const TR* rp = R + (c0 + q * 16) + (r0 + col) * n;   // column r0+col, rows c0+q*16..+16
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) dst[kk] = col < bs ? ldr(rp + kk) : 0.0;
    };
    if (b > 0) load_block(0, rv);
    double acc = 0.0;
    for (int c = 0; c < b; ++c) {
        const int64_t c0 = (int64_t)c * kTs;
        if ((tid & 31) == 0) wait_flag(&flags[c], want, spin, err);
        __syncwarp();
        double zv[16];
        const double* zp = g + c0 + q * 16;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) zv[kk] = __ldcg(zp + kk);
        double rn[16];
        if (c + 1 < b) load_block(c + 1, rn);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fma(rv[kk], zv[kk], acc);
        if (c + 1 < b) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) rv[kk] = rn[kk];
        }
    }
    part[q][col] = acc;
    __syncthreads();
    if (tid < kTs) {
        double r = 0.0;
        if (tid < bs) r = gpre - (((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid]);
        rhs[tid] = r;
    }
    __syncthreads();
    double a2 = 0.0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = q * 16 + kk;
        a2 += dsm[k + col * kTs] * rhs[k];   // (D^T rhs)_col
    }
    part[q][col] = a2;
    __syncthreads();
    if (tid >= 32) return;
    // warp 0 finishes the block (rows lane and lane + 32) and publishes it
    const int lane = tid;
    double zb[2] = {0.0, 0.0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < bs) {
            zb[h] = ((part[0][i] + part[1][i]) + part[2][i]) + part[3][i];
            g[r0 + i] = zb[h];
        }
    }
    __threadfence();
    __syncwarp();
    // publish this block first: the epilogue below touches only this block's rows
    if (lane == 0) st_release(&flags[b], want);
    double sq = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < bs) {
            if (MODE == 0) {
                if (out != g) out[r0 + i] = zb[h];
            } else {
                const double vn = MODE == 1 ? zb[h] - coef[0] * vtp[h] : zb[h];
                vt[r0 + i] = vn;
                sq += vn * vn;
            }
        }
    }
    if (MODE != 0)
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        if (MODE != 0) {
            partials[b] = sq;
            __threadfence();
        }
        unsigned prev = atomicAdd(&ctl->done, 1u);
        if (prev == (unsigned)nb - 1) {
            __threadfence();
            if (MODE != 0) {
                const double alpha_new = sqrt(sum_partials(partials, nb));
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
            ctl->ticket = 0;
            ctl->done = 0;
            __threadfence();
            atomicAdd(&ctl->epoch, 1u);
        }
    }
}

int launch_trsv_upper(const TrsvArgs& a, int mode, const double* v, double* z, int* flags, TrsvCtl* ctl,
                      LsqrState* st, double* wx, double* x, long long spin, int* err, cudaStream_t s) {
    if (a.rprec == CSLS_PREC_F64 && a.pack_up && a.nb < 65536 && trsv_cluster_usable())
        return launch_trsv_cl_upper(a, mode, v, z, flags, ctl, st, wx, x, spin, err, s);
    dim3 grid((unsigned)a.nb), block(kTsThreads);
    if (a.rprec == CSLS_PREC_F64) {
        const double* R = (const double*)a.R;
        if (mode == 0) k_trsv_upper<double, 0><<<grid, block, 0, s>>>(R, a.n, a.nb, a.Dinv, v, z, flags, ctl, st, wx, x, spin, err);
        else k_trsv_upper<double, 1><<<grid, block, 0, s>>>(R, a.n, a.nb, a.Dinv, v, z, flags, ctl, st, wx, x, spin, err);
    } else {
        const float* R = (const float*)a.R;
        if (mode == 0) k_trsv_upper<float, 0><<<grid, block, 0, s>>>(R, a.n, a.nb, a.Dinv, v, z, flags, ctl, st, wx, x, spin, err);
        else k_trsv_upper<float, 1><<<grid, block, 0, s>>>(R, a.n, a.nb, a.Dinv, v, z, flags, ctl, st, wx, x, spin, err);
    }
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

int launch_trsv_lower(const TrsvArgs& a, int mode, double* g, double* vt, double* out, int* flags, TrsvCtl* ctl,
                      LsqrState* st, double* partials, double* hist, long long spin, int* err, cudaStream_t s) {
    if (a.rprec == CSLS_PREC_F64 && a.pack_lo && a.nb < 65536 && trsv_cluster_usable())
        return launch_trsv_cl_lower(a, mode, g, vt, out, flags, ctl, st, hist, spin, err, s);
    dim3 grid((unsigned)a.nb), block(kTsThreads);
#define CSLS_LOWER(TR, MD)                                                                                      \
    k_trsv_lower<TR, MD><<<grid, block, 0, s>>>((const TR*)a.R, a.n, a.nb, a.Dinv, g, vt, out, flags, ctl, st, \
                                                 partials, hist, spin, err)
    if (a.rprec == CSLS_PREC_F64) {
        if (mode == 0) CSLS_LOWER(double, 0);
        else if (mode == 1) CSLS_LOWER(double, 1);
        else CSLS_LOWER(double, 2);
    } else {
        if (mode == 0) CSLS_LOWER(float, 0);
        else if (mode == 1) CSLS_LOWER(float, 1);
        else CSLS_LOWER(float, 2);
    }
#undef CSLS_LOWER
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

}  // namespace csls

// Block form of the LSQR solve for many right-hand sides of one A: nrhs
// independent Paige-Saunders recurrences (one LsqrState per column) that share
// every pass over A, A^T and R. Vectors are stored row-major (n x W, W = nrhs
// rounded up to 8, padded columns start converged), so SpMM gathers one 8W-byte
// row per nonzero and the triangular solves become 64 x 64 by 64 x 8 block
// products. The triangular solves are chains of per-block steps (tickets, per-block
// flags with bounded waits) with 8 right-hand sides per CTA, so the chains of the
// column groups run side by side; the products of a step with older solutions are
// split off to worker CTAs in pieces of at least 32 steps (see blk_products).
#include <algorithm>
#include <cstring>
#include <vector>

#include "lsqr.cuh"

namespace csls {

constexpr int kBT = 256;       // threads
constexpr int kNR = 8;         // right-hand sides per triangular-solve CTA
constexpr int kTB = kTrsvBlock;
constexpr int kKQ = 4;        // quarters of a block's k range per triangular-solve CTA
constexpr int kKW = kTB / kKQ; // k entries of a quarter

struct BlockCtl {
    TrsvCtl up, lo;
    unsigned spmv_cnt, all_done, iter_launched, pad;
};

__device__ __forceinline__ bool col_live(const LsqrState* st, int c) { return !*(volatile const int*)&st[c].done; }

// ------------------------------------------------------------------ start: U = B (column-major in), beta_1

__global__ void __launch_bounds__(kBT) k_blk_start(const double* B, int64_t ldb, int64_t m, int nrhs, int W, double* U,
                                                   LsqrState* st, BlockCtl* ctl, double* partials) {
    extern __shared__ double red[];   // [kBT/32][W]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sq[2] = {0.0, 0.0};
    for (int64_t i = (blockIdx.x * (int64_t)kBT + threadIdx.x) >> 5; i < m; i += ((int64_t)gridDim.x * kBT) >> 5) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            if (c < W) {
                const double v = c < nrhs ? B[(int64_t)c * ldb + i] : 0.0;
                U[i * W + c] = v;
                sq[h] += v * v;
            }
        }
    }
    for (int h = 0; h < 2; ++h)
        if (lane + 32 * h < W) red[warp * W + lane + 32 * h] = sq[h];
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += kBT) {
        double t = 0.0;
        for (int w = 0; w < kBT / 32; ++w) t += red[w * W + c];
        partials[(int64_t)blockIdx.x * W + c] = t;
    }
    if (last_cta(&ctl->spmv_cnt, gridDim.x)) {
        for (int c = threadIdx.x; c < W; c += kBT) {
            double t = 0.0;
            for (unsigned q = 0; q < gridDim.x; ++q) t += __ldcg(partials + (int64_t)q * W + c);
            const double beta = sqrt(t);
            LsqrState* s = st + c;
            s->beta = beta;
            s->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
            s->bnorm = s->bnorm_ref > 0.0 ? s->bnorm_ref : beta;   // a restart keeps ||b|| in rule S1
            s->phibar = beta;
            s->rnorm = beta;
            if (!isfinite(beta)) { set_error(&s->err, CSLS_ERR_NONFINITE); s->done = 1; }
            if (beta == 0.0) { s->done = 1; s->istop = 3; }
        }
        if (threadIdx.x == 0) ctl->spmv_cnt = 0;
    }
}

// ------------------------------------------------------------------ U = A Z - (alpha/beta) U  (per column), beta

__global__ void __launch_bounds__(kBT) k_blk_spmm(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                  const double* __restrict__ val, int64_t m, int W,
                                                  const double* __restrict__ Z, double* U, LsqrState* st,
                                                  BlockCtl* ctl, double* partials) {
    extern __shared__ double red[];   // [kBT/32][W] then coef[W]
    double* coef = red + (kBT / 32) * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = threadIdx.x; c < W; c += kBT)
        coef[c] = col_live(st, c) ? st[c].alpha / st[c].beta : 0.0;
    __syncthreads();
    double sq[2] = {0.0, 0.0};
    for (int64_t i = (blockIdx.x * (int64_t)kBT + threadIdx.x) >> 5; i < m; i += ((int64_t)gridDim.x * kBT) >> 5) {
        double acc[2] = {0.0, 0.0};
        const int64_t pe = rp[i + 1];
        for (int64_t p = rp[i]; p < pe; ++p) {
            const double a = __ldg(val + p);
            const double* zr = Z + (int64_t)__ldg(col + p) * W;
            acc[0] += a * (lane < W ? zr[lane] : 0.0);
            if (lane + 32 < W) acc[1] += a * zr[lane + 32];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            if (c < W) {
                const double un = acc[h] - coef[c] * U[i * W + c];
                U[i * W + c] = un;
                sq[h] += un * un;
            }
        }
    }
    __syncthreads();
    for (int h = 0; h < 2; ++h)
        if (lane + 32 * h < W) red[warp * W + lane + 32 * h] = sq[h];
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += kBT) {
        double t = 0.0;
        for (int w = 0; w < kBT / 32; ++w) t += red[w * W + c];
        partials[(int64_t)blockIdx.x * W + c] = t;
    }
    if (last_cta(&ctl->spmv_cnt, gridDim.x)) {
        for (int c = threadIdx.x; c < W; c += kBT) {
            if (!col_live(st, c)) continue;
            double t = 0.0;
            for (unsigned q = 0; q < gridDim.x; ++q) t += __ldcg(partials + (int64_t)q * W + c);
            const double beta = sqrt(t);
            st[c].beta = beta;
            st[c].inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
            if (!isfinite(beta)) { set_error(&st[c].err, CSLS_ERR_NONFINITE); st[c].done = 1; }
        }
        if (threadIdx.x == 0) ctl->spmv_cnt = 0;
    }
}

// G = A^T U diag(1/beta)
__global__ void __launch_bounds__(kBT) k_blk_spmtm(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                   const double* __restrict__ val, int64_t n, int W,
                                                   const double* __restrict__ U, double* G, const LsqrState* st) {
    extern __shared__ double scale[];   // [W]
    const int lane = threadIdx.x & 31;
    for (int c = threadIdx.x; c < W; c += kBT) scale[c] = col_live(st, c) ? st[c].inv_beta : 0.0;
    __syncthreads();
    for (int64_t j = (blockIdx.x * (int64_t)kBT + threadIdx.x) >> 5; j < n; j += ((int64_t)gridDim.x * kBT) >> 5) {
        double acc[2] = {0.0, 0.0};
        const int64_t pe = rp[j + 1];
        for (int64_t p = rp[j]; p < pe; ++p) {
            const double a = __ldg(val + p);
            const double* ur = U + (int64_t)__ldg(col + p) * W;
            acc[0] += a * (lane < W ? ur[lane] : 0.0);
            if (lane + 32 < W) acc[1] += a * ur[lane + 32];
        }
        if (lane < W) G[j * W + lane] = acc[0] * scale[lane];
        if (lane + 32 < W) G[j * W + lane + 32] = acc[1] * scale[lane + 32];
    }
}

// ------------------------------------------------------------------ block triangular solves

__device__ __forceinline__ bool wait_flag_b(const int* flag, int want, long long spin, int* err) {
    long long it = 0;
    while (ld_acquire(flag) != want) {
        if (++it > spin) { set_error(err, CSLS_ERR_TIMEOUT); return false; }
        __nanosleep(32);
    }
    return true;
}

// Work split of a block solve. In solve order (upper: block nb - 1 - i is step i; transposed: block i),
// step i needs the products with the solutions of steps 0 .. i - 1, in pieces of kp steps: piece 0
// (steps i - kp .. i - 1, the newest ones) belongs to the step's own CTA, which then solves the block;
// piece p >= 1 (steps i - (p + 1) kp .. i - p kp - 1) to a worker CTA that publishes its 64 x 8 partial
// sum with a flag. CTAs take tickets in the order of a table built on the host, sorted by the last step
// each one needs (workers of a step before the step's own CTA), so every wait is on a CTA with an
// earlier ticket. Far products thus run as soon as their blocks exist instead of all in the CTA of the
// step, which held the last-solved block rows (the most work) to a few SMs at the end of the launch.
// Table entry: (i << 32) | (p << 8) | column group.
__device__ __forceinline__ int blk_pieces(int i, int kp) { return i > kp ? (i + kp - 1) / kp : 1; }

// acc (this thread's row and quarter, 8 columns) += the products with the solutions of steps [jlo, jhi):
// per block, the thread's 16 entries of R are loaded before the wait for that block's solution (they do
// not depend on it), the group's 64 x 8 solution block is staged in shared memory, and each entry of R
// meets all 8 columns (8 independent FMA chains).
template <bool UPPER, class TR>
__device__ __forceinline__ void blk_products(const TR* __restrict__ R, int64_t n, int nb, int jlo, int jhi, int64_t r0,
                                             int bs, const double* Y, int W, int c0g, const int* flags, int ngroups,
                                             int grp, int want, long long spin, int* err, double (*zs)[kNR],
                                             double (&acc)[kNR]) {
    const int tid = threadIdx.x, row = tid & (kTB - 1), kq = tid >> 6;
    const int zk = tid >> 1, zj = (tid & 1) * 4;   // staging: threads 0..127, 4 values each
    for (int j = jlo; j < jhi; ++j) {
        const int c = UPPER ? nb - 1 - j : j;
        const int64_t cc0 = (int64_t)c * kTB;
        const int cs = (int)(n - cc0 < kTB ? n - cc0 : kTB);
        double r[kKW];
        if (UPPER) {   // row r0 + row of R, columns cc0 + 16 kq ..: one strided load each
            const TR* rp = R + (r0 + row) + (cc0 + kq * kKW) * n;
#pragma unroll
            for (int kk = 0; kk < kKW; ++kk)
                r[kk] = (row < bs && kq * kKW + kk < cs) ? (double)__ldg(rp + (int64_t)kk * n) : 0.0;
        } else {       // column r0 + row of R, rows cc0 + 16 kq ..: contiguous (blocks before the last are full)
            const TR* rp = R + (cc0 + kq * kKW) + (r0 + row) * n;
            if (row < bs) {
                if (sizeof(TR) == 8 && (reinterpret_cast<uintptr_t>(rp) & 15) == 0) {
                    const double2* rp2 = reinterpret_cast<const double2*>(rp);
#pragma unroll
                    for (int kk = 0; kk < kKW; kk += 2) {
                        const double2 t = __ldg(rp2 + kk / 2);
                        r[kk] = t.x;
                        r[kk + 1] = t.y;
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < kKW; ++kk) r[kk] = (double)__ldg(rp + kk);
                }
            } else {
#pragma unroll
                for (int kk = 0; kk < kKW; ++kk) r[kk] = 0.0;
            }
        }
        if (tid == 0) wait_flag_b(&flags[(int64_t)c * ngroups + grp], want, spin, err);
        __syncthreads();   // the block is published, and every thread is done with the previous zs
        if (zk < kTB) {
            double2 a = make_double2(0.0, 0.0), e = make_double2(0.0, 0.0);
            if (zk < cs) {
                const double2* yp = reinterpret_cast<const double2*>(Y + (cc0 + zk) * W + c0g + zj);
                a = __ldcg(yp);
                e = __ldcg(yp + 1);
            }
            reinterpret_cast<double2*>(&zs[zk][zj])[0] = a;
            reinterpret_cast<double2*>(&zs[zk][zj])[1] = e;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKW; ++kk) {
            const double2* zr = reinterpret_cast<const double2*>(zs[kq * kKW + kk]);
#pragma unroll
            for (int q = 0; q < kNR / 2; ++q) {
                const double2 t = zr[q];
                acc[2 * q] = fma(r[kk], t.x, acc[2 * q]);
                acc[2 * q + 1] = fma(r[kk], t.y, acc[2 * q + 1]);
            }
        }
    }
}

// A worker's end: its quarters summed in order into its slot of wpart, then its flag.
__device__ __forceinline__ void blk_publish_piece(double (*part)[kTB][kNR + 1], double* slot, int* flag, int want) {
    const int tid = threadIdx.x, row = tid & (kTB - 1), cp = tid >> 6;
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int lc = 2 * cp + h;
        slot[row * kNR + lc] = ((part[0][row][lc] + part[1][row][lc]) + part[2][row][lc]) + part[3][row][lc];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(flag, want);
}

// The step's own CTA: the right-hand side's product sums of (row, lc), its own piece first, then the
// workers' pieces in order (the waits for them are done before).
__device__ __forceinline__ double blk_sum_pieces(double (*part)[kTB][kNR + 1], const double* slots, int64_t pstride,
                                                 int np, int row, int lc) {
    double s = ((part[0][row][lc] + part[1][row][lc]) + part[2][row][lc]) + part[3][row][lc];
    for (int p = 1; p < np; ++p) s += __ldcg(slots + p * pstride + row * kNR + lc);
    return s;
}

// Z = R^{-1} (V diag(1/alpha)) for the live columns, with the x / wx epilogue.
// Thread (row, kq) of a CTA owns row `row` of the block and the quarter kq of each 64-column block of R
// it multiplies; the four quarters are summed in a fixed order, and the diagonal-inverse product is
// split the same way.
template <class TR>
__global__ void __launch_bounds__(kBT)
k_blk_trsv_upper(const TR* __restrict__ R, int64_t n, int nb, int ngroups, const double* __restrict__ Dinv, int W,
                 const double* V, double* Z, double* WX, double* X, int* flags, const long long* tick, int kp,
                 int maxp, double* wpart, int* wflags, unsigned total, BlockCtl* ctl, LsqrState* st, long long spin,
                 int* err) {
    __shared__ int tk_s;
    __shared__ unsigned epoch_s;
    __shared__ __align__(16) double zs[kTB][kNR];   // the solution block being multiplied (group columns)
    __shared__ double part[kKQ][kTB][kNR + 1];       // per-quarter partial sums (padded rows: no bank conflicts)
    __shared__ __align__(16) double rhs[kTB][kNR];
    __shared__ double cf[kNR][4];   // 1/alpha, cx, cw, first (0 for converged columns)
    const int tid = threadIdx.x;
    if (tid == 0) {
        epoch_s = *(volatile unsigned*)&ctl->up.epoch;
        tk_s = (int)atomicAdd(&ctl->up.ticket, 1u);
    }
    __syncthreads();
    const long long code = tick[tk_s];
    const int i = (int)(code >> 32), p = (int)((code >> 8) & 0xFFFFFF), grp = (int)(code & 0xFF);
    const int b = nb - 1 - i;
    const int c0g = grp * kNR;
    if (p == 0 && tid < kNR) {
        const int c = c0g + tid;
        const bool live = col_live(st, c);
        cf[tid][0] = live ? 1.0 / st[c].alpha : 0.0;
        cf[tid][1] = st[c].cx;
        cf[tid][2] = st[c].cw;
        cf[tid][3] = live ? (double)st[c].first : -1.0;
    }
    const int want = (int)(epoch_s + 1u);
    const int64_t r0 = (int64_t)b * kTB;
    const int bs = (int)(n - r0 < kTB ? n - r0 : kTB);
    const int row = tid & (kTB - 1), kq = tid >> 6;
    double acc[kNR];
#pragma unroll
    for (int j = 0; j < kNR; ++j) acc[j] = 0.0;
    const int jlo = i - (p + 1) * kp > 0 ? i - (p + 1) * kp : 0, jhi = i - p * kp;
    blk_products<true>(R, n, nb, jlo, jhi, r0, bs, Z, W, c0g, flags, ngroups, grp, want, spin, err, zs, acc);
#pragma unroll
    for (int j = 0; j < kNR; ++j) part[kq][row][j] = acc[j];
    // the pieces' slots of this step and group: piece p at slots + p pstride
    const int64_t pstride = (int64_t)ngroups * kTB * kNR;
    double* const slots = wpart + ((int64_t)i * maxp * ngroups + grp) * ((int64_t)kTB * kNR);
    if (p > 0) {
        blk_publish_piece(part, slots + p * pstride, &wflags[((int64_t)i * maxp + p) * ngroups + grp], want);
    } else {
        // the diagonal inverse's entries of this thread, before the right-hand side is complete
        const double* D = Dinv + (int64_t)b * kTB * kTB;
        double d[kKW];
#pragma unroll
        for (int kk = 0; kk < kKW; ++kk) d[kk] = D[row + (kq * kKW + kk) * kTB];
        const int np = blk_pieces(i, kp);
        if (tid == 0)
            for (int q = 1; q < np; ++q) wait_flag_b(&wflags[((int64_t)i * maxp + q) * ngroups + grp], want, spin, err);
        __syncthreads();
        const int cp = kq;   // thread (row, cp) owns columns 2 cp, 2 cp + 1 from here on
        for (int h = 0; h < 2; ++h) {
            const int lc = 2 * cp + h;
            const double s = blk_sum_pieces(part, slots, pstride, np, row, lc);
            rhs[row][lc] = row < bs ? V[(r0 + row) * W + c0g + lc] * cf[lc][0] - s : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kNR; ++j) acc[j] = 0.0;
#pragma unroll
        for (int kk = 0; kk < kKW; ++kk) {
            const double2* rr = reinterpret_cast<const double2*>(rhs[kq * kKW + kk]);
#pragma unroll
            for (int j = 0; j < kNR / 2; ++j) {
                const double2 t = rr[j];
                acc[2 * j] = fma(d[kk], t.x, acc[2 * j]);
                acc[2 * j + 1] = fma(d[kk], t.y, acc[2 * j + 1]);
            }
        }
#pragma unroll
        for (int j = 0; j < kNR; ++j) part[kq][row][j] = acc[j];
        __syncthreads();
        if (row < bs) {
            const int64_t base = (r0 + row) * W + c0g + 2 * cp;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int lc = 2 * cp + h;
                const double zv = ((part[0][row][lc] + part[1][row][lc]) + part[2][row][lc]) + part[3][row][lc];
                Z[base + h] = zv;
                const double first = cf[lc][3];
                if (first < 0.0) continue;   // converged column: x and w stay as they are
                if (first != 0.0) {
                    WX[base + h] = zv;
                } else {
                    const double w = WX[base + h];
                    X[base + h] += cf[lc][1] * w;
                    WX[base + h] = zv - cf[lc][2] * w;
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(&flags[(int64_t)b * ngroups + grp], want);
    }
    if (tid == 0) {
        const unsigned prev = atomicAdd(&ctl->up.done, 1u);
        if (prev == total - 1) {
            for (int c = 0; c < W; ++c) st[c].first = 0;
            ctl->up.ticket = 0;
            ctl->up.done = 0;
            __threadfence();
            atomicAdd(&ctl->up.epoch, 1u);
        }
    }
}

// MODE 2 (start): V = R^{-T} G, alpha_1. MODE 1: V = R^{-T} G - (beta/alpha) V, alpha, scalar steps.
// The solve runs in place in G. Step i is block i; thread (colr, kq) owns column r0 + colr of R (row
// colr of the block of R^T) and the quarter kq of each 64-row block it multiplies.
template <class TR, int MODE>
__global__ void __launch_bounds__(kBT)
k_blk_trsv_lower(const TR* __restrict__ R, int64_t n, int nb, int ngroups, const double* __restrict__ Dinv, int W,
                 double* G, double* V, int* flags, const long long* tick, int kp, int maxp, double* wpart,
                 int* wflags, unsigned total, BlockCtl* ctl, LsqrState* st, double* partials, double* hist,
                 long long spin, int* err) {
    __shared__ int tk_s;
    __shared__ unsigned epoch_s;
    __shared__ __align__(16) double zs[kTB][kNR];
    __shared__ double part[kKQ][kTB][kNR + 1];
    __shared__ __align__(16) double rhs[kTB][kNR];
    __shared__ double coef[kNR];
    __shared__ double red[4][kNR];
    const int tid = threadIdx.x;
    if (tid == 0) {
        epoch_s = *(volatile unsigned*)&ctl->lo.epoch;
        tk_s = (int)atomicAdd(&ctl->lo.ticket, 1u);
    }
    __syncthreads();
    const long long code = tick[tk_s];
    const int i = (int)(code >> 32), p = (int)((code >> 8) & 0xFFFFFF), grp = (int)(code & 0xFF);
    const int b = i;
    const int c0g = grp * kNR;
    if (p == 0 && tid < kNR) {
        const int c = c0g + tid;
        coef[tid] = (MODE == 1 && col_live(st, c)) ? st[c].beta / st[c].alpha : 0.0;
    }
    const int want = (int)(epoch_s + 1u);
    const int64_t r0 = (int64_t)b * kTB;
    const int bs = (int)(n - r0 < kTB ? n - r0 : kTB);
    const int colr = tid & (kTB - 1), kq = tid >> 6;
    double acc[kNR];
#pragma unroll
    for (int j = 0; j < kNR; ++j) acc[j] = 0.0;
    const int jlo = i - (p + 1) * kp > 0 ? i - (p + 1) * kp : 0, jhi = i - p * kp;
    blk_products<false>(R, n, nb, jlo, jhi, r0, bs, G, W, c0g, flags, ngroups, grp, want, spin, err, zs, acc);
#pragma unroll
    for (int j = 0; j < kNR; ++j) part[kq][colr][j] = acc[j];
    const int64_t pstride = (int64_t)ngroups * kTB * kNR;
    double* const slots = wpart + ((int64_t)i * maxp * ngroups + grp) * ((int64_t)kTB * kNR);
    if (p > 0) {
        blk_publish_piece(part, slots + p * pstride, &wflags[((int64_t)i * maxp + p) * ngroups + grp], want);
    } else {
        // D^T: this thread's 16 contiguous entries of column colr of the diagonal inverse
        const double2* D2 = reinterpret_cast<const double2*>(Dinv + (int64_t)b * kTB * kTB + colr * kTB + kq * kKW);
        double d[kKW];
#pragma unroll
        for (int kk = 0; kk < kKW; kk += 2) {
            const double2 t = D2[kk / 2];
            d[kk] = t.x;
            d[kk + 1] = t.y;
        }
        const int np = blk_pieces(i, kp);
        if (tid == 0)
            for (int q = 1; q < np; ++q) wait_flag_b(&wflags[((int64_t)i * maxp + q) * ngroups + grp], want, spin, err);
        __syncthreads();
        const int cp = kq;   // thread (colr, cp) owns columns 2 cp, 2 cp + 1 from here on
        for (int h = 0; h < 2; ++h) {
            const int lc = 2 * cp + h;
            const double s = blk_sum_pieces(part, slots, pstride, np, colr, lc);
            rhs[colr][lc] = colr < bs ? G[(r0 + colr) * W + c0g + lc] - s : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kNR; ++j) acc[j] = 0.0;
#pragma unroll
        for (int kk = 0; kk < kKW; ++kk) {
            const double2* rr = reinterpret_cast<const double2*>(rhs[kq * kKW + kk]);
#pragma unroll
            for (int j = 0; j < kNR / 2; ++j) {
                const double2 t = rr[j];
                acc[2 * j] = fma(d[kk], t.x, acc[2 * j]);
                acc[2 * j + 1] = fma(d[kk], t.y, acc[2 * j + 1]);
            }
        }
#pragma unroll
        for (int j = 0; j < kNR; ++j) part[kq][colr][j] = acc[j];
        __syncthreads();
        double sq0 = 0.0, sq1 = 0.0;
        if (colr < bs) {
            const int64_t base = (r0 + colr) * W + c0g + 2 * cp;
            const double z0 =
                ((part[0][colr][2 * cp] + part[1][colr][2 * cp]) + part[2][colr][2 * cp]) + part[3][colr][2 * cp];
            const double z1 = ((part[0][colr][2 * cp + 1] + part[1][colr][2 * cp + 1]) + part[2][colr][2 * cp + 1]) +
                              part[3][colr][2 * cp + 1];
            G[base] = z0;
            G[base + 1] = z1;
            const double v0 = MODE == 1 ? z0 - coef[2 * cp] * V[base] : z0;
            const double v1 = MODE == 1 ? z1 - coef[2 * cp + 1] * V[base + 1] : z1;
            V[base] = v0;
            V[base + 1] = v1;
            sq0 = v0 * v0;
            sq1 = v1 * v1;
        }
        // per-column sums over the block's 64 rows: reduce inside the 64-thread group of each column pair
        for (int o = 16; o > 0; o >>= 1) {
            sq0 += __shfl_xor_sync(0xffffffffu, sq0, o);
            sq1 += __shfl_xor_sync(0xffffffffu, sq1, o);
        }
        __shared__ double wred[kBT / 32][2];
        if ((tid & 31) == 0) { wred[tid >> 5][0] = sq0; wred[tid >> 5][1] = sq1; }
        __syncthreads();
        if (tid < 4) {   // column pair tid: warps 2 tid, 2 tid + 1
            red[tid][0] = wred[2 * tid][0] + wred[2 * tid + 1][0];
            red[tid][1] = wred[2 * tid][1] + wred[2 * tid + 1][1];
            partials[(int64_t)b * W + c0g + 2 * tid] = red[tid][0];
            partials[(int64_t)b * W + c0g + 2 * tid + 1] = red[tid][1];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(&flags[(int64_t)b * ngroups + grp], want);
    }
    if (last_cta(&ctl->lo.done, total)) {
        // one thread per column: reduce its partials in block order, then its scalar step
        int live = 0;
        for (int c = tid; c < W; c += kBT) {
            if (!col_live(st, c)) continue;
            double t = 0.0;
            for (int q = 0; q < nb; ++q) t += __ldcg(partials + (int64_t)q * W + c);
            const double alpha_new = sqrt(t);
            if (MODE == 1) {
                lsqr_scalar_step(st + c, alpha_new, c == 0 ? hist : nullptr);
            } else {
                st[c].alpha = alpha_new;
                st[c].rhobar = alpha_new;
                if (c == 0 && hist) hist[0] = alpha_new;
                if (alpha_new == 0.0 || !isfinite(alpha_new)) {
                    st[c].done = 1;
                    st[c].istop = 3;
                    if (!isfinite(alpha_new)) set_error(&st[c].err, CSLS_ERR_NONFINITE);
                }
            }
            live += st[c].done ? 0 : 1;
        }
        const int nlive = __syncthreads_count(live > 0);
        if (tid == 0) {
            ctl->all_done = nlive == 0;
            ctl->lo.ticket = 0;
            ctl->lo.done = 0;
            __threadfence();
            atomicAdd(&ctl->lo.epoch, 1u);
        }
    }
}

// x_c += cx_c wx_c for the columns that ran at least one iteration; write x (column-major, ldx).
__global__ void k_blk_finish(const double* X, const double* WX, int64_t n, int W, int nrhs, const LsqrState* st,
                             double* x, int64_t ldx) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nrhs;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / n);
        const int64_t i = idx % n;
        double v = X[i * W + c];
        if (st[c].iter > 0) v += st[c].cx * WX[i * W + c];
        x[(int64_t)c * ldx + i] = v;
    }
}

// ------------------------------------------------------------------ host driver

struct BlockWs {
    BlockCtl* ctl;
    LsqrState* st;
    double *U, *V, *Z, *G, *WX, *X, *sp_part, *lo_part, *hist, *wpart;
    int *flags_up, *flags_lo, *wflags_up, *wflags_lo, *err;
    long long* tick;
    int64_t hist_cap, ntick;
    int W, kp, maxp;
};

// Steps a piece of a block solve covers: at least 32, and at most 8 pieces a step.
static int block_piece_steps(int64_t nb) { return (int)std::max<int64_t>(32, ceil_div(nb, 8)); }
static int block_pieces_host(int64_t i, int kp) { return i > kp ? (int)ceil_div(i, kp) : 1; }

// The ticket table of a block solve (see blk_products): every (step, piece, group), sorted by the last
// step it needs, a worker piece before the step's own CTA.
static std::vector<long long> block_tickets(int64_t nb, int ngroups, int kp) {
    struct E { int64_t key; int64_t i; int p; };
    std::vector<E> es;
    for (int64_t i = 0; i < nb; ++i) {
        const int np = block_pieces_host(i, kp);
        for (int p = 0; p < np; ++p) es.push_back({p == 0 ? 2 * i + 1 : 2 * (i - (int64_t)p * kp), i, p});
    }
    std::stable_sort(es.begin(), es.end(), [](const E& x, const E& y) { return x.key < y.key; });
    std::vector<long long> out;
    out.reserve(es.size() * (size_t)ngroups);
    for (const E& e : es)
        for (int g = 0; g < ngroups; ++g) out.push_back(((long long)e.i << 32) | ((long long)e.p << 8) | g);
    return out;
}

static BlockWs block_carve(Carve& c, int64_t m, int64_t n, int64_t nb, int64_t nrhs) {
    BlockWs w;
    w.W = (int)round_up(nrhs, kNR);
    const int64_t W = w.W;
    w.ctl = c.take<BlockCtl>(1);
    w.st = c.take<LsqrState>((size_t)W);
    w.U = c.take<double>((size_t)(m * W));
    w.V = c.take<double>((size_t)(n * W));
    w.Z = c.take<double>((size_t)(n * W));
    w.G = c.take<double>((size_t)(n * W));
    w.WX = c.take<double>((size_t)(n * W));
    w.X = c.take<double>((size_t)(n * W));
    w.sp_part = c.take<double>((size_t)((int64_t)device_sm_count() * 8 * W + 64));
    w.lo_part = c.take<double>((size_t)(nb * W + 64));
    w.hist_cap = n + 4;
    w.hist = c.take<double>((size_t)(2 * (w.hist_cap + 2)));
    w.flags_up = c.take<int>((size_t)(nb * (W / kNR)));
    w.flags_lo = c.take<int>((size_t)(nb * (W / kNR)));
    w.err = c.take<int>(1);
    w.kp = block_piece_steps(nb);
    w.maxp = block_pieces_host(nb - 1, w.kp);
    int64_t pieces = 0;
    for (int64_t i = 0; i < nb; ++i) pieces += block_pieces_host(i, w.kp);
    w.ntick = pieces * (W / kNR);
    w.tick = c.take<long long>((size_t)w.ntick);
    w.wpart = c.take<double>((size_t)(nb * w.maxp * (W / kNR) * kTB * kNR));
    w.wflags_up = c.take<int>((size_t)(nb * w.maxp * (W / kNR)));
    w.wflags_lo = c.take<int>((size_t)(nb * w.maxp * (W / kNR)));
    return w;
}

size_t block_ws_bytes(int64_t m, int64_t n, int64_t nb, int64_t nrhs) {
    Carve c{nullptr, 0, 0, true};
    block_carve(c, m, n, nb, nrhs);
    return c.off;
}

// scratch of a block restart, after the block solve's own workspace: the residuals (m x nrhs) and the
// corrections (n x nrhs)
size_t block_refine_bytes(int64_t m, int64_t n, int64_t nrhs) {
    Carve c{nullptr, 0, 0, true};
    c.take<double>((size_t)(m * nrhs));
    c.take<double>((size_t)(n * nrhs));
    return c.off;
}

__global__ void k_add_cols(double* x, int64_t ldx, const double* dx, int64_t n, int nrhs) {
    const int64_t total = n * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / n, i = e - k * n;
        x[i + k * ldx] += dx[e];
    }
}

// bref (host, nrhs or NULL): the norms of the original right-hand sides when b holds a restart's residuals
// (rule S1 keeps them, as the single solve's restart does); bnorm_out (host, nrhs or NULL) receives the
// norms of b.
int block_solve(const csls_factor_t* F, const csls_csr* A, const double* b, int64_t nrhs, int64_t ldb, double* x,
                int64_t ldx, const csls_opts* o, void* work, size_t bytes, csls_report* rep, cudaStream_t st,
                int64_t* launches, const double* bref = nullptr, double* bnorm_out = nullptr) {
    if (F->variant != CSLS_VARIANT_QR) return CSLS_ERR_ARG;
    if (nrhs > 64) return CSLS_ERR_ARG;
    const int64_t m = F->m, n = F->n, nb = F->nblocks;
    Carve c{(char*)work, 0, bytes, false};
    BlockWs w = block_carve(c, m, n, nb, nrhs);
    const int W = w.W, ngroups = W / kNR;
    const long long spin = o->spin_limit;
    std::vector<LsqrState> h((size_t)W);
    for (int k = 0; k < W; ++k) {
        LsqrState s{};
        s.atol = o->atol;
        s.btol = o->btol;
        s.maxit = o->maxit > 0 ? o->maxit : n;
        s.fixed = o->fixed_iters;
        s.hist_cap = w.hist_cap;
        s.cs2 = -1.0;
        s.first = 1;
        s.bnorm_ref = (bref && k < nrhs) ? (bref[k] > 0.0 ? bref[k] : 1e-300) : 0.0;
        h[(size_t)k] = s;
    }
    CSLS_CUDA(cudaMemcpyAsync(w.st, h.data(), sizeof(LsqrState) * (size_t)W, cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(BlockCtl), st));
    CSLS_CUDA(cudaMemsetAsync(w.flags_up, 0, sizeof(int) * (size_t)(nb * ngroups), st));
    CSLS_CUDA(cudaMemsetAsync(w.flags_lo, 0, sizeof(int) * (size_t)(nb * ngroups), st));
    CSLS_CUDA(cudaMemsetAsync(w.wflags_up, 0, sizeof(int) * (size_t)(nb * w.maxp * ngroups), st));
    CSLS_CUDA(cudaMemsetAsync(w.wflags_lo, 0, sizeof(int) * (size_t)(nb * w.maxp * ngroups), st));
    const std::vector<long long> tick = block_tickets(nb, ngroups, w.kp);
    if ((int64_t)tick.size() != w.ntick) return CSLS_ERR_ARG;
    CSLS_CUDA(cudaMemcpyAsync(w.tick, tick.data(), sizeof(long long) * tick.size(), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemsetAsync(w.X, 0, sizeof(double) * (size_t)(n * W), st));
    CSLS_CUDA(cudaMemsetAsync(w.Z, 0, sizeof(double) * (size_t)(n * W), st));
    CSLS_CUDA(cudaMemsetAsync(w.V, 0, sizeof(double) * (size_t)(n * W), st));
    CSLS_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * (size_t)(n * W), st));
    CSLS_CUDA(cudaMemsetAsync(w.WX, 0, sizeof(double) * (size_t)(n * W), st));
    CSLS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    const int sms = device_sm_count();
    const int gm = (int)std::min<int64_t>(ceil_div(m * 32, kBT), (int64_t)sms * 8);
    const int gn = (int)std::min<int64_t>(ceil_div(n * 32, kBT), (int64_t)sms * 8);
    const size_t red_bytes = sizeof(double) * (size_t)((kBT / 32) * W + W);
    const dim3 tg((unsigned)w.ntick);
    const unsigned total = (unsigned)w.ntick;
    auto upper = [&]() -> int {
        if (F->prec == CSLS_PREC_F64)
            k_blk_trsv_upper<double><<<tg, kBT, 0, st>>>((const double*)F->R, n, (int)nb, ngroups, F->Dinv, W, w.V,
                                                         w.Z, w.WX, w.X, w.flags_up, w.tick, w.kp, w.maxp, w.wpart,
                                                         w.wflags_up, total, w.ctl, w.st, spin, w.err);
        else
            k_blk_trsv_upper<float><<<tg, kBT, 0, st>>>((const float*)F->R, n, (int)nb, ngroups, F->Dinv, W, w.V, w.Z,
                                                        w.WX, w.X, w.flags_up, w.tick, w.kp, w.maxp, w.wpart,
                                                        w.wflags_up, total, w.ctl, w.st, spin, w.err);
        CSLS_CUDA(cudaGetLastError());
        return CSLS_OK;
    };
    auto lower = [&](int mode) -> int {
        const double* R64 = (const double*)F->R;
        const float* R32 = (const float*)F->R;
        const bool f64 = F->prec == CSLS_PREC_F64;
#define CSLS_BLK_LOWER(T, M, RP)                                                                                   \
    k_blk_trsv_lower<T, M><<<tg, kBT, 0, st>>>(RP, n, (int)nb, ngroups, F->Dinv, W, w.G, w.V, w.flags_lo, w.tick, w.kp, \
                                               w.maxp, w.wpart, w.wflags_lo, total, w.ctl, w.st, w.lo_part, w.hist,   \
                                               spin, w.err)
        if (f64 && mode == 1) CSLS_BLK_LOWER(double, 1, R64);
        else if (f64) CSLS_BLK_LOWER(double, 2, R64);
        else if (mode == 1) CSLS_BLK_LOWER(float, 1, R32);
        else CSLS_BLK_LOWER(float, 2, R32);
#undef CSLS_BLK_LOWER
        CSLS_CUDA(cudaGetLastError());
        return CSLS_OK;
    };
    k_blk_start<<<gm, kBT, red_bytes, st>>>(b, ldb, m, (int)nrhs, W, w.U, w.st, w.ctl, w.sp_part);
    CSLS_CUDA(cudaGetLastError());
    k_blk_spmtm<<<gn, kBT, sizeof(double) * W, st>>>(F->AT.row_ptr, F->AT.col, F->AT.val, n, W, w.U, w.G, w.st);
    CSLS_CUDA(cudaGetLastError());
    CSLS_TRY(lower(2));
    int64_t nl = 3;
    const int64_t limit = o->fixed_iters > 0 ? o->fixed_iters : (o->maxit > 0 ? o->maxit : n);
    const int64_t chunk = o->check_every > 0 ? o->check_every : 16;
    for (int64_t it = 0; it < limit; it += chunk) {
        for (int64_t k = 0; k < chunk && it + k < limit; ++k) {
            CSLS_TRY(upper());
            k_blk_spmm<<<gm, kBT, red_bytes, st>>>(A->row_ptr, A->col, A->val, m, W, w.Z, w.U, w.st, w.ctl, w.sp_part);
            CSLS_CUDA(cudaGetLastError());
            k_blk_spmtm<<<gn, kBT, sizeof(double) * W, st>>>(F->AT.row_ptr, F->AT.col, F->AT.val, n, W, w.U, w.G,
                                                             w.st);
            CSLS_CUDA(cudaGetLastError());
            CSLS_TRY(lower(1));
            nl += 4;
        }
        BlockCtl hc{};
        CSLS_CUDA(cudaMemcpyAsync(&hc, w.ctl, sizeof(BlockCtl), cudaMemcpyDeviceToHost, st));
        CSLS_CUDA(cudaStreamSynchronize(st));
        if (hc.all_done) break;
    }
    k_blk_finish<<<(unsigned)std::min<int64_t>(ceil_div(n * nrhs, 256), (int64_t)sms * 8), 256, 0, st>>>(
        w.X, w.WX, n, W, (int)nrhs, w.st, x, ldx);
    CSLS_CUDA(cudaGetLastError());
    ++nl;
    std::vector<LsqrState> out((size_t)W);
    int err = 0;
    CSLS_CUDA(cudaMemcpyAsync(out.data(), w.st, sizeof(LsqrState) * (size_t)W, cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    int status = err;
    int64_t max_it = 0;
    for (int64_t k = 0; k < nrhs; ++k) {
        const LsqrState& s = out[(size_t)k];
        if (bnorm_out) bnorm_out[k] = s.bnorm;
        max_it = std::max<int64_t>(max_it, s.iter);
        if (status == CSLS_OK && s.err) status = s.err;
        if (status == CSLS_OK && o->fixed_iters <= 0 && s.istop == 0 && s.done) status = CSLS_ERR_NOT_CONVERGED;
    }
    if (rep) {
        const LsqrState& s = out[0];
        rep->istop = s.istop;
        rep->iterations = max_it;
        rep->bnorm = s.bnorm;
        rep->rnorm = s.rnorm;
        rep->arnorm = s.arnorm;
        rep->anorm = std::sqrt(s.anorm2);
        rep->ynorm = s.ynorm;
    }
    if (launches) *launches += nl;
    return status;
}

}  // namespace csls

namespace csls {

// Block LSQR with restarts (opts.refine): after the solve, each restart solves the block for the
// correction from the residuals r_k = b_k - A x_k and adds it to x (the block form of the single
// solve's restart). Reports the first solve's maximum iteration count plus the restarts' maxima.
int block_solve_refined(const csls_factor_t* F, const csls_csr* A, const double* b, int64_t nrhs, int64_t ldb,
                        double* x, int64_t ldx, const csls_opts* o, void* work, size_t bytes, csls_report* rep,
                        cudaStream_t st, int64_t* launches) {
    std::vector<double> bn((size_t)nrhs, 0.0);
    int sk = block_solve(F, A, b, nrhs, ldb, x, ldx, o, work, bytes, rep, st, launches, nullptr, bn.data());
    if (o->refine <= 0) return sk;
    const int64_t m = F->m, n = F->n;
    const size_t own = block_ws_bytes(m, n, F->nblocks, nrhs);
    if (bytes < own + block_refine_bytes(m, n, nrhs)) return CSLS_ERR_WORKSPACE;
    Carve c{(char*)work + own, 0, bytes - own, false};
    double* res = c.take<double>((size_t)(m * nrhs));
    double* dx = c.take<double>((size_t)(n * nrhs));
    int64_t its_ref = 0;
    for (int64_t p = 0; p < o->refine && (sk == CSLS_OK || sk == CSLS_ERR_NOT_CONVERGED); ++p) {
        for (int64_t k = 0; k < nrhs; ++k) CSLS_TRY(launch_residual(A, x + k * ldx, b + k * ldb, res + k * m, st));
        csls_report rr{};
        sk = block_solve(F, A, res, nrhs, m, dx, n, o, work, own, &rr, st, launches, bn.data(), nullptr);
        const int sms = device_sm_count();
        k_add_cols<<<(unsigned)std::min<int64_t>(ceil_div(n * nrhs, 256), (int64_t)sms * 8), 256, 0, st>>>(
            x, ldx, dx, n, (int)nrhs);
        CSLS_CUDA(cudaGetLastError());
        if (launches) *launches += nrhs + 1;
        its_ref += rr.iterations;
        if (rep) {
            rep->rnorm = rr.rnorm;
            rep->arnorm = rr.arnorm;
            rep->istop = rr.istop;
        }
    }
    if (rep) {
        rep->iterations += its_ref;
        rep->iterations_refine = its_ref;
    }
    return sk;
}

}  // namespace csls

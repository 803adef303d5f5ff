// Triangular solves with binary64 R on a cluster-resident chain: the per-step preconditioner
// applications z = R^{-1} v and y = R^{-T} g of the implicit form (Remark after Algorithm 2),
// one launch per solve.
//
// A solve is a chain over the nb = ceil(n / 64) diagonal blocks in solve order (upper: nb - 1 down
// to 0; transposed: 0 up to nb - 1); block b needs the solutions of every block before it. On this
// part an SM retires two FP64 FMAs per clock, so one chain step done by one CTA (the 64 x 64
// product with the newest solution block plus the 64 x 64 diagonal-inverse product) costs ~2 us of
// FP64 issue alone. Here the chain runs on one cluster of 8 CTAs, each owning 8 rows of every
// block, that exchange the step's right-hand side and solution through distributed shared memory.
// Each value travels as two 8-byte words {half of its bits, step tag}, written whole by one remote
// store, and the reader polls its own shared memory until both tags match: no fence or barrier
// round trip sits on the chain (a remote release-arrive per value measured ~1 us per exchange).
//   chain CTA q, warps 0-3  rows 8q .. 8q + 7 of the block (two rows a warp, 16 lanes a row, 4
//                           columns a lane): the product with the previous step's solution (the
//                           only product on the critical path), the right-hand side, the
//                           diagonal-inverse product, the LSQR epilogue of the rows, and the
//                           products of the new solution with the blocks of the next kLook - 1
//                           steps (kept per lane, reduced when their step comes);
//                  warp 4  publishes each solved block for the workers (fence, then a flag);
//                  warp 5  bulk-copies each step's operands into a ring of shared-memory slots:
//                           the CTA's rows of the diagonal inverse and of the kLook blocks of R that
//                           the step multiplies, packed per step and rank at factor time;
//                  warp 6  prefetches the workers' far sums of the CTA's rows, kRing steps ahead.
// Every other cluster holds 8 workers, one per block in solve order. A worker sums the products of
// its block row (upper) or column (transposed) of R with the solutions of the blocks more than
// kLook steps before it, as the chain publishes them, and publishes that far sum with a flag.
// Clusters take tickets in launch order and the first becomes the chain, so a worker waits only for
// blocks the chain can finish without it, and the chain only for workers that started earlier or
// can start once earlier ones finish. Each CTA asks for more than half an SM's shared memory, so no
// SM runs two of them (the chain's FP64 pipes serve only the chain).
//
// Every wait is bounded (poll count and wall time). A CTA that gives up sets the error word and
// its abort flag, skips its remaining work, waits (bounded by wall time alone) for its bulk copies
// in flight, and meets its cluster at the final barrier, so no CTA leaves while a peer may still
// write into its shared memory.
#include <mutex>

#include "lsqr.cuh"
#include "tc.cuh"

namespace csls {

constexpr int kCl = 8;                                     // chain cluster size
constexpr int kClRows = kTrsvBlock / kCl;                   // rows of a block per chain CTA
constexpr int kLook = 4;                                    // later blocks the chain updates itself
constexpr int kPackRegion = kClRows * kTrsvBlock;           // 8 x 64 doubles
constexpr int kPackD = (kLook + 1) * kPackRegion;           // doubles per (block, rank) slot
constexpr int kRing = 4;                                    // operand slots in shared memory
constexpr int kClThreads = 256;
constexpr size_t kClSmem = 120 * 1024;                      // > half an SM: one CTA per SM
constexpr unsigned long long kClWaitNs = 4000000000ULL;
constexpr long long kClTeardownSpin = 1LL << 62;

int64_t trsv_pack_doubles(int64_t n) { return ceil_div(n, kTrsvBlock) * kCl * kPackD; }

struct ClSmem {
    double pack[kRing][kPackD];        // per step: D (8 x 64), P (8 x 64), N_1 .. N_{kLook-1}
    // the cluster exchanges, by step parity: each row's value as two 8-byte words {half of its bits,
    // step tag}; a word is written whole, so a reader that sees both tags of the step has the value
    ulonglong2 xrhs[2][kTrsvBlock];    // right-hand sides
    ulonglong2 xz[2][kTrsvBlock];      // solutions
    double far[kRing][kClRows];        // the workers' far sums of this CTA's rows
    double sq[kTrsvBlock];             // rank 0: squared norms per row slot (transposed, LSQR)
    uint64_t pack_full[kRing], pack_free[kRing], far_full[kRing];   // local barriers of the pipeline
    unsigned role;
    int abort;
};
static_assert(sizeof(ClSmem) <= kClSmem, "chain shared memory");

// ------------------------------------------------------------------ cluster primitives

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// address of the same shared-memory object in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(const void* p, unsigned rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(tc::smem_addr(p)), "r"(rank));
    return d;
}
__device__ __forceinline__ void cl_st_f64(uint32_t a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_st_u32(uint32_t a, unsigned v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// the pipeline barriers are all CTA-local (bulk-copy completions and this CTA's warps): acquire at CTA scope
__device__ __forceinline__ bool cl_try_wait(uint64_t* bar, uint32_t parity) { return tc::mbar_try_wait(bar, parity); }
// One 16-byte store of a value with its step tag into a CTA of the cluster: two 8-byte words, each
// {half of the value's bits, tag}, each written whole.
__device__ __forceinline__ void cl_send(uint32_t a, double v, unsigned tag) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned long long w0 = ((unsigned long long)tag << 32) | (u & 0xffffffffULL);
    const unsigned long long w1 = ((unsigned long long)tag << 32) | (u >> 32);
    asm volatile("st.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(w0), "l"(w1) : "memory");
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Bounded wait for a phase of a local barrier; false (after setting the error and the abort flag)
// when it gives up.
__device__ __forceinline__ bool cl_wait(uint64_t* bar, uint32_t parity, long long spin, ClSmem& sm, int* err) {
    if (cl_try_wait(bar, parity)) return true;   // usually complete: no clock read on this path
    const uint64_t t0 = tc::global_ns();
    for (long long it = 0;; ++it) {
        if (cl_try_wait(bar, parity)) return true;
        if (*(volatile int*)&sm.abort) return false;
        // the wall clock is read every 256 polls only (its read is slow next to a poll)
        if (it > spin || ((it & 255) == 255 && tc::global_ns() - t0 > kClWaitNs)) {
            set_error(err, CSLS_ERR_TIMEOUT);
            *(volatile int*)&sm.abort = 1;
            return false;
        }
    }
}

// The same tagged 16-byte value in global memory (a plain store: the tag says the value is there).
__device__ __forceinline__ void st_tagged(ulonglong2* p, double v, unsigned tag) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned long long w0 = ((unsigned long long)tag << 32) | (u & 0xffffffffULL);
    const unsigned long long w1 = ((unsigned long long)tag << 32) | (u >> 32);
    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(w0), "l"(w1) : "memory");
}
__device__ __forceinline__ ulonglong2 ld_tagged(const ulonglong2* p) {
    ulonglong2 w;
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(w.x), "=l"(w.y) : "l"(p) : "memory");
    return w;
}
__device__ __forceinline__ bool tag_is(const ulonglong2& w, unsigned tag) {
    return (unsigned)(w.x >> 32) == tag && (unsigned)(w.y >> 32) == tag;
}
__device__ __forceinline__ double tagged_value(const ulonglong2& w) {
    return __longlong_as_double((long long)((w.x & 0xffffffffULL) | (w.y << 32)));
}
// Polls a tagged global value until it carries `tag` (one lane); bounded by poll count and wall time.
__device__ __forceinline__ bool poll_tagged(const ulonglong2* p, unsigned tag, ulonglong2& w, long long spin, ClSmem* sm,
                                            int* err) {
    if (tag_is(w, tag)) return true;
    long long it = 0;
    const uint64_t t0 = tc::global_ns();
    for (;;) {
        w = ld_tagged(p);
        if (tag_is(w, tag)) return true;
        if (sm && *(volatile int*)&sm->abort) return false;
        if (++it > spin || ((it & 255) == 255 && tc::global_ns() - t0 > kClWaitNs)) {
            set_error(err, CSLS_ERR_TIMEOUT);
            if (sm) *(volatile int*)&sm->abort = 1;
            return false;
        }
        if (it > 512) __nanosleep(32);
    }
}

// Polls four consecutive tagged values in this CTA's shared memory until every word carries `tag`;
// bounded like cl_wait.
__device__ __forceinline__ bool cl_recv4(const ulonglong2* p, unsigned tag, double (&v)[4], long long spin, ClSmem& sm,
                                         int* err) {
    uint64_t t0 = 0;
    for (long long it = 0;; ++it) {
        bool all = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            unsigned long long w0, w1;
            asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "r"(tc::smem_addr(p + k)));
            if ((unsigned)(w0 >> 32) == tag && (unsigned)(w1 >> 32) == tag)
                v[k] = __longlong_as_double((long long)((w0 & 0xffffffffULL) | (w1 << 32)));
            else
                all = false;
        }
        if (all) return true;
        if (*(volatile int*)&sm.abort) return false;
        if (it == 0) t0 = tc::global_ns();
        if (it > spin || ((it & 255) == 255 && tc::global_ns() - t0 > kClWaitNs)) {
            set_error(err, CSLS_ERR_TIMEOUT);
            *(volatile int*)&sm.abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ double sum16(double v) {
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ operand packs (factor time)

// pack[(b * 8 + q) * kPackD + region * 512 + r * 64 + c] for chain rank q, row r (block row 8q + r):
//   region 0          D: upper Dinv_b(8q + r, c); transposed Dinv_b(c, 8q + r)
//   region 1          P: the product with the previous step's solution:
//                        upper R(64b + 8q + r, 64(b + 1) + c); transposed R(64(b - 1) + c, 64b + 8q + r)
//   region 1 + k      N_k (k = 1 .. kLook - 1): the new solution's product for the step k + 1 later:
//                        upper R(64(b - 1 - k) + 8q + r, 64b + c); transposed R(64b + c, 64(b + 1 + k) + 8q + r)
// Entries outside R (or past n) are zero.
template <bool UPPER>
__global__ void __launch_bounds__(256) k_trsv_pack(const double* __restrict__ R, int64_t n, int nb,
                                                   const double* __restrict__ Dinv, double* pack) {
    const int b = blockIdx.x, q = blockIdx.y;
    double* out = pack + ((int64_t)b * kCl + q) * kPackD;
    for (int e = threadIdx.x; e < kPackD; e += blockDim.x) {
        const int reg = e / kPackRegion, r = (e / kTrsvBlock) % kClRows, c = e % kTrsvBlock;
        const int64_t i = (int64_t)q * kClRows + r;
        double v = 0.0;
        if (reg == 0) {
            if ((int64_t)b * kTrsvBlock + i < n && (int64_t)b * kTrsvBlock + c < n)
                v = UPPER ? Dinv[(int64_t)b * kTrsvBlock * kTrsvBlock + i + (int64_t)c * kTrsvBlock]
                          : Dinv[(int64_t)b * kTrsvBlock * kTrsvBlock + c + i * kTrsvBlock];
        } else {
            int64_t rb, cb, rr, cc;
            if (UPPER) {
                rb = reg == 1 ? b : b - reg;
                cb = reg == 1 ? b + 1 : b;
                rr = rb * kTrsvBlock + i;
                cc = cb * kTrsvBlock + c;
            } else {
                rb = reg == 1 ? b - 1 : b;
                cb = reg == 1 ? b : b + reg;
                rr = rb * kTrsvBlock + c;
                cc = cb * kTrsvBlock + i;
            }
            if (rb >= 0 && cb < nb && rr < n && cc < n) v = R[rr + cc * n];
        }
        out[e] = v;
    }
}

int trsv_build_packs(const double* R, int64_t n, const double* Dinv, double* pack_up, double* pack_lo,
                     cudaStream_t s) {
    const int nb = (int)ceil_div(n, kTrsvBlock);
    const dim3 grid((unsigned)nb, kCl);
    k_trsv_pack<true><<<grid, 256, 0, s>>>(R, n, nb, Dinv, pack_up);
    k_trsv_pack<false><<<grid, 256, 0, s>>>(R, n, nb, Dinv, pack_lo);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

// ------------------------------------------------------------------ the solve

// UPPER, MODE 0: z = R^{-1} v.   UPPER, MODE 1: z = R^{-1} (v / alpha), x / wx epilogue.
// transposed, MODE 0: out = R^{-T} g (out may be g).  MODE 1: g <- R^{-T} g, vt <- g - (beta/alpha) vt,
// alpha and the scalar step.  MODE 2: g <- R^{-T} g, vt <- g, alpha_1 and the start values.
// zt, ft: n tagged 16-byte words each (the chain's solutions for the workers, the workers' far sums
// for the chain), tagged with the launch's flag value; zeroed before a solve's first launch.
template <bool UPPER, int MODE>
__global__ void __launch_bounds__(kClThreads, 1)
k_trsv_cl(const double* __restrict__ R, int64_t n, int nb, const double* __restrict__ pack, const double* vin_p,
          double* out, double* g, double* vt, ulonglong2* zt, ulonglong2* ft, TrsvCtl* ctl, LsqrState* st, double* wx,
          double* x, double* hist, long long spin, int* err) {
    extern __shared__ __align__(128) unsigned char cl_dyn[];
    ClSmem& sm = *reinterpret_cast<ClSmem*>(cl_dyn);
    __shared__ unsigned epoch_s;
    __shared__ double coef[4];
    __shared__ double wpart[4][kTrsvBlock];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (MODE == 1 && *(volatile int*)&st->done) return;   // the same for every CTA of the launch
    const unsigned q = cl_rank();
    if (tid == 0) {
        epoch_s = *(volatile unsigned*)&ctl->epoch;
        sm.abort = 0;
        if (UPPER && MODE == 1) {
            coef[0] = 1.0 / st->alpha;
            coef[1] = st->cx;
            coef[2] = st->cw;
            coef[3] = (double)st->first;
        } else if (!UPPER && MODE == 1) {
            coef[0] = st->beta / st->alpha;
        } else {
            coef[0] = 1.0;
        }
        for (int i = 0; i < kRing; ++i) {
            tc::mbar_init(&sm.pack_full[i], 1);
            tc::mbar_init(&sm.pack_free[i], 4);
            tc::mbar_init(&sm.far_full[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
        }
        tc::mbar_init_fence();
    }
    for (int e = tid; e < 2 * kTrsvBlock; e += kClThreads) {
        (&sm.xrhs[0][0])[e] = make_ulonglong2(~0ULL, ~0ULL);   // a tag no step uses
        (&sm.xz[0][0])[e] = make_ulonglong2(~0ULL, ~0ULL);
    }
    // every CTA of the cluster has started (and initialised its barriers): the cluster's ticket
    // can be handed out through distributed shared memory
    __syncwarp();
    cl_sync();
    if (q == 0 && tid == 0) {
        const unsigned t = atomicAdd(&ctl->ticket, 1u);
        for (unsigned d = 0; d < kCl; ++d) cl_st_u32(cl_map(&sm.role, d), t);
    }
    __syncwarp();
    cl_sync();
    const unsigned role = sm.role;
    const int want = (int)(epoch_s + 1u);
    auto blk = [&](int i) { return UPPER ? nb - 1 - i : i; };

    if (role == 0) {
        // ---------------------------------------------------------------- chain
        if (warp < 4) {
            const int rl = 2 * warp + (lane >> 4), l16 = lane & 15;
            const bool res = l16 == 0;
            const int rin = (int)q * kClRows + rl;   // row within the block
            // lanes 0..7 of a row each send its values to one CTA of the cluster (one remote store and
            // one release-arrive per lane: a lane that sent to all eight would serialise eight round trips)
            const bool sender = l16 < kCl;
            const unsigned dst = sender ? (unsigned)l16 : 0u;
            const uint32_t r_rhs0 = cl_map(&sm.xrhs[0][rin], dst), r_rhs1 = cl_map(&sm.xrhs[1][rin], dst);
            const uint32_t r_z0 = cl_map(&sm.xz[0][rin], dst), r_z1 = cl_map(&sm.xz[1][rin], dst);
            const unsigned tag_base = ((unsigned)want & 0xFFFFu) << 16;   // tag of step i: tag_base | i
            double zprev[4] = {0.0, 0.0, 0.0, 0.0};   // this lane's 4 columns of the previous step's solution
            double nacc[kLook];   // nacc[k]: this lane's partial for the block of step i + k
#pragma unroll
            for (int k = 0; k < kLook; ++k) nacc[k] = 0.0;
            double sq = 0.0;
            // per-step inputs of the row, loaded a step ahead: the right-hand side (all lanes), and for the
            // result lane the previous vt (transposed, LSQR step) or wx and x (upper, LSQR step)
            auto load_in = [&](int i, double& vi, double& a, double& c) {
                const int64_t row = (int64_t)blk(i) * kTrsvBlock + rin;
                vi = 0.0;
                a = 0.0;
                c = 0.0;
                if (row < n) {
                    vi = UPPER ? vin_p[row] * coef[0] : g[row];
                    if (res && !UPPER && MODE == 1) a = vt[row];
                    if (res && UPPER && MODE == 1) {
                        a = wx[row];
                        c = x[row];
                    }
                }
            };
            double vin_n, a_n, c_n;
            load_in(0, vin_n, a_n, c_n);
            bool ok = true;
            for (int i = 0; i < nb; ++i) {
                const int b = blk(i);
                const int64_t row = (int64_t)b * kTrsvBlock + rin;
                const int slot = i % kRing;
                const double vin = vin_n, a_in = a_n, c_in = c_n;
                if (i + 1 < nb) load_in(i + 1, vin_n, a_n, c_n);
                if (ok) ok = __all_sync(0xffffffffu, cl_wait(&sm.pack_full[slot], (uint32_t)((i / kRing) & 1), spin, sm, err));
                const double* pk = sm.pack[slot];
                double s = 0.0;
                if (ok) {
                    // the only product on the critical path: the previous step's solution
                    if (i > 0) {
                        const double2* P = reinterpret_cast<const double2*>(pk + kPackRegion + rl * kTrsvBlock + 4 * l16);
                        const double2 p0 = P[0], p1 = P[1];
                        double t0 = fma(p0.x, zprev[0], nacc[0]);
                        double t1 = p0.y * zprev[1];
                        t0 = fma(p1.x, zprev[2], t0);
                        t1 = fma(p1.y, zprev[3], t1);
                        nacc[0] = t0 + t1;
                    }
                    s = sum16(nacc[0]);
                    ok = __all_sync(0xffffffffu, cl_wait(&sm.far_full[slot], (uint32_t)((i / kRing) & 1), spin, sm, err));
                }
                const double farv = ok ? sm.far[slot][rl] : 0.0;
                const double rhs = (ok && row < n) ? (vin - farv) - s : 0.0;
                const unsigned tag = tag_base | (unsigned)i;
                if (sender) cl_send((i & 1) ? r_rhs1 : r_rhs0, rhs, tag);
                // while the right-hand sides travel: the previous solution's products with the blocks of
                // the next kLook - 1 steps (its operand slot is released after them)
                if (i > 0) {
                    if (ok) {
                        const double* pkp = sm.pack[(i - 1) % kRing];
#pragma unroll
                        for (int k = 1; k < kLook; ++k) {
                            const double2* N =
                                reinterpret_cast<const double2*>(pkp + (1 + k) * kPackRegion + rl * kTrsvBlock + 4 * l16);
                            const double2 n0 = N[0], n1 = N[1];
                            nacc[k] = fma(n0.x, zprev[0], nacc[k]);
                            nacc[k] = fma(n0.y, zprev[1], nacc[k]);
                            nacc[k] = fma(n1.x, zprev[2], nacc[k]);
                            nacc[k] = fma(n1.y, zprev[3], nacc[k]);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&sm.pack_free[(i - 1) % kRing]);
                }
                __syncwarp();
                double rv[4] = {0.0, 0.0, 0.0, 0.0};
                if (ok) ok = __all_sync(0xffffffffu, cl_recv4(&sm.xrhs[i & 1][4 * l16], tag, rv, spin, sm, err));
                double zb = 0.0;
                if (ok) {
                    const double2* D = reinterpret_cast<const double2*>(pk + rl * kTrsvBlock + 4 * l16);
                    const double2 d0 = D[0], d1 = D[1];
                    double t0 = d0.x * rv[0];
                    double t1 = d0.y * rv[1];
                    t0 = fma(d1.x, rv[2], t0);
                    t1 = fma(d1.y, rv[3], t1);
                    zb = sum16(t0 + t1);
                    if (row >= n) zb = 0.0;
                }
                if (sender) cl_send((i & 1) ? r_z1 : r_z0, zb, tag);
                if (res) {
                    if (ok && row < n) {
                        if (UPPER) {
                            out[row] = zb;
                            if (MODE == 1) {   // x += cx wx, wx = z - cw wx (the first step: wx = z)
                                if (coef[3] != 0.0) {
                                    wx[row] = zb;
                                } else {
                                    x[row] = c_in + coef[1] * a_in;
                                    wx[row] = zb - coef[2] * a_in;
                                }
                            }
                        } else if (MODE == 0) {
                            out[row] = zb;
                        } else {
                            g[row] = zb;
                            const double vn = MODE == 1 ? zb - coef[0] * a_in : zb;
                            vt[row] = vn;
                            sq += vn * vn;
                        }
                    }
                    if (row < n) st_tagged(zt + row, zb, (unsigned)want);   // for the workers
                }
                __syncwarp();
                if (ok) ok = __all_sync(0xffffffffu, cl_recv4(&sm.xz[i & 1][4 * l16], tag, zprev, spin, sm, err));
#pragma unroll
                for (int k = 0; k + 1 < kLook; ++k) nacc[k] = nacc[k + 1];
                nacc[kLook - 1] = 0.0;
            }
            if (!UPPER && MODE != 0 && res) cl_st_f64(cl_map(&sm.sq[rin], 0), sq);
        } else if (warp == 5) {
            // operand copies, kRing steps ahead of the chain
            if (lane == 0) {
                int issued = 0;
                for (int j = 0; j < nb; ++j) {
                    const int slot = j % kRing;
                    if (j >= kRing && !cl_wait(&sm.pack_free[slot], (uint32_t)(((j - kRing) / kRing) & 1), spin, sm, err))
                        break;
                    if (*(volatile int*)&sm.abort) break;
                    tc::mbar_arrive_expect_tx(&sm.pack_full[slot], (uint32_t)(kPackD * sizeof(double)));
                    tc::bulk_g2s(sm.pack[slot], pack + ((int64_t)blk(j) * kCl + q) * kPackD,
                                 (uint32_t)(kPackD * sizeof(double)), &sm.pack_full[slot]);
                    ++issued;
                }
                // copies still in flight (those the chain has not waited for) land before the CTA leaves
                for (int j = (issued > kRing ? issued - kRing : 0); j < issued; ++j)
                    tc::mbar_wait(&sm.pack_full[j % kRing], (uint32_t)((j / kRing) & 1), kClTeardownSpin, kClWaitNs,
                                  nullptr);
            }
        } else if (warp == 6) {
            // the workers' far sums of this CTA's rows, kRing steps ahead (lanes 0..7, one row each)
            for (int j = 0; j < nb; ++j) {
                const int slot = j % kRing;
                bool ok = true;
                if (lane == 0 && j >= kRing)
                    ok = cl_wait(&sm.pack_free[slot], (uint32_t)(((j - kRing) / kRing) & 1), spin, sm, err);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok && lane < kClRows) {
                    const int64_t row = (int64_t)blk(j) * kTrsvBlock + q * kClRows + lane;
                    double f = 0.0;
                    if (row < n) {
                        ulonglong2 w = ld_tagged(ft + row);
                        ok = poll_tagged(ft + row, (unsigned)want, w, spin, &sm, err);
                        f = tagged_value(w);
                    }
                    sm.far[slot][lane] = f;
                }
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&sm.far_full[slot]);
            }
        }
        // every CTA of the chain is done with the others' shared memory
        __syncwarp();
        cl_sync();
        if (!UPPER && MODE != 0 && q == 0 && tid == 0 && !*(volatile int*)&sm.abort) {
            double t = 0.0;
            for (int k = 0; k < kTrsvBlock; ++k) t += sm.sq[k];
            const double alpha_new = sqrt(t);
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
    } else {
        // ---------------------------------------------------------------- workers
        const int64_t widx = (int64_t)(role - 1) * kCl + q;
        if (widx < nb) {
            const int b = blk((int)widx);
            const int64_t r0 = (int64_t)b * kTrsvBlock;
            const int bs = (int)(n - r0 < kTrsvBlock ? n - r0 : kTrsvBlock);
            const int rc = tid & (kTrsvBlock - 1), qq = tid >> 6;   // row (column) of the block, column group
            // solve-order steps whose solutions this block takes from the workers: the first i0
            const int i_b = UPPER ? nb - 1 - b : b;
            const int i0 = i_b - kLook;   // steps 0 .. i0 - 1
            double acc = 0.0;
            if (i0 > 0) {
                auto load_block = [&](int c, double (&dst)[16]) {
                    const int64_t c0 = (int64_t)c * kTrsvBlock;
                    if (UPPER) {
                        const int cs = (int)(n - c0 < kTrsvBlock ? n - c0 : kTrsvBlock);
                        const double* rp = R + (r0 + rc) + (c0 + qq * 16) * n;
#pragma unroll
                        for (int kk = 0; kk < 16; ++kk)
                            dst[kk] = (rc < bs && qq * 16 + kk < cs) ? __ldg(rp + (int64_t)kk * n) : 0.0;
                    } else {
                        // column r0 + rc, rows c0 + 16 qq .. + 15: contiguous, read as 16-byte pairs when aligned
                        const double* rp = R + (c0 + qq * 16) + (r0 + rc) * n;
                        if (rc < bs && ((reinterpret_cast<uintptr_t>(rp) & 15) == 0)) {
#pragma unroll
                            for (int kk = 0; kk < 16; kk += 2) {
                                const double2 t = __ldg(reinterpret_cast<const double2*>(rp + kk));
                                dst[kk] = t.x;
                                dst[kk + 1] = t.y;
                            }
                        } else {
#pragma unroll
                            for (int kk = 0; kk < 16; ++kk) dst[kk] = rc < bs ? __ldg(rp + kk) : 0.0;
                        }
                    }
                };
                // lane k < 16 of a warp polls entry k of its column group of the chain's tagged solution.
                // A worker catching up on blocks already published is bound by its FP64 pipe only if its
                // loads are in flight ahead: R two blocks ahead, the solution one block ahead (its poll is
                // issued before the current block's products).
                auto zidx = [&](int c) { return (int64_t)c * kTrsvBlock + qq * 16 + (lane & 15); };
                auto zvalid = [&](int c) { return lane < 16 && zidx(c) < n; };
                ulonglong2 zw = make_ulonglong2(0ULL, 0ULL);
                if (zvalid(blk(0))) zw = ld_tagged(zt + zidx(blk(0)));
                double rv[16], rn[16];
                load_block(blk(0), rv);
                if (i0 > 1) load_block(blk(1), rn);
                for (int i = 0; i < i0; ++i) {
                    const int c = blk(i);
                    bool ok = true;
                    double zmine = 0.0;
                    if (zvalid(c)) {
                        ok = poll_tagged(zt + zidx(c), (unsigned)want, zw, spin, nullptr, err);
                        zmine = tagged_value(zw);
                    }
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    double rnn[16];
                    if (i + 1 < i0) {
                        const int cn = blk(i + 1);
                        zw = zvalid(cn) ? ld_tagged(zt + zidx(cn)) : make_ulonglong2(0ULL, 0ULL);
                    }
                    if (i + 2 < i0) load_block(blk(i + 2), rnn);
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) acc = fma(rv[kk], __shfl_sync(0xffffffffu, zmine, kk), acc);
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) {
                        rv[kk] = rn[kk];
                        if (i + 2 < i0) rn[kk] = rnn[kk];
                    }
                }
            }
            wpart[qq][rc] = acc;
            __syncthreads();
            if (tid < bs)
                st_tagged(ft + r0 + tid, ((wpart[0][tid] + wpart[1][tid]) + wpart[2][tid]) + wpart[3][tid], (unsigned)want);
        }
    }
    // launch bookkeeping: the last CTA to finish hands the epoch on
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            ctl->ticket = 0;
            ctl->done = 0;
            if (UPPER && MODE == 1) st->first = 0;
            __threadfence();
            atomicAdd(&ctl->epoch, 1u);
        }
    }
}

// ------------------------------------------------------------------ host side

template <bool UPPER, int MODE>
static int launch_cl(const TrsvArgs& a, const double* pack, const double* vin, double* out, double* g, double* vt,
                     int* flags, TrsvCtl* ctl, LsqrState* st, double* wx, double* x, double* hist, long long spin,
                     int* err, cudaStream_t s) {
    auto kern = k_trsv_cl<UPPER, MODE>;
    CSLS_TRY(raise_smem_limit((const void*)kern, (int)kClSmem));
    ulonglong2* zt = trsv_tagged(flags, a.nb);
    ulonglong2* ft = zt + (a.n + 64);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kCl * (1 + ceil_div(a.nb, kCl))));
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = kClSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CSLS_CUDA(cudaLaunchKernelEx(&cfg, kern, (const double*)a.R, a.n, a.nb, pack, vin, out, g, vt, zt, ft, ctl, st, wx,
                                 x, hist, spin, err));
    return CSLS_OK;
}

// The chain needs two clusters resident at once (the chain and the workers of the block it waits
// for); checked once per device.
bool trsv_cluster_usable() {
    static std::mutex mu;
    static int ok_dev[64] = {};   // 0 unknown, 1 usable, 2 not
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (ok_dev[dev] == 0) {
        auto kern = k_trsv_cl<true, 0>;
        bool ok = raise_smem_limit((const void*)kern, (int)kClSmem) == CSLS_OK;
        int clusters = 0;
        if (ok) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(kCl * 4);
            cfg.blockDim = dim3(kClThreads);
            cfg.dynamicSmemBytes = kClSmem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = kCl;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            ok = cudaOccupancyMaxActiveClusters(&clusters, (const void*)kern, &cfg) == cudaSuccess && clusters >= 2;
        }
        cudaGetLastError();   // a refused query leaves no sticky error
        ok_dev[dev] = ok ? 1 : 2;
    }
    return ok_dev[dev] == 1;
}

int launch_trsv_cl_upper(const TrsvArgs& a, int mode, const double* v, double* z, int* flags, TrsvCtl* ctl,
                         LsqrState* st, double* wx, double* x, long long spin, int* err, cudaStream_t s) {
    if (mode == 0)
        return launch_cl<true, 0>(a, a.pack_up, v, z, nullptr, nullptr, flags, ctl, st, wx, x, nullptr, spin, err, s);
    return launch_cl<true, 1>(a, a.pack_up, v, z, nullptr, nullptr, flags, ctl, st, wx, x, nullptr, spin, err, s);
}

int launch_trsv_cl_lower(const TrsvArgs& a, int mode, double* g, double* vt, double* out, int* flags, TrsvCtl* ctl,
                         LsqrState* st, double* hist, long long spin, int* err, cudaStream_t s) {
    if (mode == 0)
        return launch_cl<false, 0>(a, a.pack_lo, nullptr, out ? out : g, g, vt, flags, ctl, st, nullptr, nullptr, hist,
                                   spin, err, s);
    if (mode == 1)
        return launch_cl<false, 1>(a, a.pack_lo, nullptr, g, g, vt, flags, ctl, st, nullptr, nullptr, hist, spin, err, s);
    return launch_cl<false, 2>(a, a.pack_lo, nullptr, g, g, vt, flags, ctl, st, nullptr, nullptr, hist, spin, err, s);
}

}  // namespace csls

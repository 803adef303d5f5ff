// C ABI entry points: argument checks, workspace layout, orchestration of the
// sketch, factorisation and LSQR kernels, and the host-side report.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lsqr.cuh"

namespace csls {

size_t backward_ws_bytes(int64_t m, int64_t n, int64_t nb);
size_t block_ws_bytes(int64_t m, int64_t n, int64_t nb, int64_t nrhs);
size_t block_refine_bytes(int64_t m, int64_t n, int64_t nrhs);
int block_solve_refined(const csls_factor_t* F, const csls_csr* A, const double* b, int64_t nrhs, int64_t ldb,
                        double* x, int64_t ldx, const csls_opts* o, void* work, size_t bytes, csls_report* rep,
                        cudaStream_t st, int64_t* launches);
constexpr int64_t kBlockMax = 64;   // right-hand sides per block pass

// ------------------------------------------------------------------ validation kernel

__global__ void k_validate_csr(const int64_t* rp, const int32_t* col, const double* val, int64_t m, int64_t n,
                               int64_t nnz, int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        if (b < 0 || e < b || e > nnz) { set_error(err, CSLS_ERR_ARG); continue; }
        int32_t prev = -1;
        for (int64_t p = b; p < e; ++p) {
            const int32_t j = col[p];
            if (j <= prev || j >= n) { set_error(err, CSLS_ERR_ARG); break; }
            prev = j;
            if (!isfinite(val[p])) { set_error(err, CSLS_ERR_NONFINITE); break; }
        }
    }
}

// Warm start: keep ||b|| (computed by the first start pass) for rule S1 and clear the flags that
// pass may have set; errors stay.
__global__ void k_keep_bnorm(csls::LsqrState* st) {
    st->bnorm_ref = st->bnorm > 0.0 ? st->bnorm : 1e-300;
    st->done = 0;
    st->istop = 0;
}

__global__ void k_check_finite(const double* v, int64_t len, int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) { set_error(err, CSLS_ERR_NONFINITE); return; }
}

__global__ void k_final_x(double* x, const double* wx, int64_t n, const LsqrState* st) {
    const double cx = st->cx;
    if (st->iter <= 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += cx * wx[i];
}

static int grid_small(int64_t work) {
    int64_t g = ceil_div(work, 256);
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

static bool aligned256(const void* p) { return ((uintptr_t)p & 255) == 0; }

static int check_csr(const csls_csr* A) {
    if (!A || A->m <= 0 || A->n <= 0 || A->nnz < 0) return CSLS_ERR_ARG;
    if (A->m > 2147483647LL || A->n > 2147483647LL || A->nnz > 2147483647LL) return CSLS_ERR_ARG;
    if (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val))) return CSLS_ERR_ARG;
    return CSLS_OK;
}

static int64_t sketch_rows(const csls_csr* A, const csls_opts* o) {
    int64_t s = o->s > 0 ? o->s : (int64_t)llround(o->gamma * (double)A->n);
    if (s > A->m) s = A->m;
    return s;
}

// ------------------------------------------------------------------ workspaces

struct FactorPersist {
    void* R;
    double* Dinv;
    double* pack_up;
    double* pack_lo;
    Transpose AT;
    double* P;
    double* sigma;
};

static FactorPersist persist_carve(Carve& c, const csls_csr* A, const csls_opts* o) {
    FactorPersist f;
    const int64_t n = A->n;
    const int esz = o->factor_prec == CSLS_PREC_F32 ? 4 : 8;   // R storage
    f.R = c.take<char>((size_t)(n * n * esz));
    f.Dinv = c.take<double>((size_t)(ceil_div(n, kTrsvBlock) * kTrsvBlock * kTrsvBlock));
    if (o->factor_prec != CSLS_PREC_F32 && o->variant == CSLS_VARIANT_QR) {
        f.pack_up = c.take<double>((size_t)trsv_pack_doubles(n));
        f.pack_lo = c.take<double>((size_t)trsv_pack_doubles(n));
    } else {
        f.pack_up = nullptr;
        f.pack_lo = nullptr;
    }
    f.AT.row_ptr = c.take<int64_t>((size_t)n + 1);
    f.AT.col = c.take<int32_t>((size_t)std::max<int64_t>(A->nnz, 1));
    f.AT.val = c.take<double>((size_t)std::max<int64_t>(A->nnz, 1));
    f.AT.perm = c.take<int32_t>((size_t)std::max<int64_t>(A->nnz, 1));
    if (o->variant == CSLS_VARIANT_SVD) {
        f.P = c.take<double>((size_t)(n * n));
        f.sigma = c.take<double>((size_t)n);
    } else {
        f.P = nullptr;
        f.sigma = nullptr;
    }
    return f;
}

struct FactorTemp {
    void* SA;
    int64_t ld;
    SketchScratch sk;
    QrScratch qr;
    int* tcounts;
    int* tcursor;
    double* stats;
    int* err;
    double* G;
    double* V;
    int* order;
    void* emu;
    size_t emu_bytes;
    double* z0;          // warm start: (Q^T S b)(0:n), sign-normalised like R
    TrsvCtl* ctl;        // warm start: x0 = R^-1 z0
    int* flags;
};

// The sketch always has room for one more column (S b of the warm-start factorisation).
static FactorTemp temp_carve(Carve& c, const csls_csr* A, const csls_opts* o, int64_t s) {
    FactorTemp t;
    const int64_t n = A->n;
    const int esz = o->factor_prec == CSLS_PREC_F32 ? 4 : 8;
    t.ld = round_up(s, 32);
    t.SA = c.take<char>((size_t)(t.ld * (n + 1) * esz));
    t.sk = sketch_scratch_carve(c, A->m, s);
    t.qr = qr_scratch_carve(c, s, n + 1, esz);
    t.tcounts = c.take<int>((size_t)n);
    t.tcursor = c.take<int>((size_t)n);
    t.stats = c.take<double>(4);
    t.err = c.take<int>(1);
    if (o->variant == CSLS_VARIANT_SVD) {
        t.G = c.take<double>((size_t)(n * n));
        t.V = c.take<double>((size_t)(n * n));
        t.order = c.take<int>((size_t)n + 1);
    } else {
        t.G = t.V = nullptr;
        t.order = nullptr;
    }
    t.emu = nullptr;
    t.emu_bytes = 0;
    if (o->factor_prec == CSLS_PREC_F64_EMU) {
        t.emu_bytes = qr_emu_scratch_bytes(s, n + 1);
        t.emu = c.take<char>(t.emu_bytes);
    }
    t.z0 = c.take<double>((size_t)n);
    t.ctl = c.take<TrsvCtl>(1);
    t.flags = c.take<int>((size_t)trsv_flag_ints(ceil_div(n, kTrsvBlock), n));
    return t;
}

struct SolveWs {
    LsqrState* st;
    double *ut, *vt, *z, *g, *wx, *sp_part, *lo_part, *hist;
    int *flags_up, *flags_lo;
    int64_t hist_cap;
};

static SolveWs solve_carve(Carve& c, const csls_factor_t* F) {
    SolveWs w;
    const int64_t n = F->n, m = F->m;
    w.st = c.take<LsqrState>(1);
    w.ut = c.take<double>((size_t)m);
    w.vt = c.take<double>((size_t)n);
    w.z = c.take<double>((size_t)n);
    w.g = c.take<double>((size_t)n);
    w.wx = c.take<double>((size_t)n);
    w.sp_part = c.take<double>((size_t)device_sm_count() * 8 + 64);
    w.lo_part = c.take<double>((size_t)std::max<int64_t>(F->nblocks, (int64_t)device_sm_count() * 8) + 64);
    w.hist_cap = n + 4;
    w.hist = c.take<double>((size_t)(2 * (w.hist_cap + 2)));
    w.flags_up = c.take<int>((size_t)trsv_flag_ints(F->nblocks, n));
    w.flags_lo = c.take<int>((size_t)trsv_flag_ints(F->nblocks, n));
    return w;
}

struct ApplyWs {
    TrsvCtl* ctl;
    int* flags;
    int* err;
};

static ApplyWs apply_carve(Carve& c, const csls_factor_t* F) {
    ApplyWs w;
    w.ctl = c.take<TrsvCtl>(1);
    w.flags = c.take<int>((size_t)trsv_flag_ints(F->nblocks, F->n));
    w.err = c.take<int>(1);
    return w;
}

// ------------------------------------------------------------------ host helpers

static int read_err(const int* derr, cudaStream_t st) {
    int e = 0;
    CSLS_CUDA(cudaMemcpyAsync(&e, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    return e;
}

static int solve_one(const csls_factor_t* F, const csls_csr* A, const double* b, double* x, const csls_opts* o,
                     const SolveWs& w, csls_report* rep, cudaStream_t st, int64_t* launches) {
    const int64_t n = F->n, m = F->m;
    const int64_t r = F->variant == CSLS_VARIANT_SVD ? F->r : n;
    const long long spin = o->spin_limit;
    LsqrState h{};
    h.atol = o->atol;
    h.btol = o->btol;
    h.maxit = o->maxit > 0 ? o->maxit : n;
    h.fixed = o->fixed_iters;
    h.hist_cap = w.hist_cap;
    h.cs2 = -1.0;
    h.first = 1;
    CSLS_CUDA(cudaMemcpyAsync(w.st, &h, sizeof(LsqrState), cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemsetAsync(w.flags_up, 0, sizeof(int) * (size_t)trsv_flag_count(F->nblocks, F->n), st));
    CSLS_CUDA(cudaMemsetAsync(w.flags_lo, 0, sizeof(int) * (size_t)trsv_flag_count(F->nblocks, F->n), st));
    const bool warm = o->warm_start != 0;
    if (!warm) CSLS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st));
    CSLS_CUDA(cudaMemsetAsync(w.wx, 0, sizeof(double) * (size_t)n, st));
    CSLS_CUDA(cudaMemsetAsync(w.hist, 0, sizeof(double) * (size_t)(2 * (w.hist_cap + 2)), st));
    k_check_finite<<<grid_small(m), 256, 0, st>>>(b, m, &w.st->err);
    CSLS_CUDA(cudaGetLastError());
    if (warm) {
        k_check_finite<<<grid_small(n), 256, 0, st>>>(x, n, &w.st->err);
        CSLS_CUDA(cudaGetLastError());
    }
    const int spg = spmv_grid(A);
    TrsvArgs ta{F->R, F->prec, F->Dinv, n, (int)F->nblocks, F->pack_up, F->pack_lo};
    double* hist = w.hist;
    if (warm) {
        // ||b|| for the stopping rule, then the start below runs on r0 = b - A x (the correction
        // starts at 0 and is accumulated onto x)
        CSLS_TRY(launch_spmv(A, 2, b, w.ut, w.st, w.sp_part, spg, st));
        k_keep_bnorm<<<1, 1, 0, st>>>(w.st);
        CSLS_CUDA(cudaGetLastError());
        CSLS_TRY(launch_residual(A, x, b, w.ut, st));
        *launches += 3;
    }
    const double* rhs = warm ? w.ut : b;
    // start: beta_1 u_1 = rhs ; alpha_1 v_1 = M^T A^T u_1
    CSLS_TRY(launch_spmv(A, 2, rhs, w.ut, w.st, w.sp_part, spg, st));
    CSLS_TRY(launch_spmv_t(F->AT, n, m, F->nnz, 1, w.ut, w.g, w.st, st));
    if (F->variant == CSLS_VARIANT_QR)
        CSLS_TRY(launch_trsv_lower(ta, 2, w.g, w.vt, nullptr, w.flags_lo, &w.st->lo, w.st, w.lo_part, hist, spin,
                                   &w.st->err, st));
    else
        CSLS_TRY(launch_pgemv_t(F->P, n, r, 2, w.g, w.vt, nullptr, w.st, w.lo_part, hist, st));
    *launches += 4;
    const int64_t limit = o->fixed_iters > 0 ? o->fixed_iters : h.maxit;
    const int64_t chunk = o->check_every > 0 ? o->check_every : 16;
    const bool guarded = F->prec == CSLS_PREC_F32 && o->guard_cond > 0 && o->fixed_iters <= 0;
    int64_t next_guard = 32;
    for (int64_t it = 0; it < limit + 1; it += chunk) {
        for (int64_t k = 0; k < chunk && it + k < limit; ++k) {
            if (F->variant == CSLS_VARIANT_QR)
                CSLS_TRY(launch_trsv_upper(ta, 1, w.vt, w.z, w.flags_up, &w.st->up, w.st, w.wx, x, spin, &w.st->err, st));
            else
                CSLS_TRY(launch_pgemv(F->P, n, r, 1, w.vt, w.z, w.st, w.wx, x, st));
            CSLS_TRY(launch_spmv(A, 1, w.z, w.ut, w.st, w.sp_part, spg, st));
            CSLS_TRY(launch_spmv_t(F->AT, n, m, F->nnz, 1, w.ut, w.g, w.st, st));
            if (F->variant == CSLS_VARIANT_QR)
                CSLS_TRY(launch_trsv_lower(ta, 1, w.g, w.vt, nullptr, w.flags_lo, &w.st->lo, w.st, w.lo_part, hist,
                                           spin, &w.st->err, st));
            else
                CSLS_TRY(launch_pgemv_t(F->P, n, r, 1, w.g, w.vt, nullptr, w.st, w.lo_part, hist, st));
            *launches += 4;
        }
        int done = 0;
        CSLS_CUDA(cudaMemcpyAsync(&done, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CSLS_CUDA(cudaStreamSynchronize(st));
        if (done) break;
        if (it + chunk >= limit) break;
        const int64_t k_now = std::min<int64_t>(it + chunk, w.hist_cap);
        if (guarded && k_now >= next_guard) {
            // early guard: the bidiagonal's cond only grows with k, so once it passes the
            // guard the binary32 factor is rejected without running to the iteration limit
            std::vector<double> hh((size_t)(2 * (k_now + 1) + 2));
            CSLS_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, st));
            CSLS_CUDA(cudaStreamSynchronize(st));
            if (!(bidiag_cond_hist(hh.data(), k_now) < o->guard_cond)) break;
            next_guard *= 4;
        }
    }
    k_final_x<<<grid_small(n), 256, 0, st>>>(x, w.wx, n, w.st);
    CSLS_CUDA(cudaGetLastError());
    *launches += 1;
    LsqrState out{};
    CSLS_CUDA(cudaMemcpyAsync(&out, w.st, sizeof(LsqrState), cudaMemcpyDeviceToHost, st));
    const int64_t kk = std::min<int64_t>(out.iter, w.hist_cap);
    std::vector<double> hh((size_t)(2 * (kk + 1) + 2));
    CSLS_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    const double cond = bidiag_cond_hist(hh.data(), kk);
    if (rep) {
        rep->istop = out.istop;
        rep->iterations = out.iter;
        rep->bnorm = out.bnorm;
        rep->rnorm = out.rnorm;
        rep->arnorm = out.arnorm;
        rep->anorm = std::sqrt(out.anorm2);
        rep->ynorm = out.ynorm;
        rep->cond_est = cond;
    }
    if (out.err) return out.err;
    if (F->prec == CSLS_PREC_F32 && o->guard_cond > 0 && kk > 0 && !(cond < o->guard_cond))
        return CSLS_ERR_PRECOND_GUARD;
    if (o->fixed_iters <= 0 && out.istop == 0 && out.done) return CSLS_ERR_NOT_CONVERGED;
    return CSLS_OK;
}

// Per-family QR kernel timing for one csls_factor call (opts->time_kernels).
struct KtScope {
    bool on;
    explicit KtScope(bool o) : on(o) {
        if (on) kt_install(true);
    }
    void collect(csls_report* rep) {
        if (!on) return;
        double ms[3], fl[3];
        int64_t nl[3];
        kt_collect(ms, nl, fl);
        on = false;
        if (rep)
            for (int f = 0; f < 3; ++f) {
                rep->kern_ms[f] = ms[f];
                rep->kern_launches[f] = nl[f];
                rep->kern_flop[f] = fl[f];
            }
    }
    ~KtScope() {
        if (on) collect(nullptr);
    }
};

struct EventTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit EventTimer(cudaStream_t st) : s(st) {
        if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) cudaEventRecord(a, s);
    }
    double stop() {
        if (!a || !b) return 0.0;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~EventTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace csls

// ======================================================================= C ABI

using namespace csls;

extern "C" {

const char* csls_last_cuda_error(void) { return csls::last_cuda_error(); }

const char* csls_status_string(int status) {
    switch (status) {
        case CSLS_OK: return "CSLS_OK";
        case CSLS_ERR_ARG: return "CSLS_ERR_ARG: invalid argument";
        case CSLS_ERR_RANK_DEFICIENT: return "CSLS_ERR_RANK_DEFICIENT: R has a zero or non-finite diagonal";
        case CSLS_ERR_NOT_CONVERGED: return "CSLS_ERR_NOT_CONVERGED: LSQR reached maxit";
        case CSLS_ERR_BREAKDOWN: return "CSLS_ERR_BREAKDOWN";
        case CSLS_ERR_NONFINITE: return "CSLS_ERR_NONFINITE: NaN or Inf in the data or the iteration";
        case CSLS_ERR_PRECOND_GUARD: return "CSLS_ERR_PRECOND_GUARD: binary32 factor rejected by the cond guard";
        case CSLS_ERR_TIMEOUT: return "CSLS_ERR_TIMEOUT: a bounded device wait gave up";
        case CSLS_ERR_CUDA: return "CSLS_ERR_CUDA: CUDA runtime error";
        case CSLS_ERR_WORKSPACE: return "CSLS_ERR_WORKSPACE: workspace missing, misaligned or too small";
        default: return "CSLS: unknown status";
    }
}

void csls_opts_default(csls_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->gamma = 4.0;
    o->s = 0;
    o->seed = 1;
    o->variant = CSLS_VARIANT_QR;
    o->factor_prec = CSLS_PREC_F64;
    o->rcond = 0.0;
    o->atol = 1e-12;
    o->btol = 1e-12;
    o->maxit = 0;
    o->fixed_iters = 0;
    o->guard_cond = 10.0;
    o->time_kernels = 0;
    o->spin_limit = 20000000;
    o->check_every = 16;
    o->warm_start = 0;
    o->refine = 0;
}

int csls_sketch_workspace(const csls_csr* A, int64_t s, size_t* bytes) {
    CSLS_TRY(check_csr(A));
    if (!bytes || s <= 0 || s > 2147483647LL) return CSLS_ERR_ARG;
    *bytes = sketch_scratch_bytes(A->m, s) + 256;
    return CSLS_OK;
}

int csls_sketch(const csls_csr* A, int64_t s, uint64_t seed, int prec, void* SA, int64_t ld, void* work,
                size_t work_bytes, csls_stream_t stream) {
    CSLS_TRY(check_csr(A));
    if (s <= 0 || s > 2147483647LL || ld < s || !SA) return CSLS_ERR_ARG;
    if (prec != CSLS_PREC_F64 && prec != CSLS_PREC_F32) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_sketch_workspace(A, s, &need));
    if (!work || work_bytes < need || !aligned256(work)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Carve c{(char*)work, 0, work_bytes, false};
    SketchScratch sc = sketch_scratch_carve(c, A->m, s);
    int* err = c.take<int>(1);
    CSLS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    k_validate_csr<<<grid_small(A->m), 256, 0, st>>>(A->row_ptr, A->col, A->val, A->m, A->n, A->nnz, err);
    CSLS_CUDA(cudaGetLastError());
    int e = read_err(err, st);
    if (e) return e;
    CSLS_TRY(sketch_run(A, s, seed, prec, SA, ld, sc, err, st, nullptr));
    return CSLS_OK;
}

int csls_factor_workspace(const csls_csr* A, const csls_opts* o, size_t* persist_bytes, size_t* temp_bytes) {
    CSLS_TRY(check_csr(A));
    if (!o || !persist_bytes || !temp_bytes) return CSLS_ERR_ARG;
    const int64_t s = sketch_rows(A, o);
    if (s < A->n || A->m < A->n) return CSLS_ERR_ARG;
    Carve p{nullptr, 0, 0, true};
    persist_carve(p, A, o);
    Carve t{nullptr, 0, 0, true};
    temp_carve(t, A, o, s);
    *persist_bytes = p.off;
    *temp_bytes = t.off;
    return CSLS_OK;
}

// The factorisation of csls_factor; with b (warm start, QR variant only) the sketch carries S b as
// column n, the QR runs over n + 1 columns, and x0 = R^-1 (Q^T S b)(0:n) is written to x0.
static int factor_impl(const csls_csr* A, const double* b, double* x0, const csls_opts* o, void* persist,
                       size_t persist_bytes, void* temp, size_t temp_bytes, csls_factor_t** factor, csls_report* rep,
                       csls_stream_t stream) {
    if (factor) *factor = nullptr;
    CSLS_TRY(check_csr(A));
    if (!o || !factor) return CSLS_ERR_ARG;
    if (b && (!x0 || o->variant != CSLS_VARIANT_QR || sketch_rows(A, o) < A->n + 1)) return CSLS_ERR_ARG;
    if (o->variant != CSLS_VARIANT_QR && o->variant != CSLS_VARIANT_SVD) return CSLS_ERR_ARG;
    if (o->factor_prec != CSLS_PREC_F64 && o->factor_prec != CSLS_PREC_F32 && o->factor_prec != CSLS_PREC_F64_EMU)
        return CSLS_ERR_ARG;
    if (o->variant == CSLS_VARIANT_SVD && o->factor_prec == CSLS_PREC_F32) return CSLS_ERR_ARG;
    size_t pb = 0, tb = 0;
    CSLS_TRY(csls_factor_workspace(A, o, &pb, &tb));
    if (!persist || !temp || persist_bytes < pb || temp_bytes < tb || !aligned256(persist) || !aligned256(temp))
        return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n, s = sketch_rows(A, o);
    Carve pc{(char*)persist, 0, persist_bytes, false};
    FactorPersist fp = persist_carve(pc, A, o);
    Carve tc{(char*)temp, 0, temp_bytes, false};
    FactorTemp ft = temp_carve(tc, A, o, s);
    int64_t launches = 0;
    if (rep) { std::memset(rep, 0, sizeof(*rep)); rep->s = s; }
    CSLS_CUDA(cudaMemsetAsync(ft.err, 0, sizeof(int), st));
    k_validate_csr<<<grid_small(A->m), 256, 0, st>>>(A->row_ptr, A->col, A->val, A->m, A->n, A->nnz, ft.err);
    CSLS_CUDA(cudaGetLastError());
    ++launches;
    int e = read_err(ft.err, st);
    if (e) { if (rep) rep->status = e; return e; }
    // A^T for the solve
    CSLS_TRY(transpose_build(A, fp.AT, ft.tcounts, ft.tcursor, ft.err, st, &launches));
    // sketch + QR
    EventTimer t_sk(st);
    const int sk_prec = o->factor_prec == CSLS_PREC_F32 ? CSLS_PREC_F32 : CSLS_PREC_F64;
    CSLS_TRY(sketch_run(A, s, o->seed, sk_prec, ft.SA, ft.ld, ft.sk, ft.err, st, &launches));
    const int esz = sk_prec == CSLS_PREC_F32 ? 4 : 8;
    if (b) {
        k_check_finite<<<grid_small(A->m), 256, 0, st>>>(b, A->m, ft.err);
        CSLS_CUDA(cudaGetLastError());
        CSLS_TRY(sketch_vec_run(ft.sk, b, s, o->seed, sk_prec, (char*)ft.SA + (size_t)(n * ft.ld * esz), st,
                                &launches));
        ++launches;
    }
    const int64_t ncols = b ? n + 1 : n;
    const double ms_sk = t_sk.stop();
    KtScope kts(o->time_kernels != 0);
    EventTimer t_qr(st);
    const long long spin = o->spin_limit;
    if (o->factor_prec == CSLS_PREC_F64 || o->factor_prec == CSLS_PREC_F64_EMU) {
        if (o->factor_prec == CSLS_PREC_F64)
            CSLS_TRY(qr_factor_f64((double*)ft.SA, ft.ld, s, ncols, ft.qr, ft.err, spin, st, &launches));
        else
            CSLS_TRY(qr_factor_f64_emu((double*)ft.SA, ft.ld, s, ncols, ft.qr, ft.emu, ft.emu_bytes, ft.err, spin, st,
                                       &launches));
        CSLS_TRY(qr_extract_r_f64((const double*)ft.SA, ft.ld, n, (double*)fp.R, ft.stats, st));
        CSLS_TRY(diag_block_inverses_f64((const double*)fp.R, n, fp.Dinv, st));
        if (fp.pack_up) {
            CSLS_TRY(trsv_build_packs((const double*)fp.R, n, fp.Dinv, fp.pack_up, fp.pack_lo, st));
            launches += 2;
        }
        if (b) CSLS_TRY(qr_extract_qtb_f64((const double*)ft.SA, ft.ld, n, ft.z0, st));
    } else {
        CSLS_TRY(qr_factor_f32((float*)ft.SA, ft.ld, s, ncols, ft.qr, ft.err, spin, st, &launches));
        CSLS_TRY(qr_extract_r_f32((const float*)ft.SA, ft.ld, n, (float*)fp.R, ft.stats, st));
        CSLS_TRY(diag_block_inverses_f32((const float*)fp.R, n, fp.Dinv, st));
        if (b) CSLS_TRY(qr_extract_qtb_f32((const float*)ft.SA, ft.ld, n, ft.z0, st));
    }
    if (b) {
        // x0 = R^-1 z0: the minimiser of ||S (A x - b)|| (Remark 3.1's y0 = Q^T S b, x0 = R^-1 y0)
        TrsvArgs ta{fp.R, o->factor_prec == CSLS_PREC_F32 ? CSLS_PREC_F32 : CSLS_PREC_F64, fp.Dinv, n,
                    (int)ceil_div(n, kTrsvBlock), fp.pack_up, fp.pack_lo};
        CSLS_CUDA(cudaMemsetAsync(ft.ctl, 0, sizeof(TrsvCtl), st));
        CSLS_CUDA(cudaMemsetAsync(ft.flags, 0, sizeof(int) * (size_t)trsv_flag_count(ta.nb, n), st));
        CSLS_TRY(launch_trsv_upper(ta, 0, ft.z0, x0, ft.flags, ft.ctl, nullptr, nullptr, nullptr, spin, ft.err, st));
        launches += 2;
    }
    launches += 3;
    int64_t r = n;
    if (o->variant == CSLS_VARIANT_SVD) {
        // default RCOND = max(s, n) x the unit roundoff of the factorisation: 2^-53 for binary64, 2^-38 for
        // the emulated products (their relative error per product), so that the noise the emulation leaves
        // in numerically zero singular values is truncated
        const double eps = o->factor_prec == CSLS_PREC_F64_EMU ? 3.637978807091713e-12 : 1.1102230246251565e-16;
        const double rc = o->rcond > 0 ? o->rcond : (double)std::max(s, n) * eps;
        CSLS_TRY(svd_precond((const double*)fp.R, n, rc, ft.G, ft.V, fp.sigma, fp.P, ft.order, &r, ft.qr.bar, spin,
                             ft.err, st, &launches));
    }
    const double ms_qr = t_qr.stop();
    kts.collect(rep);
    double stats[4] = {0, 0, 0, 0};
    CSLS_CUDA(cudaMemcpyAsync(stats, ft.stats, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    e = read_err(ft.err, st);
    if (rep) {
        rep->ms_sketch = ms_sk;
        rep->ms_factor = ms_qr;
        rep->rdiag_min = stats[0];
        rep->rdiag_max = stats[1];
        rep->r = r;
        rep->launches = launches;
        rep->status = e;
    }
    if (e) return e;
    if (o->variant == CSLS_VARIANT_QR && stats[2] > 0) {
        if (rep) rep->status = CSLS_ERR_RANK_DEFICIENT;
        return CSLS_ERR_RANK_DEFICIENT;
    }
    if (o->variant == CSLS_VARIANT_SVD && r == 0) return CSLS_ERR_RANK_DEFICIENT;
    csls_factor_t* F = new (std::nothrow) csls_factor_t;
    if (!F) return CSLS_ERR_ARG;
    F->m = A->m; F->n = n; F->nnz = A->nnz; F->s = s; F->r = r;
    F->variant = o->variant;
    F->prec = o->factor_prec == CSLS_PREC_F32 ? CSLS_PREC_F32 : CSLS_PREC_F64;   // storage type of R
    F->R = fp.R; F->Dinv = fp.Dinv; F->P = fp.P; F->AT = fp.AT;
    F->pack_up = fp.pack_up; F->pack_lo = fp.pack_lo;
    F->rdiag_min = stats[0]; F->rdiag_max = stats[1];
    F->nblocks = ceil_div(n, kTrsvBlock);
    F->a_col = A->col;
    F->spmv_group = 0;
    F->spmv_group_t = 0;
    *factor = F;
    return CSLS_OK;
}

int csls_factor(const csls_csr* A, const csls_opts* o, void* persist, size_t persist_bytes, void* temp,
                size_t temp_bytes, csls_factor_t** factor, csls_report* rep, csls_stream_t stream) {
    return factor_impl(A, nullptr, nullptr, o, persist, persist_bytes, temp, temp_bytes, factor, rep, stream);
}

int csls_factor_warm(const csls_csr* A, const double* b, const csls_opts* o, void* persist, size_t persist_bytes,
                     void* temp, size_t temp_bytes, csls_factor_t** factor, double* x0, csls_report* rep,
                     csls_stream_t stream) {
    if (!b || !x0) return CSLS_ERR_ARG;
    return factor_impl(A, b, x0, o, persist, persist_bytes, temp, temp_bytes, factor, rep, stream);
}

int csls_factor_destroy(csls_factor_t* F) {
    delete F;
    return CSLS_OK;
}

int csls_factor_view(const csls_factor_t* F, int64_t* n, int64_t* s, int64_t* r, int* variant, int* prec,
                     const void** R, const double** P) {
    if (!F) return CSLS_ERR_ARG;
    if (n) *n = F->n;
    if (s) *s = F->s;
    if (r) *r = F->r;
    if (variant) *variant = F->variant;
    if (prec) *prec = F->prec;
    if (R) *R = F->R;
    if (P) *P = F->P;
    return CSLS_OK;
}

static int check_factor_matches(const csls_factor_t* F, const csls_csr* A) {
    if (!F || !A) return CSLS_ERR_ARG;
    CSLS_TRY(check_csr(A));
    if (A->m != F->m || A->n != F->n || A->nnz != F->nnz) return CSLS_ERR_ARG;
    return CSLS_OK;
}

int csls_apply_workspace(const csls_factor_t* F, size_t* bytes) {
    if (!F || !bytes) return CSLS_ERR_ARG;
    Carve c{nullptr, 0, 0, true};
    apply_carve(c, F);
    *bytes = c.off;
    return CSLS_OK;
}

int csls_precond_apply(const csls_factor_t* F, int trans, const double* v, double* z, void* work, size_t work_bytes,
                       csls_stream_t stream) {
    if (!F || !v || !z || v == z) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_apply_workspace(F, &need));
    if (!work || work_bytes < need || !aligned256(work)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Carve c{(char*)work, 0, work_bytes, false};
    ApplyWs w = apply_carve(c, F);
    CSLS_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(TrsvCtl), st));
    CSLS_CUDA(cudaMemsetAsync(w.flags, 0, sizeof(int) * (size_t)trsv_flag_count(F->nblocks, F->n), st));
    CSLS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    if (F->variant == CSLS_VARIANT_QR) {
        TrsvArgs ta{F->R, F->prec, F->Dinv, F->n, (int)F->nblocks, F->pack_up, F->pack_lo};
        if (!trans) {
            CSLS_TRY(launch_trsv_upper(ta, 0, v, z, w.flags, w.ctl, nullptr, nullptr, nullptr, 20000000LL, w.err, st));
        } else {
            CSLS_CUDA(cudaMemcpyAsync(z, v, sizeof(double) * (size_t)F->n, cudaMemcpyDeviceToDevice, st));
            CSLS_TRY(launch_trsv_lower(ta, 0, z, nullptr, z, w.flags, w.ctl, nullptr, nullptr, nullptr, 20000000LL, w.err, st));
        }
    } else {
        if (!trans) CSLS_TRY(launch_pgemv(F->P, F->n, F->r, 0, v, z, nullptr, nullptr, nullptr, st));
        else CSLS_TRY(launch_pgemv_t(F->P, F->n, F->r, 0, v, nullptr, z, nullptr, nullptr, nullptr, st));
    }
    return read_err(w.err, st);
}

int csls_spmv(const csls_factor_t* F, const csls_csr* A, int trans, const double* x, double* y, csls_stream_t stream) {
    CSLS_TRY(check_factor_matches(F, A));
    if (!x || !y) return CSLS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!trans) CSLS_TRY(launch_spmv(A, 0, x, y, nullptr, nullptr, spmv_grid(A), st));
    else CSLS_TRY(launch_spmv_t(F->AT, F->n, F->m, F->nnz, 0, x, y, nullptr, st));
    return CSLS_OK;
}

int csls_read_probe(const void* buf, int64_t count, int ctas_per_sm, int unroll, unsigned long long* partials,
                    csls_stream_t stream) {
    if ((!buf && count > 0) || !partials || count < 0 || ((uintptr_t)buf & 15) != 0 || ctas_per_sm < 1 || ctas_per_sm > 4 ||
        (unroll != 1 && unroll != 2 && unroll != 4 && unroll != 8))
        return CSLS_ERR_ARG;
    return csls::launch_read_probe(buf, count, ctas_per_sm, unroll, partials, (cudaStream_t)stream);
}

int csls_solve_workspace(const csls_factor_t* F, int64_t nrhs, size_t* bytes) {
    if (!F || !bytes || nrhs <= 0) return CSLS_ERR_ARG;
    Carve c{nullptr, 0, 0, true};
    solve_carve(c, F);
    size_t need = c.off;
    if (nrhs > 1 && F->variant == CSLS_VARIANT_QR)
        need = std::max(need, block_ws_bytes(F->m, F->n, F->nblocks, std::min(nrhs, kBlockMax)) +
                                  block_refine_bytes(F->m, F->n, std::min(nrhs, kBlockMax)));
    *bytes = need;
    return CSLS_OK;
}

int csls_solve(const csls_factor_t* F, const csls_csr* A, const double* b, int64_t nrhs, int64_t ldb, double* x,
               int64_t ldx, const csls_opts* o, void* work, size_t work_bytes, csls_report* rep,
               csls_stream_t stream) {
    CSLS_TRY(check_factor_matches(F, A));
    if (!o || !b || !x || nrhs <= 0 || ldb < F->m || ldx < F->n) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_solve_workspace(F, nrhs, &need));
    if (!work || work_bytes < need || !aligned256(work)) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Carve c{(char*)work, 0, work_bytes, false};
    SolveWs w = solve_carve(c, F);
    if (rep) std::memset(rep, 0, sizeof(*rep));
    EventTimer t(st);
    int64_t launches = 0, max_it = 0;
    int status = CSLS_OK;
    if (nrhs > 1 && F->variant == CSLS_VARIANT_QR && !o->warm_start) {
        // block form: independent recurrences sharing each pass over A and R (a warm start runs the
        // columns one by one below, each from its own x)
        for (int64_t k0 = 0; k0 < nrhs; k0 += kBlockMax) {
            const int64_t nk = std::min(kBlockMax, nrhs - k0);
            csls_report rk{};
            int sk = block_solve_refined(F, A, b + k0 * ldb, nk, ldb, x + k0 * ldx, ldx, o, work, work_bytes, &rk, st,
                                 &launches);
            if (k0 == 0 && rep) *rep = rk;
            max_it = std::max<int64_t>(max_it, rk.iterations);
            if (status == CSLS_OK && sk != CSLS_OK) status = sk;
            if (sk == CSLS_ERR_CUDA || sk == CSLS_ERR_TIMEOUT) break;
        }
    } else {
        for (int64_t k = 0; k < nrhs; ++k) {
            csls_report rk{};
            int sk = solve_one(F, A, b + k * ldb, x + k * ldx, o, w, &rk, st, &launches);
            int64_t its = rk.iterations, its_ref = 0;
            // restarts: LSQR again from the x just found, on the correction from r = b - A x
            csls_opts orf = *o;
            orf.warm_start = 1;
            for (int64_t p = 0; p < o->refine && (sk == CSLS_OK || sk == CSLS_ERR_NOT_CONVERGED); ++p) {
                csls_report rr{};
                sk = solve_one(F, A, b + k * ldb, x + k * ldx, &orf, w, &rr, st, &launches);
                its_ref += rr.iterations;
                rr.bnorm = rk.bnorm;   // of the original right-hand side
                rr.cond_est = std::max(rr.cond_est, rk.cond_est);   // the longer bidiagonal bounds it better
                rk = rr;
            }
            its += its_ref;
            rk.iterations = its;
            rk.iterations_refine = its_ref;
            if (k == 0 && rep) *rep = rk;
            max_it = std::max<int64_t>(max_it, its);
            if (status == CSLS_OK && sk != CSLS_OK) status = sk;
            if (sk == CSLS_ERR_CUDA || sk == CSLS_ERR_TIMEOUT) break;
        }
    }
    const double ms = t.stop();
    if (rep) {
        rep->iterations = max_it;   // first right-hand side's refine count stays as reported
        rep->ms_solve = ms;
        rep->launches = launches;
        rep->s = F->s;
        rep->r = F->r;
        rep->rdiag_min = F->rdiag_min;
        rep->rdiag_max = F->rdiag_max;
        rep->status = status;
    }
    return status;
}

int csls_backward_workspace(const csls_factor_t* F, size_t* bytes) {
    if (!F || !bytes) return CSLS_ERR_ARG;
    *bytes = backward_ws_bytes(F->m, F->n, F->nblocks);
    return CSLS_OK;
}

}  // extern "C"


// Internal declarations shared by the csls CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "csls.h"

#define CSLS_TRY(expr)                                  \
    do {                                                \
        int csls_rc_ = (expr);                          \
        if (csls_rc_ != CSLS_OK) return csls_rc_;       \
    } while (0)

namespace csls {
void note_cuda_error(cudaError_t e, const char* where);   // kept per host thread for csls_last_cuda_error
const char* last_cuda_error();
}
#define CSLS_STR2_(x) #x
#define CSLS_STR_(x) CSLS_STR2_(x)
#define CSLS_CUDA(expr)                                                            \
    do {                                                                           \
        cudaError_t csls_ce_ = (expr);                                             \
        if (csls_ce_ != cudaSuccess) {                                             \
            csls::note_cuda_error(csls_ce_, __FILE__ ":" CSLS_STR_(__LINE__));     \
            return CSLS_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

namespace csls {

constexpr int kWarp = 32;
constexpr int kTrsvBlock = 64;      // diagonal block size of the blocked triangular solves
constexpr int kPanel = 32;          // Householder panel width

// ------------------------------------------------------------------ device helpers

// First error wins; later codes are dropped.
__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire_u(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// SplitMix64 output function (Steele, Lea and Flood 2014).
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Barrier for a grid whose blocks are all co-resident (cooperative launch).
// Waits are bounded by spin_limit; on timeout the error word is set and the
// function returns false (callers then return without touching shared data).
struct GridBarrier {
    unsigned count;
    unsigned gen;
};

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned nblocks, long long spin_limit,
                                          int* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g = ld_acquire_u(&bar->gen);
        __threadfence();
        unsigned prev = atomicAdd(&bar->count, 1u);
        if (prev == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            st_release_u(&bar->gen, g + 1u);
        } else {
            long long it = 0;
            while (ld_acquire_u(&bar->gen) == g) {
                if (++it > spin_limit) {
                    set_error(err, CSLS_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok && (*(volatile int*)err != CSLS_ERR_TIMEOUT);
    }
    __syncthreads();
    return ok_s != 0;
}

// Barrier for a co-resident grid on a counter that only grows: every CTA adds 1 (a release
// reduction, no returned value, so the G arrivals pipeline in the L2 instead of serialising on
// a read-modify-write round trip each) and waits until the counter reaches G x (k + 1) for its
// k-th barrier. The counter must start at 0 for the launch (the caller gives each launch a zeroed
// slot). Bounded by spin_limit like grid_sync.
__device__ __forceinline__ bool grid_sync_count(unsigned* cnt, unsigned nblocks, unsigned k, long long spin_limit,
                                                int* err) {
    __shared__ int okc_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(cnt), "r"(1u) : "memory");
        const unsigned target = nblocks * (k + 1u);
        long long it = 0;
        while (ld_acquire_u(cnt) < target) {
            if (++it > spin_limit) {
                set_error(err, CSLS_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            if (it > 256) __nanosleep(32);
        }
        okc_s = ok && (*(volatile int*)err != CSLS_ERR_TIMEOUT);
    }
    __syncthreads();
    return okc_s != 0;
}

// Deterministic block-wide sum (fixed shuffle tree, then warps in order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch /* NT/32 doubles */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) t += scratch[i];
    }
    return t;  // valid in thread 0 only
}

// ------------------------------------------------------------------ host helpers

struct Carve {
    char* base;
    size_t off;
    size_t cap;
    bool counting;  // true: only measure
    template <class T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
        T* p = counting ? nullptr : reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
    bool fits() const { return counting || off <= cap; }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

int device_sm_count();   // of the current device (cached per device)
// Raises a kernel's dynamic shared-memory limit to `bytes` on the current device, once per
// (kernel, device) pair (the attribute is per device); thread-safe.
int raise_smem_limit(const void* kernel, int bytes);

// Optional per-family kernel timing for the factorisation: while timing is on for the
// calling thread, launch sites bracket their kernels with events on the launching
// stream; kt_collect sums the intervals once the stream has drained.
enum { kFamPanel = 0, kFamVtc = 1, kFamUpdate = 2 };
void kt_install(bool on);
int kt_begin(int fam, cudaStream_t st);               // token for kt_end; -1 when timing is off
void kt_end(int token, double flop, cudaStream_t st);
void kt_collect(double ms[3], int64_t launches[3], double flop[3]);   // call after a stream sync; turns timing off

// ------------------------------------------------------------------ building blocks (host launchers)

// Exclusive scan of `len` int32 counts into out[0..len] (out[len] = total), int64 output.
int scan_counts(const int* counts, int64_t* out, int64_t len, cudaStream_t st);

// Sort each segment [off[k], off[k+1]) of (key, payload) ascending by key.
// keys are non-negative int32 (compared as given); payload may be NULL.
int segmented_sort(int32_t* keys, int32_t* payload, const int64_t* off, int64_t nseg, int64_t max_hint,
                   cudaStream_t st);

// Count sketch pieces
struct SketchScratch {
    int* counts;        // s
    int64_t* offsets;   // s + 1
    int* cursor;        // s
    int32_t* list;      // m   (row | sign << 31)
};
size_t sketch_scratch_bytes(int64_t m, int64_t s);
SketchScratch sketch_scratch_carve(Carve& c, int64_t m, int64_t s);
int sketch_run(const csls_csr* A, int64_t s, uint64_t seed, int prec, void* SA, int64_t ld,
               const SketchScratch& sc, int* err, cudaStream_t st, int64_t* launches);
// S b (s entries, binary64 or binary32 by prec) from the bucket lists left by sketch_run.
int sketch_vec_run(const SketchScratch& sc, const double* b, int64_t s, uint64_t seed, int prec, void* out,
                   cudaStream_t st, int64_t* launches);

// Transpose of A (CSR of A^T) with the permutation back to A's nonzeros.
struct Transpose {
    int64_t* row_ptr;   // n + 1
    int32_t* col;       // nnz (row index of A)
    double* val;        // nnz
    int32_t* perm;      // nnz: position in A
};
int transpose_build(const csls_csr* A, Transpose& T, int* counts /* n */, int* cursor /* n */,
                    int* err, cudaStream_t st, int64_t* launches);
int transpose_gather_values(const csls_csr* A, const Transpose& T, cudaStream_t st);

// Householder QR of an s x n column-major matrix (s >= n), in place.
struct QrScratch {
    double* tau;        // n
    double* T;          // kPanel^2
    double* partials;   // panel reductions
    double* Wp;         // split-K partials of V^T C
    double* Wn;         // -T^T V^T C  (kPanel x n)
    GridBarrier* bar;
    int64_t wp_elems;
    int64_t part_elems;
};
size_t qr_scratch_bytes(int64_t s, int64_t n, int elem_bytes);
QrScratch qr_scratch_carve(Carve& c, int64_t s, int64_t n, int elem_bytes);
int qr_factor_f64(double* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, int* err,
                  long long spin_limit, cudaStream_t st, int64_t* launches);
int qr_factor_f32(float* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, int* err,
                  long long spin_limit, cudaStream_t st, int64_t* launches);
// The FP64 (DMMA) update of columns [j0 + nbw, n_end) by the panel at j0 whose T is in q.T
// (used inside the emulated path's outer blocks; not timed by the kernel timer).
int qr_trailing_update_f64(double* A, int64_t lda, int64_t s, int64_t n_end, int64_t j0, int nbw, const QrScratch& q,
                           cudaStream_t st);
// The same factorisation with the trailing-update products emulated exactly on the bf16
// tensor cores (digit splitting, int64 fixed-point trailing matrix); needs emu scratch.
size_t qr_emu_scratch_bytes(int64_t s, int64_t n);
int64_t obpanel_partial_elems(int sms);   // doubles the emulated path's panel needs in QrScratch::partials
int qr_factor_f64_emu(double* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, void* emu_work,
                      size_t emu_bytes, int* err, long long spin, cudaStream_t st, int64_t* launches);
// R (n x n, ld n, non-negative diagonal, zero below) from the factored matrix; stats[0..2] =
// min |R_jj|, max |R_jj|, count of zero or non-finite diagonal entries.
int qr_extract_r_f64(const double* A, int64_t lda, int64_t n, double* R, double* stats, cudaStream_t st);
int qr_extract_r_f32(const float* A, int64_t lda, int64_t n, float* R, double* stats, cudaStream_t st);
// (Q^T S b)(0:n) from column n of a factored augmented sketch, sign-normalised like R.
int qr_extract_qtb_f64(const double* A, int64_t lda, int64_t n, double* z, cudaStream_t st);
int qr_extract_qtb_f32(const float* A, int64_t lda, int64_t n, double* z, cudaStream_t st);

// Inverses of the kTrsvBlock diagonal blocks of R, in double (NB blocks of 64 x 64).
int diag_block_inverses_f64(const double* R, int64_t n, double* Dinv, cudaStream_t st);
int diag_block_inverses_f32(const float* R, int64_t n, double* Dinv, cudaStream_t st);

// Jacobi SVD of R (n x n): sigma (desc), V (n x n), P = V_r Sigma_r^{-1}; returns r in *r_out (host).
int svd_precond(const double* R, int64_t n, double rcond, double* work_G, double* work_V, double* sigma,
                double* P, int* order, int64_t* r_out, GridBarrier* bar, long long spin, int* err, cudaStream_t st,
                int64_t* launches);

}  // namespace csls

// The factor handle (host memory; device pointers inside point into caller workspace).
struct csls_factor_s {
    int64_t m, n, nnz, s, r;
    int variant, prec;
    void* R;               // n x n, ld n (double or float)
    double* Dinv;          // ceil(n/64) blocks of 64 x 64
    double* pack_up;       // operand packs of the cluster-chain triangular solves (binary64 R, QR)
    double* pack_lo;
    double* P;             // n x r (SVD)
    csls::Transpose AT;
    double rdiag_min, rdiag_max;
    int64_t nblocks;       // ceil(n/64)
    const int32_t* a_col;  // identity of the matrix the factor was built from
    int spmv_group;        // threads per row for A x (0: heuristic), set by the autotuner
    int spmv_group_t;      // threads per row for A^T u
};

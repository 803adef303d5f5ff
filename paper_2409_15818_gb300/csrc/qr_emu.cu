// Blocked Householder QR of the sketch with the trailing-matrix products done on
// the bf16 tensor cores at FP64-level accuracy (Algorithm 1 step 3).
//
// GB300 runs FP64 MMA at ~1.1 TFLOP/s but bf16 mma.sync at ~600 TFLOP/s, so the two
// products of every trailing update (W = V^T C and C += V Wn) are computed from
// exact integer pieces, in the spirit of Ozaki, Ogita, Oishi and Rump's
// error-free splitting of matrix products:
//   * every operand entry is written as a signed integer of 47 bits relative to a
//     power-of-two scale shared along the contraction (per row of the left
//     operand, per column of the right one) and cut into 6 balanced base-256
//     digits in [-128, 128], each exact in bf16;
//   * digit-plane products are exact integers below 2^14, and a sum of at most
//     6 x 32 of them stays below 2^22, so the FP32 accumulation of mma.sync
//     (started from 1.5 * 2^23, where the float grid is the integers) is exact; digit pairs of the same weight (level l = p + q) share one
//     accumulator; levels 0..5 are kept (21 of 36 pairs), the dropped ones weigh
//     2^-48 of the leading term;
//   * levels are combined in int64.
// The trailing matrix is held in int64 fixed point per column: value =
// Cfix * 2^(E_c - 62) with 2^E_c above the column's 2-norm. Orthogonal updates
// never increase the norm of a trailing column, so the scale is fixed for the
// whole factorisation and C += V Wn is an exact integer addition -- the update
// never touches the FP64 pipe. A column switches to FP64 (in place, same bytes)
// when it becomes part of a panel; the panel is factored in FP64 by k_panel.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "csls_internal.cuh"
#include "tc.cuh"

namespace csls {

constexpr int kDig = 6;          // digits per operand
constexpr int kLev = 5;          // highest kept level p + q
constexpr int kFixBits = 62;     // fixed-point fraction bits of the trailing matrix
constexpr int kNumBits = 8 * kDig - 1;   // integer bits of an operand before cutting into digits (47)
constexpr int kVtcStep = 32;     // rows per exact FP32 accumulation in W = V^T C
// FP32 accumulators start at 1.5 * 2^23: while |sum| < 2^22 the integer sum sits exactly in the
// low mantissa bits, so it is read back with one integer subtraction (no conversion instruction).
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;
constexpr int kEmuThreads = 256;

// ------------------------------------------------------------------ digit helpers

__device__ __forceinline__ int exp_of(double amax) {
    // smallest e with amax < 2^e (amax > 0), else 0
    return amax > 0.0 ? ilogb(amax) + 1 : 0;
}

// Balanced base-256 digits of |N| < 2^47: N = sum_q d[q] 256^(5 - q), d[1..5] in [-128, 127], d[0] in
// [-128, 128]. Adding 128 to each of the five low bytes (0x8080808080) removes the borrow chain of digit
// by digit extraction: each low digit is then a plain byte of the sum minus 128, and the top digit is the
// sum shifted right by 40 (arithmetic).
static_assert(kDig == 6 && kNumBits == 47, "cut_digits is written for six digits of a 47-bit integer");
__device__ __forceinline__ void cut_digits(long long N, int (&d)[kDig]) {
    const long long M = N + 0x8080808080LL;
    const unsigned lo = (unsigned)M;
    const int hi = (int)(M >> 32);
    d[5] = (int)(lo & 255u) - 128;
    d[4] = (int)((lo >> 8) & 255u) - 128;
    d[3] = (int)((lo >> 16) & 255u) - 128;
    d[2] = (int)(lo >> 24) - 128;
    d[1] = (hi & 255) - 128;
    d[0] = hi >> 8;
}

// digits of x relative to scale 2^e (|x| < 2^e)
__device__ __forceinline__ void digits_f64(double x, int e, int (&d)[kDig]) {
    const long long N = __double2ll_rn(ldexp(x, kNumBits - e));
    cut_digits(N, d);
}

// digits of a fixed-point entry (|Cfix| < 2^62): N = round(Cfix / 2^(62 - 47))
__device__ __forceinline__ void digits_fix(long long c, int (&d)[kDig]) {
    const long long N = (c + (1LL << (kFixBits - kNumBits - 1))) >> (kFixBits - kNumBits);
    cut_digits(N, d);
}

__device__ __forceinline__ unsigned short bf16_of_int(int v) {
    // |v| <= 128: exactly representable. int -> float by the same magic-number trick
    // (one integer add, one float subtract), then the top 16 bits are the bf16 pattern.
    const float f = __int_as_float(kMagicBits + v) - kMagic;
    return (unsigned short)(__float_as_uint(f) >> 16);
}

__device__ __forceinline__ int magic_to_int(float acc) { return __float_as_int(acc) - kMagicBits; }

__device__ __forceinline__ void hmma(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Four 8x8 b16 matrices from shared memory in the mma.sync fragment order; `row` is this
// lane's row address.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* row) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// ------------------------------------------------------------------ setup kernels

// E_c = exponent bound of column c of SA: 2^E_c > ||SA(:, c)||_2 >= every |entry| at any later stage.
__global__ void __launch_bounds__(256) k_col_exponent(const double* A, int64_t lda, int64_t s, int64_t n, int* E) {
    __shared__ double red[8];
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
        const double* col = A + c * lda;
        double acc = 0.0;
        for (int64_t r = threadIdx.x; r < s; r += 256) acc += col[r] * col[r];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red[w];
            const double nrm = sqrt(t) * (1.0 + 1e-12);
            E[c] = nrm > 0.0 ? ilogb(nrm) + 1 : -1000;
        }
        __syncthreads();
    }
}

// In place: SA (double) -> fixed point (int64) per column.
__global__ void k_to_fixed(double* A, int64_t lda, int64_t s, int64_t n, const int* E) {
    for (int64_t c = blockIdx.y; c < n; c += gridDim.y) {
        const int sh = kFixBits - E[c];
        long long* colf = reinterpret_cast<long long*>(A + c * lda);
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s; r += (int64_t)gridDim.x * blockDim.x) {
            const double v = A[r + c * lda];
            colf[r] = E[c] > -1000 ? __double2ll_rn(ldexp(v, sh)) : 0LL;
        }
    }
}

// In place: panel columns [j0, j0 + nbw), rows [j0, s): fixed point -> double.
__global__ void k_panel_to_f64(double* A, int64_t lda, int64_t s, int64_t j0, int nbw, const int* E) {
    for (int64_t c = j0 + blockIdx.y; c < j0 + nbw; c += gridDim.y) {
        const int sh = E[c] - kFixBits;
        long long* colf = reinterpret_cast<long long*>(A + c * lda);
        for (int64_t r = j0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
             r += (int64_t)gridDim.x * blockDim.x)
            A[r + c * lda] = E[c] > -1000 ? ldexp((double)colf[r], sh) : 0.0;
    }
}

// Rows above the trailing block in the not-yet-factored columns also hold fixed point
// (rows [0, j0) of columns >= j0 are final R entries): convert those rows of the panel too.
__global__ void k_panel_top_to_f64(double* A, int64_t lda, int64_t j0, int nbw, const int* E) {
    const int64_t c = j0 + blockIdx.y;
    if (c >= j0 + nbw) return;
    const int sh = E[c] - kFixBits;
    long long* colf = reinterpret_cast<long long*>(A + c * lda);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < j0; r += (int64_t)gridDim.x * blockDim.x)
        A[r + c * lda] = E[c] > -1000 ? ldexp((double)colf[r], sh) : 0.0;
}

// ------------------------------------------------------------------ outer-block digit kernels
//
// The emulated products act on outer blocks of kOB = 64 columns: two 32-wide panels are
// factored in binary64 (the second after the first one's update, on the FP64 MMA pipe),
// their compact-WY factors are merged, and the trailing matrix is updated once per 64
// columns. A product with K = 64 keeps every level sum below 6 x 64 x 2^14 < 2^24, so it
// is exact in FP32 and is read back with one rounding conversion per level.

constexpr int kOB = 2 * kPanel;   // 64

// Tiles of the tcgen05 update C += V Wn: 128 rows (one TMEM lane each) x 32 columns. Its digit
// planes are stored tile by tile (the 6 planes of a tile contiguous) in the canonical K-major
// core-matrix order, so that one bulk copy moves a tile's planes into shared memory ready for
// the MMA: in a V plane the 16-byte chunk holding row r, columns 8 kg .. 8 kg + 7 sits at chunk
// index kg x 128 + r (Wn planes: kg x 32 + c).
constexpr int kTcM = 128;
constexpr int kTcN = 32;
__device__ __forceinline__ int64_t vd_chunk(int p, int64_t lr, int kg) {
    return (((lr >> 7) * kDig + p) * 8 + kg) * kTcM + (lr & (kTcM - 1));
}
__device__ __forceinline__ int64_t wd_chunk(int q, int64_t c, int kg) {
    return (((c >> 5) * kDig + q) * 8 + kg) * kTcN + (c & (kTcN - 1));
}

// Masked Householder vector entry of the outer block starting at J0: 0 above the diagonal,
// 1 on it, the stored tail below.
__device__ __forceinline__ double vmask(const double* A, int64_t lda, int64_t r, int64_t J0, int a) {
    const int64_t d = J0 + a;
    return r < d ? 0.0 : (r == d ? 1.0 : A[r + d * lda]);
}

// Column maxima of V (for the V^T C digits), as ordered bit patterns (|x| >= 0).
__global__ void __launch_bounds__(256) k_vcolmax(const double* A, int64_t lda, int64_t s, int64_t J0, int nbo,
                                                 unsigned long long* colmax) {
    __shared__ unsigned long long red[kOB];
    if (threadIdx.x < kOB) red[threadIdx.x] = 0ULL;
    __syncthreads();
    const int a = threadIdx.x & (kOB - 1);
    unsigned long long best = 0ULL;
    if (a < nbo) {
        for (int64_t r = J0 + blockIdx.x * 4 + (threadIdx.x >> 6); r < s; r += (int64_t)gridDim.x * 4) {
            const unsigned long long b = __double_as_longlong(fabs(vmask(A, lda, r, J0, a)));
            best = b > best ? b : best;
        }
        atomicMax(&red[a], best);
    }
    __syncthreads();
    if (threadIdx.x < nbo) atomicMax(&colmax[threadIdx.x], red[threadIdx.x]);
}

// Digits of V: per-row scale for C += V Wn (Vd: plane tiles of 128 rows in core-matrix order,
// ldv a multiple of 128) and per-column scale for V^T C (VTd[p][a][r], r contiguous). Rows are
// local row indices r - J0; columns a >= nbo and rows past the block are zero digits.
__global__ void __launch_bounds__(256) k_vdigits(const double* A, int64_t lda, int64_t s, int64_t J0, int nbo,
                                                 const unsigned long long* colmax, int64_t ldv,
                                                 unsigned short* Vd, unsigned short* VTd, int* frow, int* ecol) {
    __shared__ int ecol_s[kOB];
    if (threadIdx.x < kOB) {
        const int e = threadIdx.x < nbo ? exp_of(__longlong_as_double((long long)colmax[threadIdx.x])) : 0;
        ecol_s[threadIdx.x] = e;
        if (blockIdx.x == 0) ecol[threadIdx.x] = e;
    }
    __syncthreads();
    const int64_t L = s - J0;
    for (int64_t lr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lr < ldv; lr += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = J0 + lr;
        double mx = 0.0;
        for (int a = 0; a < nbo; ++a)
            if (lr < L) mx = fmax(mx, fabs(vmask(A, lda, r, J0, a)));
        const int f = exp_of(mx);
        frow[lr] = f;
        // the row-scaled digits of 8 consecutive columns go out as one 16-byte chunk per plane
        // (consecutive rows are consecutive chunks); the column-scaled planes are written entry by
        // entry, consecutive across the threads
        for (int a0 = 0; a0 < kOB; a0 += 8) {
            uint32_t pk[kDig][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int a = a0 + j;
                const double v = (lr < L && a < nbo) ? vmask(A, lda, r, J0, a) : 0.0;
                int d[kDig], dt[kDig];
                digits_f64(v, f, d);
                digits_f64(v, ecol_s[a], dt);
#pragma unroll
                for (int p = 0; p < kDig; ++p) {
                    const uint32_t h = bf16_of_int(d[p]);
                    if (j & 1) pk[p][j >> 1] |= h << 16;
                    else pk[p][j >> 1] = h;
                    VTd[((int64_t)p * kOB + a) * ldv + lr] = bf16_of_int(dt[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < kDig; ++p)
                reinterpret_cast<uint4*>(Vd)[vd_chunk(p, lr, a0 >> 3)] =
                    make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
        }
    }
}

// Wn = -T^T (sum of the split-K partials of W = V^T C) for the outer block (T: nbo x nbo upper
// triangular, column-major with ld kOB); Wp[k] and Wn are kOB x nprime row-major. A CTA owns 64
// columns: it sums their partials (coalesced along the columns) into shared memory, then each
// thread forms entries of -T^T W from the shared copies of T and W.
constexpr int kWrCols = 64;
constexpr size_t kWrSmem = sizeof(double) * (kOB * kOB + kOB * kWrCols);

__global__ void __launch_bounds__(256) k_wreduce_ob(const double* Wp, int ks, const double* Tb, int nbo, double* Wn,
                                                    int64_t nprime) {
    extern __shared__ __align__(16) unsigned char wr_raw[];
    double* Ts = reinterpret_cast<double*>(wr_raw);   // [b + a kOB]
    double* Ws = Ts + kOB * kOB;                      // [b][cl]
    const int64_t c0 = (int64_t)blockIdx.x * kWrCols;
    for (int i = threadIdx.x; i < kOB * kOB; i += blockDim.x) Ts[i] = Tb[i];
    for (int i = threadIdx.x; i < kOB * kWrCols; i += blockDim.x) {
        const int b = i / kWrCols, cl = i % kWrCols;
        const int64_t c = c0 + cl;
        double t = 0.0;
        if (b < nbo && c < nprime)
            for (int k = 0; k < ks; ++k) t += Wp[((int64_t)k * kOB + b) * nprime + c];
        Ws[i] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOB * kWrCols; i += blockDim.x) {
        const int a = i / kWrCols, cl = i % kWrCols;
        const int64_t c = c0 + cl;
        if (a >= nbo || c >= nprime) continue;
        double t = 0.0;
        for (int b = 0; b <= a; ++b) t += Ts[b + a * kOB] * Ws[b * kWrCols + cl];
        Wn[(int64_t)a * nprime + c] = -t;
    }
}

// Digits of Wn (kOB x nprime, row-major): per-column scale; Wd in plane tiles of 32 columns in
// core-matrix order (ldw a multiple of 32).
__global__ void k_wdigits(const double* Wn, int nbo, int64_t nprime, int64_t ldw, unsigned short* Wd, int* gcol) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ldw; c += (int64_t)gridDim.x * blockDim.x) {
        double mx = 0.0;
        for (int a = 0; a < nbo; ++a)
            if (c < nprime) mx = fmax(mx, fabs(Wn[(int64_t)a * nprime + c]));
        const int g = exp_of(mx);
        gcol[c] = g;
        for (int a0 = 0; a0 < kOB; a0 += 8) {   // 16-byte chunks, as in k_vdigits
            uint32_t pk[kDig][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int a = a0 + j;
                const double w = (c < nprime && a < nbo) ? Wn[(int64_t)a * nprime + c] : 0.0;
                int d[kDig];
                digits_f64(w, g, d);
#pragma unroll
                for (int p = 0; p < kDig; ++p) {
                    const uint32_t h = bf16_of_int(d[p]);
                    if (j & 1) pk[p][j >> 1] |= h << 16;
                    else pk[p][j >> 1] = h;
                }
            }
#pragma unroll
            for (int p = 0; p < kDig; ++p)
                reinterpret_cast<uint4*>(Wd)[wd_chunk(p, c, a0 >> 3)] =
                    make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
        }
    }
}

// ------------------------------------------------------------------ merging the two panels' T

// Partial Gram block G12(a, b) = V1(:, a)^T V2(:, b) over one row chunk per CTA (rows from
// J0 + 32: V1 is zero-free below its diagonal there, V2 is masked). part[g][a + 32 b].
__global__ void __launch_bounds__(256) k_gram12(const double* A, int64_t lda, int64_t s, int64_t J0, int nb2,
                                                int64_t chunk, double* part) {
    __shared__ double V1s[64][kPanel + 1];
    __shared__ double V2s[64][kPanel + 1];
    const int tid = threadIdx.x, a = tid & 31, bq = tid >> 5;   // outputs (a, 4 bq .. 4 bq + 3)
    const int64_t rb = J0 + kPanel + (int64_t)blockIdx.x * chunk;
    const int64_t re = rb + chunk < s ? rb + chunk : s;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t t0 = rb; t0 < re; t0 += 64) {
        for (int i = tid; i < 64 * kPanel; i += 256) {
            const int rr = i % 64, cc = i / 64;
            const int64_t r = t0 + rr;
            const bool in = r < re;
            V1s[rr][cc] = in ? A[r + (J0 + cc) * lda] : 0.0;
            V2s[rr][cc] = (in && cc < nb2) ? vmask(A, lda, r, J0 + kPanel, cc) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 64; ++rr) {
            const double v1 = V1s[rr][a];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fma(v1, V2s[rr][4 * bq + i], acc[i]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) part[(int64_t)blockIdx.x * kPanel * kPanel + a + (4 * bq + i) * kPanel] = acc[i];
}

// part[0][e] = sum over the nparts partials of entry e (a warp per entry, fixed order).
__global__ void __launch_bounds__(256) k_gsum(double* part, int nparts) {
    const int lane = threadIdx.x & 31;
    const int e = (blockIdx.x * 256 + threadIdx.x) >> 5;
    if (e >= kPanel * kPanel) return;
    double t = 0.0;
    for (int k = lane; k < nparts; k += 32) t += part[(int64_t)k * kPanel * kPanel + e];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) part[e] = t;
}

// Tb (kOB x kOB, column-major) = [[T1, -T1 G12 T2], [0, T2]] with G12 the sum of the partials
// (fixed order); T1, T2 are the panels' 32 x 32 T, nb2 the second panel's width.
__global__ void __launch_bounds__(256) k_tmerge(const double* T1, const double* T2, const double* part, int nparts,
                                                int nb2, double* Tb) {
    __shared__ double G[kPanel * kPanel], X[kPanel * kPanel], t1[kPanel * kPanel], t2[kPanel * kPanel];
    const int tid = threadIdx.x;
    for (int i = tid; i < kPanel * kPanel; i += 256) {
        double t = 0.0;
        for (int k = 0; k < nparts; ++k) t += part[(int64_t)k * kPanel * kPanel + i];
        G[i] = t;
        t1[i] = T1[i];
        t2[i] = T2[i];
    }
    __syncthreads();
    for (int i = tid; i < kPanel * kPanel; i += 256) {   // X = G12 T2
        const int a = i % kPanel, b = i / kPanel;
        double t = 0.0;
        for (int k = 0; k < nb2; ++k) t += G[a + k * kPanel] * t2[k + b * kPanel];
        X[i] = t;
    }
    __syncthreads();
    for (int i = tid; i < kOB * kOB; i += 256) {
        const int a = i % kOB, b = i / kOB;
        double v = 0.0;
        if (a < kPanel && b < kPanel) {
            v = t1[a + b * kPanel];
        } else if (a >= kPanel && b >= kPanel) {
            v = t2[(a - kPanel) + (b - kPanel) * kPanel];
        } else if (a < kPanel && b >= kPanel) {   // -(T1 X)(a, b - 32)
            double t = 0.0;
            for (int k = 0; k < kPanel; ++k) t += t1[a + k * kPanel] * X[k + (b - kPanel) * kPanel];
            v = -t;
        }
        Tb[i] = v;
    }
}

// Tb = T1 zero-padded to kOB x kOB (outer block with one panel).
__global__ void k_tpad(const double* T1, double* Tb) {
    for (int i = threadIdx.x; i < kOB * kOB; i += blockDim.x) {
        const int a = i % kOB, b = i / kOB;
        Tb[i] = (a < kPanel && b < kPanel) ? T1[a + b * kPanel] : 0.0;
    }
}

// ------------------------------------------------------------------ W = V^T C  (split over row chunks)

constexpr int kVtcCols = 32;
constexpr int kVtcPad = 8;                     // bf16 elements of padding per k-row
constexpr int kVtcLdk = kVtcStep + kVtcPad;    // 40

struct VtcSmem {
    unsigned short As[2][kDig][kOB][kVtcLdk];     // V^T digits, two pipeline stages: [p][a][k]
    long long Craw[2][kVtcCols][kVtcStep];        // raw fixed-point C rows, two stages: [c][k]
    unsigned short Bs[kDig][kVtcCols][kVtcLdk];   // C digits of the current step: [q][c][k]
};

// Wp[chunk](a, c) for c in the column tile: sum over the chunk's rows of V(r, a) C(r, c).
// Tile: all kOB rows of W x 32 columns, so each C digit feeds 64 outputs. Two-stage cp.async
// pipeline: the V^T digits and raw C rows of step k + 1 are in flight while step k is cut
// into digits and multiplied.
__global__ void __launch_bounds__(kEmuThreads, 2)
k_emu_vtc(const long long* Cfix, int64_t lda, int64_t s, int64_t n, int64_t J0, int nbo, int64_t kc,
          const unsigned short* VTd, int64_t ldv, const int* ecol, const int* E, double* Wp, int64_t nprime) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VtcSmem& sm = *reinterpret_cast<VtcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int64_t jc = J0 + nbo;
    const int64_t c0 = (int64_t)blockIdx.x * kVtcCols;
    const int64_t L = s - J0;
    const int64_t lb = (int64_t)blockIdx.y * kc;               // local row range [lb, le)
    const int64_t le = lb + kc < L ? lb + kc : L;
    const int mi = warp & 3, nt = warp >> 2;                   // warp: a in mi*16.., cols nt*16..
    // Per output, the level sums are packed into two int64 fixed-point words:
    // hi = sum_{l<3} T_l 2^(8 (2 - l)), lo = sum_{l>=3} T_l 2^(8 (5 - l)); per K-step each T_l < 2^22,
    // so both stay below 2^50 over 1600 steps.
    long long hi[2][4], lo[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 4; ++h) { hi[j][h] = 0; lo[j][h] = 0; }

    auto issue = [&](int stage, int64_t k0) {
        // V^T digits: per (p, a) 32 contiguous bf16 = 4 chunks of 16 B
        for (int idx = tid; idx < kDig * kOB * 4; idx += kEmuThreads) {
            const int ch = idx & 3, a = (idx >> 2) % kOB, p = (idx >> 2) / kOB;
            const int64_t lr = k0 + ch * 8;
            const bool ok = lr < ldv;
            const unsigned short* src = VTd + ((int64_t)p * kOB + a) * ldv + (ok ? lr : 0);
            cp_async16(&sm.As[stage][p][a][ch * 8], src, ok ? 16 : 0);
        }
        // raw C: per column 32 rows = 16 chunks of two int64
        for (int idx = tid; idx < kVtcCols * (kVtcStep / 2); idx += kEmuThreads) {
            const int ch = idx % (kVtcStep / 2), c = idx / (kVtcStep / 2);
            const int64_t lr = k0 + 2 * ch, gc = jc + c0 + c;
            const int rows = (gc < n) ? (int)(le - lr < 0 ? 0 : (le - lr > 2 ? 2 : le - lr)) : 0;
            const long long* src = Cfix + (rows > 0 ? (J0 + lr) + gc * lda : 0);
            cp_async16(&sm.Craw[stage][c][2 * ch], src, rows * 8);
        }
        cp_async_commit();
    };

    int stage = 0;
    issue(0, lb);
    for (int64_t k0 = lb; k0 < le; k0 += kVtcStep) {
        if (k0 + kVtcStep < le) issue(stage ^ 1, k0 + kVtcStep);
        else cp_async_commit();                                // keep the group count uniform
        cp_async_wait<1>();
        __syncthreads();
        // cut this step's C entries into digits: a warp takes the 32 rows of one column at a time, so
        // its int64 reads from shared memory are consecutive words (no bank conflicts)
#pragma unroll
        for (int e = 0; e < (kVtcCols * kVtcStep) / kEmuThreads; ++e) {
            const int idx = e * kEmuThreads + tid;
            const int c = idx / kVtcStep, k = idx % kVtcStep;
            int d[kDig];
            digits_fix(sm.Craw[stage][c][k], d);
#pragma unroll
            for (int q = 0; q < kDig; ++q) sm.Bs[q][c][k] = bf16_of_int(d[q]);
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l <= kLev; ++l) {
            float acc[2][4] = {{kMagic, kMagic, kMagic, kMagic}, {kMagic, kMagic, kMagic, kMagic}};
#pragma unroll
            for (int p = 0; p <= l; ++p) {
                const int q = l - p;
#pragma unroll
                for (int ks = 0; ks < kVtcStep; ks += 16) {
                    uint32_t af[4], bq[4];
                    ldsm_x4(af, &sm.As[stage][p][mi * 16 + (lane & 15)][ks + (lane >> 4) * 8]);
                    ldsm_x4(bq, &sm.Bs[q][nt * 16 + (lane & 7) + ((lane >> 4) & 1) * 8][ks + ((lane >> 3) & 1) * 8]);
                    const uint32_t b0[2] = {bq[0], bq[1]}, b1[2] = {bq[2], bq[3]};
                    hmma(acc[0], af, b0);
                    hmma(acc[1], af, b1);
                }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const long long v = (long long)magic_to_int(acc[j][h]);
                    if (l < 3) hi[j][h] += v << (8 * (2 - l));
                    else lo[j][h] += v << (8 * (5 - l));
                }
        }
        __syncthreads();
        stage ^= 1;
    }
    cp_async_wait<0>();
    // W(a, c) = 2^(e_a + E_c - 14) sum_l 2^(-8 l) T_l   (C entries carry scale 2^(E_c - 47))
    double* out = Wp + (int64_t)blockIdx.y * kOB * nprime;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int a = mi * 16 + g + (h >> 1) * 8;
            const int64_t col = c0 + nt * 16 + j * 8 + 2 * t + (h & 1);
            if (col < nprime && a < nbo) {
                const int sc = ecol[a] + E[jc + col] - 14;
                const double v = ldexp((double)hi[j][h], -16) + ldexp((double)lo[j][h], -40);
                out[(int64_t)a * nprime + col] = ldexp(v, sc);
            }
        }
}

// ------------------------------------------------------------------ C += V Wn  (exact integer update, tcgen05)

// One CTA per SM owns a 128-row tile of C and walks `cpt` consecutive 32-column tiles. Roles:
//   warp 0 (one thread)  copies: the V digit planes of the row tile once (one bulk copy), then
//                        per column tile its Wn digit planes (one bulk copy) and its 128 x 32 C
//                        block (one 2D tensor copy; rows past s and columns past n read as zero)
//                        into one of two stages, on separate barriers so the MMAs never wait
//                        for C;
//   warp 1 (one thread)  tcgen05.mma: per level l the products of digit pairs p + q = l
//                        accumulate in their own FP32 TMEM block (exact: every level sum is an
//                        integer below 6 x 64 x 2^14 < 2^23); two accumulator sets of 6 x 32
//                        columns, so the MMAs of tile i + 1 run while tile i is written back;
//   warps 2..9           epilogue: TMEM -> registers, levels combined in int64, scaled onto the
//                        column's fixed-point grid and added to the staged C entry; one thread
//                        per row and 16 columns, so each column store of a warp is 256
//                        contiguous bytes.
// Every wait is bounded (spin polls and 2 s of wall time); a role that gives up sets the CTA's
// abort flag and the error word, and the CTA still waits for its copies and MMAs in flight and
// frees its tensor memory before it returns.
constexpr int kTcLevels = kLev + 1;
constexpr int kTcPlaneA = kTcM * kOB * 2;        // bytes of one V digit plane tile (16 KB)
constexpr int kTcPlaneB = kTcN * kOB * 2;        // bytes of one Wn digit plane tile (4 KB)
constexpr int kTcBufCols = kTcLevels * kTcN;     // TMEM columns of one accumulator set (192)
constexpr int kTcTmemCols = 512;
constexpr int kTcEpiWarps = 8;
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr unsigned long long kTcWaitNs = 2000000000ULL;
constexpr long long kTeardownSpin = 1LL << 62;   // teardown waits: bounded by kTcWaitNs alone

struct TcUpdSmem {
    unsigned char A[kDig][kTcPlaneA];
    unsigned char B[2][kDig][kTcPlaneB];
    long long C[2][kTcN][kTcM];
    uint64_t full_a, full_b[2], full_c[2], done[2], freed[2], drain;
    uint32_t tmem;
    int abort;
};

// 2D tiled tensor copy global -> shared (box of the tensor map at coordinates x, y)
__device__ __forceinline__ void tensor_g2s_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc::smem_addr(bar))
        : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_emu_update_tc(const __grid_constant__ CUtensorMap cmap, long long* Cfix, int64_t lda, int64_t s, int64_t J0, int nbo,
                const unsigned short* Vd, const int* frow, const unsigned short* Wd, const int* gcol, const int* E,
                int64_t nprime, int cpt, long long spin, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcUpdSmem& sm = *reinterpret_cast<TcUpdSmem*>(tc_smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t L = s - J0, jc = J0 + nbo;
    const int64_t rt = blockIdx.y, rb = rt * kTcM;
    const int64_t nct = (nprime + kTcN - 1) / kTcN;
    const int64_t ct0 = (int64_t)blockIdx.x * cpt;
    const int ntile = (int)(nct - ct0 < cpt ? nct - ct0 : cpt);
    volatile int* abort = &sm.abort;
    // tensor copies write shared memory at 128-byte boundaries: the staging area must start on one
    if ((tc::smem_addr(tc_smem_raw) & 127) != 0) {
        if (threadIdx.x == 0) set_error(err, CSLS_ERR_ARG);
        return;
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&sm.full_a, 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&sm.full_b[b], 1);
            tc::mbar_init(&sm.full_c[b], 1);
            tc::mbar_init(&sm.done[b], 1);
            tc::mbar_init(&sm.freed[b], 32 * kTcEpiWarps);
        }
        tc::mbar_init(&sm.drain, 1);
        sm.abort = 0;
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(&sm.tmem, kTcTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;

    if (warp == 0) {
        if (lane == 0) {
            int armed0 = 0, armed1 = 0;   // uses of each stage whose copies were issued
            tc::mbar_arrive_expect_tx(&sm.full_a, kDig * kTcPlaneA);
            tc::bulk_g2s(sm.A[0], reinterpret_cast<const unsigned char*>(Vd) + rt * (kDig * kTcPlaneA),
                         kDig * kTcPlaneA, &sm.full_a);
            for (int i = 0; i < ntile; ++i) {
                const int b = i & 1, u = i >> 1;
                if (u > 0 && !tc::mbar_wait(&sm.freed[b], (u - 1) & 1, spin, kTcWaitNs, abort)) {
                    *abort = 1;
                    set_error(err, CSLS_ERR_TIMEOUT);
                    break;
                }
                const int64_t ct = ct0 + i;
                tc::mbar_arrive_expect_tx(&sm.full_b[b], kDig * kTcPlaneB);
                tc::bulk_g2s(sm.B[b][0], reinterpret_cast<const unsigned char*>(Wd) + ct * (kDig * kTcPlaneB),
                             kDig * kTcPlaneB, &sm.full_b[b]);
                tc::mbar_arrive_expect_tx(&sm.full_c[b], kTcN * kTcM * 8);
                tensor_g2s_2d(sm.C[b][0], &cmap, (int)(J0 + rb), (int)(jc + ct * kTcN), &sm.full_c[b]);
                if (b) armed1 = u + 1;
                else armed0 = u + 1;
            }
            // copies in flight land before the CTA can leave. Issued copies always complete, so
            // these waits are bounded by wall time only (not by the caller's spin count, which
            // may be tiny): a CTA never exits with a copy still writing its shared memory.
            tc::mbar_wait(&sm.full_a, 0, kTeardownSpin, kTcWaitNs, nullptr);
            if (armed0) {
                tc::mbar_wait(&sm.full_b[0], (armed0 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
                tc::mbar_wait(&sm.full_c[0], (armed0 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
            }
            if (armed1) {
                tc::mbar_wait(&sm.full_b[1], (armed1 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
                tc::mbar_wait(&sm.full_c[1], (armed1 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            bool issued = false;
            if (tc::mbar_wait(&sm.full_a, 0, spin, kTcWaitNs, abort)) {
                const uint32_t idesc = tc::idesc_bf16_f32(kTcM, kTcN);
                const uint64_t adesc = tc::smem_desc(tc::smem_addr(sm.A[0]), kTcM * 16, 128);
                for (int i = 0; i < ntile; ++i) {
                    const int b = i & 1, u = i >> 1;
                    // the accumulator set of this stage was drained by the epilogue of tile i - 2
                    if ((u > 0 && !tc::mbar_wait(&sm.freed[b], (u - 1) & 1, spin, kTcWaitNs, abort)) ||
                        !tc::mbar_wait(&sm.full_b[b], u & 1, spin, kTcWaitNs, abort)) {
                        *abort = 1;
                        set_error(err, CSLS_ERR_TIMEOUT);
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t bdesc = tc::smem_desc(tc::smem_addr(sm.B[b][0]), kTcN * 16, 128);
                    const uint32_t d0 = tmem + (uint32_t)(b * kTcBufCols);
                    // 84 MMAs, fully unrolled: each descriptor is the stage's base plus a constant
                    // (the start address sits in the low bits, in 16-byte units); a K step of 16 is
                    // two core-matrix columns
#pragma unroll
                    for (int l = 0; l <= kLev; ++l)
#pragma unroll
                        for (int p = 0; p <= l; ++p)
#pragma unroll
                            for (int k = 0; k < kOB / 16; ++k)
                                tc::mma_bf16(d0 + l * kTcN,
                                             adesc + (uint64_t)((p * kTcPlaneA + k * 2 * (kTcM * 16)) >> 4),
                                             bdesc + (uint64_t)(((l - p) * kTcPlaneB + k * 2 * (kTcN * 16)) >> 4),
                                             idesc, (p | k) != 0);
                    tc::mma_commit(&sm.done[b]);
                    issued = true;
                }
            } else {
                *abort = 1;
                set_error(err, CSLS_ERR_TIMEOUT);
            }
            if (issued) {   // every MMA has completed before the tensor memory is freed (wall-time bound only)
                tc::mma_commit(&sm.drain);
                tc::mbar_wait(&sm.drain, 0, kTeardownSpin, kTcWaitNs, nullptr);
            }
        }
        __syncwarp();
    } else {
        const int quarter = warp & 3;              // a warp reads TMEM lanes 32 (warp % 4) .. + 31
        const int half = (warp - 2) >> 2;          // columns 16 half .. + 15 of each tile
        const int r = quarter * 32 + lane;
        const int64_t lr = rb + r;
        const bool rok = lr < L;
        const int fr = rok ? frow[lr] : 0;
        for (int i = 0; i < ntile; ++i) {
            const int b = i & 1, u = i >> 1;
            bool ok = tc::mbar_wait(&sm.done[b], u & 1, spin, kTcWaitNs, abort) &&
                      tc::mbar_wait(&sm.full_c[b], u & 1, spin, kTcWaitNs, abort);
            ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld is warp-wide
            if (!ok) {
                *abort = 1;
                set_error(err, CSLS_ERR_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTcBufCols + half * 16);
            uint32_t v[kTcLevels][16];
#pragma unroll
            for (int l = 0; l < kTcLevels; ++l) tc::tmem_ld16(ta + l * kTcN, v[l]);
            tc::tmem_ld_wait();
            tc::fence_before_sync();
            const int64_t cbase = (ct0 + i) * kTcN + half * 16;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int64_t col = cbase + j;
                if (rok && col < nprime) {
                    long long acc = 0;
#pragma unroll
                    for (int l = 0; l < kTcLevels; ++l)
                        acc = acc * 256 + (long long)__float2int_rn(__uint_as_float(v[l][j]));
                    // Cfix += acc * 2^(f_r + g_c - 14 - 8 kLev + 62 - E_c), rounded to the fixed-point grid
                    const int sh = fr + gcol[col] - 14 - 8 * kLev + kFixBits - E[jc + col];
                    long long dlt;
                    if (acc == 0) dlt = 0;
                    else if (sh >= 0) dlt = sh < 63 ? acc << sh : 0;
                    else dlt = -sh < 63 ? (acc + (1LL << (-sh - 1))) >> (-sh) : 0;
                    Cfix[(J0 + lr) + (jc + col) * lda] = sm.C[b][half * 16 + j][r] + dlt;
                }
            }
            tc::mbar_arrive(&sm.freed[b]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTcTmemCols);
    }
}

// Tensor map of the int64 trailing matrix for the update's C tiles: rows (contiguous, s of
// them) x columns (n, stride lda), 128 x 32 boxes, zero fill outside.
static int make_c_map(CUtensorMap* map, void* A, int64_t lda, int64_t s, int64_t n) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return CSLS_ERR_CUDA;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)s, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)lda * 8};
    const cuuint32_t box[2] = {(cuuint32_t)kTcM, (cuuint32_t)kTcN};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, A, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return CSLS_ERR_CUDA;
    return CSLS_OK;
}

// Column tiles per CTA: the split of each row tile's columns that minimises the waves of
// one-CTA-per-SM launches times the tiles a CTA walks (plus ~2 tiles for its V planes and the
// pipeline fill).
static int tc_update_cpt(int64_t nrt, int64_t nct, int sms) {
    int best = (int)nct;
    double best_cost = 1e300;
    for (int64_t c = 1; c <= nct; ++c) {
        const int64_t ncs = (nct + c - 1) / c;
        const double cost = (double)((nrt * ncs + sms - 1) / sms) * (double)(c + 2);
        if (cost < best_cost) {
            best_cost = cost;
            best = (int)c;
        }
    }
    return best;
}

// ------------------------------------------------------------------ scratch and driver

struct EmuScratch {
    int* E;                       // n column exponents
    unsigned long long* colmax;   // kOB
    int* ecol;                    // kOB
    int* frow;                    // s
    int* gcol;                    // n
    unsigned short* Vd;           // kDig * s * kOB (s rounded up to 128)
    unsigned short* VTd;          // kDig * kOB * s
    unsigned short* Wd;           // kDig * n * kOB (n rounded up to 32)
    double* Wp;                   // split-K partials of W (kOB x n per chunk)
    int64_t wp_elems;
    double* Wn;                   // kOB x n
    double* T1;                   // first panel's T (32 x 32)
    double* Tb;                   // outer block's T (kOB x kOB)
    double* gpart;                // Gram partials of the two panels
    int64_t gparts;
};

static int64_t emu_wp_elems(int64_t n) {
    const int64_t a = (int64_t)kOB * (n + kVtcCols);
    const int64_t b = (int64_t)kOB * kVtcCols * (8LL * device_sm_count() + 8);
    return a > b ? a : b;
}

static EmuScratch emu_carve(Carve& c, int64_t s, int64_t n) {
    const int64_t ldv = round_up(s, kTcM), ldw = round_up(n, kTcN);
    EmuScratch e;
    e.E = c.take<int>((size_t)n);
    e.colmax = c.take<unsigned long long>(kOB);
    e.ecol = c.take<int>(kOB);
    e.frow = c.take<int>((size_t)ldv);
    e.gcol = c.take<int>((size_t)ldw);
    e.Vd = c.take<unsigned short>((size_t)(kDig * ldv * kOB));
    e.VTd = c.take<unsigned short>((size_t)(kDig * ldv * kOB));
    e.Wd = c.take<unsigned short>((size_t)(kDig * ldw * kOB));
    e.wp_elems = emu_wp_elems(n);
    e.Wp = c.take<double>((size_t)e.wp_elems);
    e.Wn = c.take<double>((size_t)(kOB * (n + kOB)));
    e.T1 = c.take<double>(kPanel * kPanel);
    e.Tb = c.take<double>(kOB * kOB);
    e.gparts = 2LL * device_sm_count();
    e.gpart = c.take<double>((size_t)(e.gparts * kPanel * kPanel));
    return e;
}

size_t qr_emu_scratch_bytes(int64_t s, int64_t n) {
    Carve c{nullptr, 0, 0, true};
    emu_carve(c, s, n);
    return c.off;
}

int qr_panel_launch_f64(double* A, int64_t lda, int64_t s, int64_t j0, int nbw, const QrScratch& q, int* err,
                        long long spin, cudaStream_t st);

int qr_factor_f64_emu(double* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, void* emu_work,
                      size_t emu_bytes, int* err, long long spin, cudaStream_t st, int64_t* launches) {
    if (s < n || n <= 0) return CSLS_ERR_ARG;
    if (emu_bytes < qr_emu_scratch_bytes(s, n)) return CSLS_ERR_WORKSPACE;
    Carve c{(char*)emu_work, 0, emu_bytes, false};
    EmuScratch e = emu_carve(c, s, n);
    // the update's tensor copies read C from 16-byte boundaries
    if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (lda & 1) != 0) return CSLS_ERR_ARG;
    CUtensorMap cmap;
    CSLS_TRY(make_c_map(&cmap, A, lda, s, n));
    CSLS_TRY(raise_smem_limit((const void*)k_emu_vtc, (int)sizeof(VtcSmem)));
    CSLS_TRY(raise_smem_limit((const void*)k_emu_update_tc, (int)sizeof(TcUpdSmem)));
    CSLS_TRY(raise_smem_limit((const void*)k_wreduce_ob, (int)kWrSmem));
    const int sms = device_sm_count();
    CSLS_CUDA(cudaMemsetAsync(q.bar, 0, sizeof(GridBarrier), st));
    k_col_exponent<<<(unsigned)std::min<int64_t>(n, 65535), 256, 0, st>>>(A, lda, s, n, e.E);
    CSLS_CUDA(cudaGetLastError());
    dim3 fg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(s, 1024), 64)), (unsigned)std::min<int64_t>(n, 65535));
    k_to_fixed<<<fg, 256, 0, st>>>(A, lda, s, n, e.E);
    CSLS_CUDA(cudaGetLastError());
    int64_t nl = 2;
    for (int64_t J0 = 0; J0 < n; J0 += kOB) {
        const int nbo = (int)(n - J0 < kOB ? n - J0 : kOB);
        const int nb1 = nbo < kPanel ? nbo : kPanel;
        const int nb2 = nbo - nb1;
        const int64_t L = s - J0;
        // the outer block's columns return to binary64 (rows below and above the diagonal block)
        dim3 pg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 256), 256)), (unsigned)nbo);
        k_panel_to_f64<<<pg, 256, 0, st>>>(A, lda, s, J0, nbo, e.E);
        CSLS_CUDA(cudaGetLastError());
        if (J0 > 0) {
            dim3 tg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(J0, 256), 64)), (unsigned)nbo);
            k_panel_top_to_f64<<<tg, 256, 0, st>>>(A, lda, J0, nbo, e.E);
            CSLS_CUDA(cudaGetLastError());
        }
        // first panel, its update of the second one (FP64 MMA), second panel
        int tk = kt_begin(kFamPanel, st);
        CSLS_TRY(qr_panel_launch_f64(A, lda, s, J0, nb1, q, err, spin, st));
        kt_end(tk, 0.0, st);
        nl += 3;
        if (nb2 > 0) {
            CSLS_CUDA(cudaMemcpyAsync(e.T1, q.T, sizeof(double) * kPanel * kPanel, cudaMemcpyDeviceToDevice, st));
            CSLS_TRY(qr_trailing_update_f64(A, lda, s, J0 + nbo, J0, nb1, q, st));
            tk = kt_begin(kFamPanel, st);
            CSLS_TRY(qr_panel_launch_f64(A, lda, s, J0 + kPanel, nb2, q, err, spin, st));
            kt_end(tk, 0.0, st);
            // merged T of the outer block
            const int64_t L2 = s - J0 - kPanel;
            int gp = (int)std::min<int64_t>(e.gparts, std::max<int64_t>(1, ceil_div(L2, 128)));
            const int64_t chunk = round_up(ceil_div(L2, gp), 64);
            gp = (int)ceil_div(L2, chunk);
            k_gram12<<<gp, 256, 0, st>>>(A, lda, s, J0, nb2, chunk, e.gpart);
            CSLS_CUDA(cudaGetLastError());
            // the partials of each Gram entry summed by a warp (in place into partial 0), so the
            // single-CTA merge reads one value per entry
            k_gsum<<<kPanel * kPanel / 8, 256, 0, st>>>(e.gpart, gp);
            CSLS_CUDA(cudaGetLastError());
            k_tmerge<<<1, 256, 0, st>>>(e.T1, q.T, e.gpart, 1, nb2, e.Tb);
            CSLS_CUDA(cudaGetLastError());
            nl += 6;
        } else {
            k_tpad<<<1, 256, 0, st>>>(q.T, e.Tb);
            CSLS_CUDA(cudaGetLastError());
            nl += 1;
        }
        const int64_t nprime = n - J0 - nbo;
        if (nprime <= 0) continue;
        // digits of V
        CSLS_CUDA(cudaMemsetAsync(e.colmax, 0, sizeof(unsigned long long) * kOB, st));
        k_vcolmax<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 4), (int64_t)sms * 4)), 256, 0, st>>>(
            A, lda, s, J0, nbo, e.colmax);
        CSLS_CUDA(cudaGetLastError());
        const int64_t ldvp = round_up(L, kTcM);   // digit planes use the current block height
        k_vdigits<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ldvp, 256), (int64_t)sms * 8)), 256, 0, st>>>(
            A, lda, s, J0, nbo, e.colmax, ldvp, e.Vd, e.VTd, e.frow, e.ecol);
        CSLS_CUDA(cudaGetLastError());
        // W = V^T C over row chunks
        const int64_t ntn = ceil_div(nprime, kVtcCols);
        int64_t ks = ceil_div(8LL * sms, ntn);
        const int64_t maxks = ceil_div(L, kVtcStep);
        if (ks > maxks) ks = maxks;
        if (ks > 64) ks = 64;   // narrow trailing blocks: a few long row chunks keep the partial sums short
        if (ks < 1) ks = 1;
        while (ks > 1 && ks * kOB * ntn * kVtcCols > e.wp_elems) --ks;
        const int64_t kc = round_up(ceil_div(L, ks), kVtcStep);
        ks = ceil_div(L, kc);
        const double prod_flop = 2.0 * (double)L * (double)nprime * (double)nbo;
        tk = kt_begin(kFamVtc, st);
        k_emu_vtc<<<dim3((unsigned)ntn, (unsigned)ks), kEmuThreads, sizeof(VtcSmem), st>>>(
            reinterpret_cast<const long long*>(A), lda, s, n, J0, nbo, kc, e.VTd, ldvp, e.ecol, e.E, e.Wp, nprime);
        CSLS_CUDA(cudaGetLastError());
        kt_end(tk, prod_flop, st);
        k_wreduce_ob<<<(unsigned)ceil_div(nprime, kWrCols), 256, kWrSmem, st>>>(e.Wp, (int)ks, e.Tb, nbo, e.Wn, nprime);
        CSLS_CUDA(cudaGetLastError());
        // digits of Wn, then the exact update
        const int64_t ldwp = round_up(nprime, kTcN);
        k_wdigits<<<(unsigned)std::max<int64_t>(1, ceil_div(ldwp, 256)), 256, 0, st>>>(e.Wn, nbo, nprime, ldwp, e.Wd,
                                                                                        e.gcol);
        CSLS_CUDA(cudaGetLastError());
        // a trailing block exists only right of a full 64-column outer block: the update's
        // products always run over K = 64
        if (nbo != kOB) return CSLS_ERR_ARG;
        tk = kt_begin(kFamUpdate, st);
        const int64_t nrt = ceil_div(L, kTcM), nct = ceil_div(nprime, kTcN);
        const int cpt = tc_update_cpt(nrt, nct, sms);
        k_emu_update_tc<<<dim3((unsigned)ceil_div(nct, cpt), (unsigned)nrt), kTcThreads, sizeof(TcUpdSmem), st>>>(
            cmap, reinterpret_cast<long long*>(A), lda, s, J0, nbo, e.Vd, e.frow, e.Wd, e.gcol, e.E, nprime, cpt, spin,
            err);
        CSLS_CUDA(cudaGetLastError());
        kt_end(tk, prod_flop, st);
        nl += 7;
    }
    if (launches) *launches += nl;
    return CSLS_OK;
}

}  // namespace csls

// Blocked Householder QR of the sketch with the trailing-matrix products done on
// the bf16 tensor cores at FP64-level accuracy (Algorithm 1 step 3).
//
// GB300 runs FP64 arithmetic at ~1.1 TFLOP/s but bf16 tcgen05 MMA at ~1.7 PFLOP/s, so the two
// products of every trailing update (W = V^T C and C += V Wn) are computed from
// exact integer pieces, in the spirit of Ozaki, Ogita, Oishi and Rump's
// error-free splitting of matrix products:
//   * every operand entry is written as a signed integer of 47 bits relative to a
//     power-of-two scale shared along the contraction (per row of the left
//     operand, per column of the right one) and cut into 6 balanced base-256
//     digits in [-128, 128], each exact in bf16;
//   * digit-plane products are exact integers of at most 2^14; digit pairs of the
//     same weight (level l = p + q) share one FP32 accumulator in tensor memory, and
//     every level sum is kept below 2^24 so the FP32 accumulation is exact; levels
//     0..5 are kept (21 of 36 pairs), the dropped ones weigh 2^-48 of the leading term;
//   * levels are combined in int64.
// The trailing matrix is held in int64 fixed point per column: value =
// Cfix * 2^(E_c - 62) with 2^E_c above the column's 2-norm. Orthogonal updates
// never increase the norm of a trailing column, so the scale is fixed for the
// whole factorisation and C += V Wn is an exact integer addition -- the update
// never touches the FP64 pipe. A column switches to FP64 (in place, same bytes)
// when it becomes part of a panel; the panel is factored in FP64 by k_obpanel.
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
// FP32 accumulators start at 1.5 * 2^23: while |sum| < 2^22 the integer sum sits exactly in the
// low mantissa bits, so it is read back with one integer subtraction (no conversion instruction).
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

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

// N = x 2^(BITS - e) rounded to the nearest integer (ties to even), for |x| < 2^e, from the bit
// pattern of x alone (integer instructions; FP64 ones are scarce on this part): x = m 2^e2 with the
// 53-bit significand m, so N = m 2^-sh with sh = e - BITS - e2, and a shift with round-to-nearest-even
// gives it exactly (the same integer as rounding the exact product; |N| < 2^BITS).
template <int BITS>
__device__ __forceinline__ long long fix_bits(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ev = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (ev != 0) m |= 1ull << 52;
    const int sh = e - BITS - ((ev != 0 ? ev : 1) - 1075);
    unsigned long long q;
    if (sh <= 0) {
        q = sh > -64 ? m << (-sh) : 0ull;
    } else if (sh >= 64) {
        q = 0ull;
    } else {
        q = m >> sh;
        const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

// digits of x relative to scale 2^e (|x| < 2^e)
__device__ __forceinline__ void digits_f64(double x, int e, int (&d)[kDig]) {
    cut_digits(fix_bits<kNumBits>(x, e), d);
}

// digits of a fixed-point entry (|Cfix| < 2^62): N = round(Cfix / 2^(62 - 47))
__device__ __forceinline__ void digits_fix(long long c, int (&d)[kDig]) {
    const long long N = (c + (1LL << (kFixBits - kNumBits - 1))) >> (kFixBits - kNumBits);
    cut_digits(N, d);
}

// The six digits of a fixed-point entry (|Cfix| < 2^62) as floats, the same digits as digits_fix:
// after adding 128 to each of the five low bytes of N, byte b of the sum is digit + 128, and one
// byte permute places it under the exponent of 2^23 (the float 2^23 + byte), so one FP32 subtract
// gives the digit exactly; the top digit is the sum shifted right by 40.
__device__ __forceinline__ void digit_floats_fix(long long c, float (&f)[kDig]) {
    const long long M = ((c + (1LL << (kFixBits - kNumBits - 1))) >> (kFixBits - kNumBits)) + 0x8080808080LL;
    const uint32_t lo = (uint32_t)M, hi = (uint32_t)(M >> 32);
    const float base = 8388736.0f;   // 2^23 + 128
    f[5] = __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7540)) - base;
    f[4] = __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7541)) - base;
    f[3] = __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7542)) - base;
    f[2] = __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7543)) - base;
    f[1] = __uint_as_float(__byte_perm(hi, 0x4B000000u, 0x7540)) - base;
    f[0] = __int_as_float(kMagicBits + ((int)hi >> 8)) - kMagic;
}

// two floats holding small integers (exact in bf16) as one bf16x2 word: lo in bits 0..15
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ unsigned short bf16_of_int(int v) {
    // |v| <= 128: exactly representable. int -> float by the same magic-number trick
    // (one integer add, one float subtract), then the top 16 bits are the bf16 pattern.
    const float f = __int_as_float(kMagicBits + v) - kMagic;
    return (unsigned short)(__float_as_uint(f) >> 16);
}

// |x| as an ordered integer (the bit pattern without its sign); NaN maps to 0, as fmax ignores it
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    return u > 0x7FF0000000000000ull ? 0ull : u;
}

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// a + x 2^32 (two's complement, modulo 2^64): x added to the high word
__device__ __forceinline__ long long add_hi32(long long a, int x) {
    long long r;
    asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tadd.s32 hi, hi, %2;\n\tmov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r) : "l"(a), "r"(x));
    return r;
}
// a x b + c with a 64-bit product and sum
__device__ __forceinline__ long long mad_wide_s32(int a, int b, long long c) {
    long long r;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
    return r;
}

// An integer-valued float f with |f| <= 2^22, as an int: f + 1.5 x 2^23 lies in [2^23, 2^24], where
// the float grid is the integers, so its bit pattern is 0x4B400000 + f exactly.
__device__ __forceinline__ int magic_int(float f) { return __float_as_int(__fadd_rn(f, kMagic)) - kMagicBits; }

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

// In place: SA (double) -> fixed point (int64) per column, N = round(v 2^(62 - E_c)) by integer operations.
__global__ void k_to_fixed(double* A, int64_t lda, int64_t s, int64_t n, const int* E) {
    for (int64_t c = blockIdx.y; c < n; c += gridDim.y) {
        const int ec = E[c];
        long long* colf = reinterpret_cast<long long*>(A + c * lda);
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s; r += (int64_t)gridDim.x * blockDim.x) {
            const double v = A[r + c * lda];
            colf[r] = ec > -1000 ? fix_bits<kFixBits>(v, ec) : 0LL;
        }
    }
}

// ------------------------------------------------------------------ outer-block digit kernels
//
// The emulated products act on outer blocks of kOB = 64 columns: the block is factored in
// binary64 by one cooperative kernel (k_obpanel, which also forms the block's compact-WY T and
// the digit planes of V), and the trailing matrix is updated once per 64 columns. A product with
// K = 64 keeps every level sum below 6 x 64 x 2^14 < 2^24, so it is exact in FP32 and is read
// back with one rounding conversion per level.

constexpr int kOB = 2 * kPanel;   // 64

// Tiles of the tcgen05 update C += V Wn: 128 rows (one TMEM lane each) x 32 columns. Its digit
// planes are stored tile by tile in the canonical K-major core-matrix order, so that one bulk
// copy moves a tile's planes into shared memory ready for the MMA. In a V plane the 16-byte
// chunk holding row r, columns 8 kg .. 8 kg + 7 sits at chunk index kg x 128 + r. The six Wn
// planes of a column tile are stacked along N (row q x 32 + c of a 192-row operand), chunk
// index kg x 192 + q x 32 + c: one MMA with N = 32 (6 - p) then multiplies V plane p by Wn
// planes 0 .. 5 - p at once, writing levels p .. 5, whose TMEM blocks are adjacent.
constexpr int kTcM = 128;
constexpr int kTcN = 32;
constexpr int kTcNStack = kDig * kTcN;   // 192 rows of the stacked Wn operand
__device__ __forceinline__ int64_t vd_chunk(int p, int64_t lr, int kg) {
    return (((lr >> 7) * kDig + p) * 8 + kg) * kTcM + (lr & (kTcM - 1));
}
// Column-scaled V digits for W = V^T C, in the K-major core-matrix order of that product's B operand:
// the six planes stacked along N (row p x 64 + a), 16-byte chunks of 8 consecutive rows, chunk
// index (lr / 8) x 384 + p x 64 + a -- so the digits of any 32 rows starting at a multiple of 32 are
// one contiguous 24 KB block (one bulk copy).
__device__ __forceinline__ int64_t vtd_index(int p, int a, int64_t lr) {
    return (((lr >> 3) * (kDig * kOB) + p * kOB + a) << 3) + (lr & 7);
}
__device__ __forceinline__ int64_t wd_chunk(int q, int64_t c, int kg) {
    return ((c >> 5) * 8 + kg) * kTcNStack + q * kTcN + (c & (kTcN - 1));
}

// Wn = -T^T (sum of the split-K partials of W = V^T C) for the outer block (T: nbo x nbo upper
// triangular, column-major with ld kOB); Wp[k] and Wn are kOB x nprime row-major. A CTA owns 16
// columns (several CTAs share an SM, so their FP64 dot products hide each other's latency): it sums
// their partials (coalesced along the columns) into shared memory, then each thread forms entries of
// -T^T W from the shared copies of T and W.
constexpr int kWrCols = 16;
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
        double t = 0.0, t1 = 0.0;
        int b = 0;
        for (; b + 1 <= a; b += 2) {
            t = fma(Ts[b + a * kOB], Ws[b * kWrCols + cl], t);
            t1 = fma(Ts[b + 1 + a * kOB], Ws[(b + 1) * kWrCols + cl], t1);
        }
        if (b <= a) t = fma(Ts[b + a * kOB], Ws[b * kWrCols + cl], t);
        Wn[(int64_t)a * nprime + c] = -(t + t1);
    }
}

// Digits of Wn (kOB x nprime, row-major): per-column scale 2^g_c; Wd in plane tiles of 32 columns in
// core-matrix order (ldw a multiple of 32). gsh[c] = g_c - E_(jc + c) + 62 - 14 - 8 kLev is the column's
// part of the shift that puts an update product onto the fixed-point grid of trailing column jc + c.
__global__ void k_wdigits(const double* Wn, int nbo, int64_t nprime, int64_t ldw, unsigned short* Wd, const int* E,
                          int64_t jc, int* gsh) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ldw; c += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long mxb = 0ull;
        for (int a = 0; a < nbo; ++a)
            if (c < nprime) {
                const unsigned long long u = abs_bits(Wn[(int64_t)a * nprime + c]);
                mxb = u > mxb ? u : mxb;
            }
        const int g = exp_of(__longlong_as_double((long long)mxb));
        gsh[c] = c < nprime ? g - E[jc + c] + kFixBits - 14 - 8 * kLev : 0;
        for (int a0 = 0; a0 < kOB; a0 += 8) {   // 16-byte chunks of 8 K-consecutive digits
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

// ------------------------------------------------------------------ fused outer-block panel
//
// The Householder factorisation of one outer block (nbo <= 64 columns, rows J0 .. s - 1) as one
// cooperative launch, plus everything the emulated trailing products need from it. A CTA owns a
// contiguous chunk of rows, converts its part of the block from fixed point to binary64 (kept in
// shared memory when it fits) and applies every reflector to it locally. Column c needs one
// grid-wide reduction: for x = A(j:s, j), j = J0 + c, the tail norm sigma = ||x(1:)||^2, the
// diagonal alpha = x(0), and for every later block column k the tail product d_k = x(1:)^T A(j+1:s, k)
// and the entry top_k = A(j, k). With beta = -sign(alpha) sqrt(alpha^2 + sigma), tau = (beta -
// alpha) / beta and v = [1; x(1:) / (alpha - beta)], the product v^T A(j:s, k) = top_k + d_k /
// (alpha - beta), so every CTA forms the reflector and updates its rows without a second
// reduction. Partials are summed in a fixed order (lane-strided, then a fixed shuffle tree) by every
// CTA alike, so all CTAs hold identical bits and results are reproducible.
//
// FP64 instructions are the scarce resource of this kernel (each FP64 warp instruction holds its
// sub-partition's pipe for the same time whatever its active lanes), so the step is arranged to
// issue few of them and to fill the pipe while the grid barrier settles:
//  * the cross-CTA sums of a step cover only its live slots, packed onto full warps (8, 16 or 32
//    lanes a slot by the number of live slots); thread 0 forms the reflector's scalars as soon as
//    sigma is summed, with one reciprocal square root and one reciprocal;
//  * dot products and the update spread over more lanes (and more warps) as the block's remaining
//    columns shrink, so every sub-partition keeps work; the update's multipliers are formed once a
//    column by 64 lanes, and the update is one FMA an element;
//  * column c stays unscaled while the later columns are updated (the update uses w / (alpha -
//    beta) on x), and becomes v in the same pass that forms the next column's sums;
//  * each CTA arrives at the barrier of step c, then computes the Gram column V(:, 0:b)^T v_b and
//    the maximum |v_b| of the finished column b = c - 1 over its rows, and only then waits (when the
//    block sits in global scratch instead of shared memory, the Gram matrix is formed after the loop).
// CTA 0 holds no rows and CTA 1 only the block's diagonal rows (the CTA that owns them runs its loops
// slower per row); the others share the rest. When the block does not fit in shared memory, each CTA
// keeps its rows in a contiguous region of global scratch.
// The Gram matrix V^T V and the column maxima are reduced once at the end; CTA 0 forms T of the
// compact WY form from them (right-looking: T(0:i, i) = -tau_i sum_b T(0:i, b) G(b, i), each
// column of T added into the later ones as soon as it is final), every CTA writes its rows of V / R
// back in binary64 and cuts them into the row-scaled (Vd) and column-scaled (VTd) digit planes
// with integer operations.
constexpr int kObThreads = 512;
constexpr int kObWarps = kObThreads / 32;
// reduced values of a step: sigma, alpha, d_k (64), top_k (64)
constexpr int kRedSig = 0, kRedAlpha = 1, kRedD = 2, kRedTop = 2 + kOB, kRedSlots = 2 + 2 * kOB;
constexpr size_t kObSmemCap = 188 * 1024;   // dynamic part (the static part is ~36 KB of the 227 KB)

// Row stride of the block in shared memory: at least `rows`, and 8 mod 16 in doubles, so that the two
// columns a half-warp reads in the eight-lane dot products (columns ldw apart) fall on distinct banks.
__host__ __device__ __forceinline__ int64_t ob_ldw(int64_t rows) { return (rows + 15) / 16 * 16 + 8; }

// lanes given to one of n products (or sums) so that n of them fill the CTA's warps: 8, 16 or 32
__device__ __forceinline__ int ob_lanes(int n) { return n > 32 ? 8 : (n > 16 ? 16 : 32); }

// The grid barrier in two halves: arrive (after every thread's prior writes) and wait, so that a CTA
// can do local work while the other CTAs arrive.
__device__ __forceinline__ void ob_arrive(unsigned* cnt) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(cnt), "r"(1u) : "memory");
    }
}
__device__ __forceinline__ bool ob_wait(unsigned* cnt, unsigned nblocks, unsigned k, long long spin_limit, int* err,
                                        int* ok_s) {
    if (threadIdx.x == 0) {
        int ok = 1;
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
        *ok_s = ok && (*(volatile int*)err != CSLS_ERR_TIMEOUT);
    }
    __syncthreads();
    return *ok_s != 0;
}

template <bool SMEM>
__global__ void __launch_bounds__(kObThreads, 1)
k_obpanel(double* A, int64_t lda, int64_t s, int64_t J0, int nbo, int64_t chunk, const int* E, double* tau,
          double* Tb, unsigned short* Vd, unsigned short* VTd, int64_t ldvp, int* frow, int* ecol, double* part,
          unsigned* bar, long long spin, int* err, double* wsc) {
    extern __shared__ __align__(16) double ob_dyn[];
    __shared__ double red[kRedSlots];
    __shared__ double refl[4];   // tau, 1 / (alpha - beta), beta, alpha - beta of the current column
    __shared__ double taus[kOB];
    __shared__ double cmax[kOB];
    __shared__ double gT[kOB * kOB];   // Gram columns (strict upper part), turned into T by CTA 0
    __shared__ double mult[kOB];   // update multipliers of the current column
    __shared__ int ok_s;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t L = s - J0;
    // CTA 0 holds no rows (it forms T at the end while the others cut their digits); CTA 1 holds the
    // block's nd = min(nbo, L) diagonal rows only (the CTA that owns them runs its loops slower per row,
    // so it gets few); CTA g >= 2 holds rows J0 + nd + (g - 2) chunk .. + chunk - 1
    const int64_t nd = (int64_t)nbo < L ? (int64_t)nbo : L;
    const int64_t r0 = g == 0 ? s : (g == 1 ? J0 : J0 + nd + (int64_t)(g - 2) * chunk);
    const int64_t r1 = g == 0 ? s : (g == 1 ? J0 + nd : (r0 + chunk < s ? r0 + chunk : s));
    const int nloc = r1 > r0 ? (int)(r1 - r0) : 0;
    long long* Af = reinterpret_cast<long long*>(A);
    double* W;
    int64_t ldw;
    if (SMEM) {
        W = ob_dyn;
        ldw = ob_ldw(chunk > nd ? chunk : nd);
    } else {
        // a contiguous region of global scratch per CTA (its rows of the block, column-major): the
        // matrix's own column stride would put a CTA's 64 column segments far apart
        W = wsc + (r0 - J0) * kOB;
        ldw = nloc > 0 ? nloc : 1;
    }
    // fixed point -> binary64: this CTA's rows of the block, and (grid-stride) rows 0 .. J0 - 1
    for (int c = 0; c < nbo; ++c) {
        const int e = E[J0 + c];
        const int64_t base = (J0 + c) * lda;
        for (int r = tid; r < nloc; r += kObThreads) {
            const long long v = Af[base + r0 + r];
            W[c * ldw + r] = e > -1000 ? ldexp((double)v, e - kFixBits) : 0.0;
        }
    }
    for (int64_t idx = (int64_t)g * kObThreads + tid; idx < J0 * nbo; idx += (int64_t)G * kObThreads) {
        const int64_t c = J0 + idx / J0, r = idx % J0;
        const int e = E[c];
        A[r + c * lda] = e > -1000 ? ldexp((double)Af[r + c * lda], e - kFixBits) : 0.0;
    }
    for (int i = tid; i < kOB * kOB; i += kObThreads) gT[i] = 0.0;
    __syncthreads();

    auto own = [&](int64_t row) { return row >= r0 && row < r1; };
    // Per step the CTAs exchange (a) summed partials, 64 slots per CTA: sigma (slot 0) and d_k (slot
    // k, k = 1..63), stored CTA-major so that a reduction reads each CTA's slots contiguously; (b) the
    // owner CTA's diagonal-row values alpha and top_k (own[0], own[k]), which need no reduction. Both
    // come in two buffers that alternate by step, so a CTA that runs ahead never overwrites values
    // another CTA is still reading. The Gram matrix V^T V and the column maxima of V are reduced once
    // at the end.
    constexpr int kSlots = kOB;
    constexpr int kGram = kOB * (kOB - 1) / 2;        // strict upper Gram entries, column b at b (b - 1) / 2
    constexpr int kGramSlots = kGram + kOB;            // then the column maxima
    double* const own_base = part + 2 * (int64_t)G * kSlots;
    double* const gram_part = own_base + 2 * (kOB + 1);      // G x kGramSlots, then the reduced entries
    double* const gram_red = gram_part + (int64_t)G * kGramSlots;
    double* const gp = gram_part + (int64_t)g * kGramSlots;
    auto owns = [&](int step) { return own_base + (step & 1) * (kOB + 1); };

    // partial sums that column c (global row jj = J0 + c) needs, written for step c: task 0 is sigma,
    // task t >= 1 is d_{c+t}; P lanes a task (lane q of P takes rows rs + q, rs + q + P, ...), combined
    // by a fixed shuffle tree; a warp whose tasks are all absent issues nothing
    auto column_sums = [&](int c) {
        const int64_t jj = J0 + c;
        const int rs = (int)(jj + 1 - r0 > 0 ? (jj + 1 - r0 < nloc ? jj + 1 - r0 : nloc) : 0);
        double* ps = part + (int64_t)(c & 1) * G * kSlots + (int64_t)g * kSlots;
        double* po = owns(c);
        const int ntask = nbo - c;
        const int P = ob_lanes(ntask);
        const int t = tid / P, q = tid & (P - 1);
        if (warp * (32 / P) < ntask) {
            const bool active = t < ntask;
            const double* xs = W + c * ldw;
            const double* ys = W + (c + (active ? t : 0)) * ldw;
            double acc = 0.0;
            for (int r = (active ? rs : nloc) + q; r < nloc; r += P) acc = fma(xs[r], ys[r], acc);
            for (int o = 1; o < P; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (active && q == 0) {
                ps[t == 0 ? 0 : c + t] = acc;
                if (own(jj)) po[t == 0 ? 0 : c + t] = W[(c + t) * ldw + (jj - r0)];
            }
        }
    };
    // The sums of step c: live slots sigma and d_k (c < k < nbo), P lanes a slot; lane h of P sums
    // the slot over CTAs h, h + P, ... (independent loads), then a fixed shuffle tree; all CTAs obtain
    // the same bits. The lane that finishes a slot also fetches the owner value (alpha or top_k), and
    // thread 0 forms the reflector of column c right away.
    auto reduce_step = [&](int c) {
        const int nlive = nbo - c;
        const int P = ob_lanes(nlive);
        const int i = tid / P, h = tid & (P - 1);
        if (warp * (32 / P) >= nlive) return;   // warp-uniform
        const bool act = i < nlive;
        const int sl = i == 0 ? 0 : c + i;
        double ov = 0.0, acc = 0.0;
        if (act && h == 0) ov = __ldcg(owns(c) + sl);
        if (act) {
            const double* src = part + (int64_t)(c & 1) * G * kSlots + sl;
#pragma unroll 4
            for (int q = h; q < G; q += P) acc += __ldcg(src + (int64_t)q * kSlots);
        }
        for (int o = 1; o < P; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (!act || h != 0) return;
        if (i != 0) {
            red[kRedD + sl] = acc;
            red[kRedTop + sl] = ov;
            return;
        }
        // reflector of column c: beta = -sign(alpha) sqrt(alpha^2 + sigma), tau = (beta - alpha) / beta,
        // 1 / (alpha - beta); 1 / |beta| from one reciprocal square root
        const double sigma = acc, alpha = ov;
        double tau_c = 0.0, scal = 1.0, beta = alpha, amb = 1.0;
        if (sigma != 0.0) {
            const double n2 = fma(alpha, alpha, sigma);
            const double rn = rsqrt(n2);
            const double nrm = n2 * rn;
            beta = alpha >= 0.0 ? -nrm : nrm;
            amb = alpha - beta;   // sign(alpha) (|alpha| + nrm): never 0
            tau_c = fabs(amb) * rn;
            scal = __drcp_rn(amb);
        }
        red[kRedSig] = sigma;
        red[kRedAlpha] = alpha;
        refl[0] = tau_c;
        refl[1] = scal;
        refl[2] = beta;
        refl[3] = amb;
        taus[c] = tau_c;
        if (g == 0) tau[J0 + c] = tau_c;
    };
    // Gram column b (a < b: G(a, b) = v_a^T v_b over this CTA's rows; v_a is 0 above its diagonal row
    // and 1 on it, so only rows from J0 + b on contribute) and the column maximum |v_b| (with its unit
    // entry), into this CTA's partial slots
    auto gram_column = [&](int b) {
        const int64_t db = J0 + b;
        const int rd = (int)(db - r0);
        const int rs = (int)(db - r0 > 0 ? (db - r0 < nloc ? db - r0 : nloc) : 0);
        const int t = tid >> 3, q = tid & 7;
        const double* vb = W + b * ldw;
        if (warp * 4 < b) {   // warp-uniform: some entry a < b in this warp
            const bool active = t < b;
            const double* va = W + (active ? t : 0) * ldw;
            double acc = 0.0;
            for (int r = (active ? rs : nloc) + q; r < nloc; r += 8) acc = fma(va[r], r == rd ? 1.0 : vb[r], acc);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            if (active && q == 0) gp[b * (b - 1) / 2 + t] = acc;
        }
        if (warp == kObWarps - 1) {
            unsigned long long mx = 0x3FF0000000000000ull;   // the unit entry
            for (int r = (rs > rd + 1 ? rs : rd + 1) + lane; r < nloc; r += 32) {
                const unsigned long long u = abs_bits(vb[r]);
                mx = u > mx ? u : mx;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long u = __shfl_xor_sync(0xffffffffu, mx, o);
                mx = u > mx ? u : mx;
            }
            if (lane == 0) gp[kGram + b] = __longlong_as_double((long long)mx);
        }
    };

    unsigned nbar = 0;   // barriers passed (the counter slot of this launch starts at 0)
    column_sums(0);
    for (int c = 0; c < nbo; ++c) {
        ob_arrive(bar);
        if (SMEM && c > 0) gram_column(c - 1);   // the block in global memory: the Gram matrix at the end
        if (!ob_wait(bar, G, nbar++, spin, err, &ok_s)) return;
        reduce_step(c);
        __syncthreads();
        const int64_t jj = J0 + c;
        const double tau_c = refl[0], scal = refl[1], beta = refl[2], amb = refl[3];
        const bool live = red[kRedSig] != 0.0;
        const int rj = (int)(jj - r0);   // local index of the diagonal row (may be outside [0, nloc))
        // A(j:s, k) -= w_k v for the later block columns (rows of this CTA), with w_k = tau v^T A(j:s, k)
        // and v = x / (alpha - beta) below the diagonal row: A(r, k) -= (w_k / (alpha - beta)) y(r) with y = x
        // below the diagonal row and alpha - beta on it (one multiplier a column, formed once by 64 lanes,
        // so one FMA an element); WPC warps a column when few remain
        if (live) {
            if (tid > c && tid < nbo) mult[tid] = -(tau_c * fma(scal, red[kRedD + tid], red[kRedTop + tid])) * scal;
            __syncthreads();
            const int nk = nbo - c - 1;
            const int WPC = nk >= 16 ? 1 : (nk >= 8 ? 2 : (nk >= 4 ? 4 : (nk >= 2 ? 8 : 16)));
            const int cpp = kObWarps / WPC;
            const int rs = rj > 0 ? (rj < nloc ? rj : nloc) : 0;
            const double* x = W + c * ldw;
            for (int k = c + 1 + warp / WPC; k < nbo; k += cpp) {
                const double nws = mult[k];
                double* col = W + k * ldw;
                for (int r = rs + (warp % WPC) * 32 + lane; r < nloc; r += 32 * WPC)
                    col[r] = fma(nws, r == rj ? amb : x[r], col[r]);
            }
        }
        __syncthreads();
        // column c becomes v (beta on the diagonal row); the next column's sums read only later columns
        if (live)
            for (int r = tid; r < nloc; r += kObThreads) {
                if (r > rj) W[c * ldw + r] *= scal;
                else if (r == rj) W[c * ldw + r] = beta;
            }
        if (c + 1 < nbo) column_sums(c + 1);
    }
    __syncthreads();
    if (SMEM) gram_column(nbo - 1);
    if (!SMEM) {
        // the block in global memory: the Gram matrix of V once the loop is done (entries a < b over this
        // CTA's rows, v masked: 0 above its diagonal row, 1 on it; four lanes an entry) and the column
        // maxima of |v| (a warp a column)
        {
            // strict upper entries, four threads per entry: e -> (a, b), a < b, b (b - 1) / 2 <= e < b (b + 1) / 2
            const int ngram = kGramSlots - kOB;
            for (int e0 = 0; e0 < ngram; e0 += kObThreads / 4) {
                const int e = e0 + (tid >> 2), q = tid & 3;
                const bool active = e < ngram;
                int bcol = 1, acol = 0;
                if (active) {
                    bcol = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
                    while (bcol * (bcol - 1) / 2 > e) --bcol;
                    while ((bcol + 1) * bcol / 2 <= e) ++bcol;
                    acol = e - bcol * (bcol - 1) / 2;
                }
                const bool real = active && bcol < nbo;
                const int64_t db = J0 + (real ? bcol : 0);   // rows >= db carry v_b (1 on db)
                const int rs = real ? (int)(db - r0 > 0 ? (db - r0 < nloc ? db - r0 : nloc) : 0) : nloc;
                const int rd = (int)(db - r0);
                const double* va = W + (real ? acol : 0) * ldw;
                const double* vb = W + (real ? bcol : 0) * ldw;
                double a0 = 0.0, a1 = 0.0;
                int r = rs + q;
                for (; r + 4 < nloc; r += 8) {
                    a0 += va[r] * (r == rd ? 1.0 : vb[r]);
                    a1 += va[r + 4] * (r + 4 == rd ? 1.0 : vb[r + 4]);
                }
                if (r < nloc) a0 += va[r] * (r == rd ? 1.0 : vb[r]);
                double acc = a0 + a1;
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                if (active && q == 0) gp[e] = real ? acc : 0.0;
            }
            for (int e = ngram + warp; e < kGramSlots; e += kObWarps) {
                {
                    const int a = e - (kGramSlots - kOB);
                    double mx = a < nbo ? 1.0 : 0.0;   // the unit diagonal entry
                    if (a < nbo) {
                        const int64_t da = J0 + a;
                        const int rs = (int)(da + 1 - r0 > 0 ? (da + 1 - r0 < nloc ? da + 1 - r0 : nloc) : 0);
                        for (int r = rs + lane; r < nloc; r += 32) mx = fmax(mx, fabs(W[a * ldw + r]));
                    }
                    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    if (lane == 0) gp[e] = mx;
                }
            }
        }
    }
    if (nbo < kOB) {   // the entries of absent columns
        for (int e = nbo * (nbo - 1) / 2 + tid; e < kGram; e += kObThreads) gp[e] = 0.0;
        for (int b = nbo + tid; b < kOB; b += kObThreads) gp[kGram + b] = 0.0;
    }
    if (!grid_sync_count(bar, G, nbar++, spin, err)) return;
    // each CTA reduces a share of the entries over the G partials (fixed order), then all CTAs take
    // the column maxima and CTA 0 the Gram matrix
    for (int e = g * kObWarps + warp; e < kGramSlots; e += G * kObWarps) {
        double acc = 0.0;
        const bool is_max = e >= kGram;
        for (int q = lane; q < G; q += 32) {
            const double v = __ldcg(gram_part + (int64_t)q * kGramSlots + e);
            acc = is_max ? fmax(acc, v) : acc + v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = is_max ? fmax(acc, v) : acc + v;
        }
        if (lane == 0) gram_red[e] = acc;
    }
    if (!grid_sync_count(bar, G, nbar++, spin, err)) return;
    if (tid < kOB) cmax[tid] = __ldcg(gram_red + kGram + tid);
    // T of the block (CTA 0): T(i,i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) (V^T V)(0:i, i), right-looking.
    // Column i of the Gram matrix is first scaled by -tau_i (G'), so T(0:i, i) = sum over b < i of
    // T(0:i, b) G'(b, i). Thread (i, a0) keeps acc(a, i) for rows a = a0 + 8k in registers; at step b the
    // threads of column b store it as T(:, b), then every later column adds T(0:b, b) G'(b, i). Column b
    // of gT holds G'(0:b, b) until step b and T(0:b, b) from then on, and only the eight threads of
    // column b touch it in between (ordered by the warp barrier).
    if (g == 0) {
        for (int e = tid; e < kGram; e += kObThreads) {
            int bcol = (int)((1.0 + sqrt(1.0 + 8.0 * (double)e)) * 0.5);
            while (bcol * (bcol - 1) / 2 > e) --bcol;
            while ((bcol + 1) * bcol / 2 <= e) ++bcol;
            gT[(e - bcol * (bcol - 1) / 2) + bcol * kOB] = -taus[bcol] * __ldcg(gram_red + e);
        }
        __syncthreads();
        const int ti = tid >> 3, a0 = tid & 7;
        double acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.0;
        for (int b = 0; b < nbo; ++b) {
            if (ti == b) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int a = a0 + 8 * k;
                    if (a < b) gT[a + b * kOB] = acc[k];
                    else if (a == b) gT[a + b * kOB] = taus[b];
                }
            }
            __syncthreads();
            if (ti > b && ti < nbo) {
                const double gbi = gT[b + ti * kOB];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (8 * k <= b) {
                        const int a = a0 + 8 * k;
                        if (a <= b) acc[k] = fma(gT[a + b * kOB], gbi, acc[k]);
                    }
            }
            __syncwarp();
        }
        __syncthreads();
        for (int i = tid; i < kOB * kOB; i += kObThreads) {
            const int a = i % kOB, b = i / kOB;
            Tb[i] = (a <= b && b < nbo) ? gT[i] : 0.0;
        }
    }
    __syncthreads();
    // column exponents of V (for V^T C) and the digits of this CTA's rows
    __shared__ int ecol_s[kOB];
    if (tid < kOB) {
        ecol_s[tid] = tid < nbo ? exp_of(cmax[tid]) : 0;
        if (g == 0) ecol[tid] = ecol_s[tid];
    }
    __syncthreads();
    for (int r = tid; r < nloc; r += kObThreads) {
        const int64_t grow = r0 + r, lr = grow - J0;
        unsigned long long mxb = 0ull;
        for (int a = 0; a < nbo; ++a) {
            const int64_t d = J0 + a;
            const double v = grow < d ? 0.0 : (grow == d ? 1.0 : W[a * ldw + r]);
            const unsigned long long u = abs_bits(v);
            mxb = u > mxb ? u : mxb;
        }
        const int f = exp_of(__longlong_as_double((long long)mxb));
        frow[lr] = f;
        for (int a0 = 0; a0 < kOB; a0 += 8) {
            uint32_t pk[kDig][4];
#pragma unroll
            for (int jq = 0; jq < 8; ++jq) {
                const int a = a0 + jq;
                const int64_t d = J0 + a;
                const double v = a < nbo ? (grow < d ? 0.0 : (grow == d ? 1.0 : W[a * ldw + r])) : 0.0;
                int dg[kDig], dt[kDig];
                digits_f64(v, f, dg);
                digits_f64(v, ecol_s[a], dt);
#pragma unroll
                for (int p = 0; p < kDig; ++p) {
                    const uint32_t h = bf16_of_int(dg[p]);
                    if (jq & 1) pk[p][jq >> 1] |= h << 16;
                    else pk[p][jq >> 1] = h;
                    VTd[vtd_index(p, a, lr)] = bf16_of_int(dt[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < kDig; ++p)
                reinterpret_cast<uint4*>(Vd)[vd_chunk(p, lr, a0 >> 3)] = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
        }
    }
    // padding rows L .. ldvp - 1 of the digit planes: zero digits
    for (int64_t lr = L + (int64_t)g * kObThreads + tid; lr < ldvp; lr += (int64_t)G * kObThreads) {
        frow[lr] = 0;
        const uint32_t z = (uint32_t)bf16_of_int(0) * 0x10001u;
        for (int a0 = 0; a0 < kOB; a0 += 8)
            for (int p = 0; p < kDig; ++p) reinterpret_cast<uint4*>(Vd)[vd_chunk(p, lr, a0 >> 3)] = make_uint4(z, z, z, z);
        for (int p = 0; p < kDig; ++p)
            for (int a = 0; a < kOB; ++a) VTd[vtd_index(p, a, lr)] = (unsigned short)(z & 0xFFFFu);
    }
    {   // the factored rows back to the matrix, in binary64
        for (int c = 0; c < nbo; ++c)
            for (int r = tid; r < nloc; r += kObThreads) A[(r0 + r) + (J0 + c) * lda] = W[c * ldw + r];
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
//                        integer below 6 x 64 x 2^14 < 2^23); one MMA per V plane p and K step
//                        covers the levels p .. 5 (Wn planes stacked along N); two accumulator
//                        sets of 6 x 32 columns, so the MMAs of tile i + 1 run while tile i is
//                        written back;
//   warps 2..17          epilogue: TMEM -> registers, levels combined in int64, scaled onto the
//                        column's fixed-point grid and added into the staged C block in shared
//                        memory (one thread per row and 8 columns); warp 0 writes the block back
//                        with one 2D tensor store (outside the matrix nothing is written) before
//                        the stage takes the next C block, and fetches the block two tiles ahead
//                        into L2.
// Every wait is bounded (spin polls and 2 s of wall time); a role that gives up sets the CTA's
// abort flag and the error word, and the CTA still waits for its copies and MMAs in flight and
// frees its tensor memory before it returns.
constexpr int kTcLevels = kLev + 1;
constexpr int kTcPlaneA = kTcM * kOB * 2;        // bytes of one V digit plane tile (16 KB)
constexpr int kTcPlaneB = kTcN * kOB * 2;        // bytes of one Wn digit plane tile (4 KB)
constexpr int kTcBufCols = kTcLevels * kTcN;     // TMEM columns of one accumulator set (192)
constexpr int kTcTmemCols = 512;
constexpr int kTcEpiWarps = 16;
constexpr int kTcEpiCols = kTcN / (kTcEpiWarps / 4);   // columns of a tile per epilogue warp (8)
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr unsigned long long kTcWaitNs = 2000000000ULL;
constexpr long long kTeardownSpin = 1LL << 62;   // teardown waits: bounded by kTcWaitNs alone

struct TcUpdSmem {
    unsigned char A[kDig][kTcPlaneA];
    unsigned char B[2][kDig][kTcPlaneB];
    long long C[2][kTcN][kTcM];
    uint64_t full_a, full_b[2], full_c[2], done[2], tfree[2], freed[2], drain;
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

// 2D tiled tensor copy shared -> global (the box at coordinates x, y; parts outside the tensor are not
// written), as one bulk group; the box at x, y into L2 only; and the waits for this thread's bulk
// groups: reads of shared memory done, or the whole copy done
__device__ __forceinline__ void tensor_s2g_2d(const void* src, const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n"
                 "cp.async.bulk.commit_group;" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(tc::smem_addr(src))
                 : "memory");
}
__device__ __forceinline__ void tensor_prefetch_l2_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(kTcThreads, 1)
k_emu_update_tc(const __grid_constant__ CUtensorMap cmap, long long* Cfix, int64_t lda, int64_t s, int64_t J0, int nbo,
                const unsigned short* Vd, const int* frow, const unsigned short* Wd, const int* gsh,
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
            tc::mbar_init(&sm.tfree[b], 32 * kTcEpiWarps);
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
            // uses of each stage whose B (Wn digits) and C copies were issued
            int armedB0 = 0, armedB1 = 0, armedC0 = 0, armedC1 = 0;
            int stored = 0;   // tiles written back by a tensor store
            tc::mbar_arrive_expect_tx(&sm.full_a, kDig * kTcPlaneA);
            tc::bulk_g2s(sm.A[0], reinterpret_cast<const unsigned char*>(Vd) + rt * (kDig * kTcPlaneA),
                         kDig * kTcPlaneA, &sm.full_a);
            for (int i = 0; i < ntile; ++i) {
                const int b = i & 1, u = i >> 1;
                // stage b's Wn digits are free once tile i - 2's accumulators were read (its MMAs are
                // done); its C block once tile i - 2's updated values, folded into it by the epilogue,
                // have been read out by that tile's tensor store
                if (u > 0 && !tc::mbar_wait(&sm.tfree[b], (u - 1) & 1, spin, kTcWaitNs, abort)) {
                    *abort = 1;
                    set_error(err, CSLS_ERR_TIMEOUT);
                    break;
                }
                const int64_t ct = ct0 + i;
                tc::mbar_arrive_expect_tx(&sm.full_b[b], kDig * kTcPlaneB);
                tc::bulk_g2s(sm.B[b][0], reinterpret_cast<const unsigned char*>(Wd) + ct * (kDig * kTcPlaneB),
                             kDig * kTcPlaneB, &sm.full_b[b]);
                if (b) armedB1 = u + 1;
                else armedB0 = u + 1;
                if (u > 0) {
                    if (!tc::mbar_wait(&sm.freed[b], (u - 1) & 1, spin, kTcWaitNs, abort)) {
                        *abort = 1;
                        set_error(err, CSLS_ERR_TIMEOUT);
                        break;
                    }
                    tensor_s2g_2d(sm.C[b][0], &cmap, (int)(J0 + rb), (int)(jc + (ct - 2) * kTcN));
                    ++stored;
                    bulk_wait_read_all();
                }
                tc::mbar_arrive_expect_tx(&sm.full_c[b], kTcN * kTcM * 8);
                tensor_g2s_2d(sm.C[b][0], &cmap, (int)(J0 + rb), (int)(jc + ct * kTcN), &sm.full_c[b]);
                // two stages hold only about one C block in flight per SM: tile i + 2's block is fetched
                // into L2 now, so its copy into shared memory (after tile i's write-back) hits L2
                if (i + 2 < ntile) tensor_prefetch_l2_2d(&cmap, (int)(J0 + rb), (int)(jc + (ct + 2) * kTcN));
                if (b) armedC1 = u + 1;
                else armedC0 = u + 1;
            }
            // the last tiles' write-backs (tiles stored .. ntile - 1, one per stage)
            for (int t = stored; t < ntile && !*abort; ++t) {
                const int b = t & 1, u = t >> 1;
                if (!tc::mbar_wait(&sm.freed[b], u & 1, spin, kTcWaitNs, abort)) {
                    *abort = 1;
                    set_error(err, CSLS_ERR_TIMEOUT);
                    break;
                }
                tensor_s2g_2d(sm.C[b][0], &cmap, (int)(J0 + rb), (int)(jc + (ct0 + t) * kTcN));
            }
            bulk_wait_all();   // tensor stores complete before the CTA leaves
            // copies in flight land before the CTA can leave. Issued copies always complete, so
            // these waits are bounded by wall time only (not by the caller's spin count, which
            // may be tiny): a CTA never exits with a copy still writing its shared memory.
            tc::mbar_wait(&sm.full_a, 0, kTeardownSpin, kTcWaitNs, nullptr);
            if (armedB0) tc::mbar_wait(&sm.full_b[0], (armedB0 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
            if (armedC0) tc::mbar_wait(&sm.full_c[0], (armedC0 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
            if (armedB1) tc::mbar_wait(&sm.full_b[1], (armedB1 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
            if (armedC1) tc::mbar_wait(&sm.full_c[1], (armedC1 - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            bool issued = false;
            if (tc::mbar_wait(&sm.full_a, 0, spin, kTcWaitNs, abort)) {
                const uint64_t adesc = tc::smem_desc(tc::smem_addr(sm.A[0]), kTcM * 16, 128);
                for (int i = 0; i < ntile; ++i) {
                    const int b = i & 1, u = i >> 1;
                    // the accumulator set of this stage was drained by the epilogue of tile i - 2
                    if ((u > 0 && !tc::mbar_wait(&sm.tfree[b], (u - 1) & 1, spin, kTcWaitNs, abort)) ||
                        !tc::mbar_wait(&sm.full_b[b], u & 1, spin, kTcWaitNs, abort)) {
                        *abort = 1;
                        set_error(err, CSLS_ERR_TIMEOUT);
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t bdesc = tc::smem_desc(tc::smem_addr(sm.B[b][0]), kTcNStack * 16, 128);
                    const uint32_t d0 = tmem + (uint32_t)(b * kTcBufCols);
                    // 24 MMAs, fully unrolled: for V plane p one MMA per K step of 16 against the
                    // stacked Wn planes 0 .. 5 - p (N = 32 (6 - p)), accumulating levels p .. 5 in
                    // their adjacent TMEM blocks. The first MMA (p = 0, N = 192) starts every level
                    // block from zero. Each descriptor is the stage's base plus a constant (the start
                    // address sits in the low bits, in 16-byte units); a K step is two core matrices.
#pragma unroll
                    for (int p = 0; p <= kLev; ++p)
#pragma unroll
                        for (int k = 0; k < kOB / 16; ++k)
                            tc::mma_bf16(d0 + p * kTcN,
                                         adesc + (uint64_t)((p * kTcPlaneA + k * 2 * (kTcM * 16)) >> 4),
                                         bdesc + (uint64_t)((k * 2 * (kTcNStack * 16)) >> 4),
                                         tc::idesc_bf16_f32(kTcM, kTcN * (kDig - p)), (p | k) != 0);
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
        const int part = (warp - 2) >> 2;          // columns kTcEpiCols part .. + kTcEpiCols - 1 of each tile
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
            const uint32_t ta =
                tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTcBufCols + part * kTcEpiCols);
            uint32_t v[kTcLevels][kTcEpiCols];
#pragma unroll
            for (int l = 0; l < kTcLevels; ++l) tc::tmem_ld8(ta + l * kTcN, v[l]);
            tc::tmem_ld_wait();
            tc::fence_before_sync();
            tc::mbar_arrive(&sm.tfree[b]);   // the accumulator set may take tile i + 2's MMAs now
            const int64_t cbase = (ct0 + i) * kTcN + part * kTcEpiCols;
#pragma unroll
            for (int j = 0; j < kTcEpiCols; ++j) {
                const int64_t col = cbase + j;
                if (rok && col < nprime) {
                    // acc = sum_l T_l 256^(5 - l): T_0 256 + T_1 fits 32 bits (|T_0| <= 64 x 2^14), the
                    // rest is three 32 x 32 -> 64-bit multiply-adds. Levels 0..3 have at most 4 digit
                    // pairs, |T_l| <= 4 x 64 x 2^14 = 2^22, and are read by the magic-number add (one
                    // FP32 add, one integer subtract); levels 4 and 5 by a conversion instruction.
                    const int t0 = magic_int(__uint_as_float(v[0][j]));
                    const int t1 = magic_int(__uint_as_float(v[1][j]));
                    const int t2 = magic_int(__uint_as_float(v[2][j]));
                    const int t3 = magic_int(__uint_as_float(v[3][j]));
                    const int t4 = __float2int_rn(__uint_as_float(v[4][j]));
                    const int t5 = __float2int_rn(__uint_as_float(v[5][j]));
                    long long acc = (long long)t2 * (1LL << 24) + ((long long)t3 * 65536 + ((long long)t4 * 256 + t5));
                    acc += (long long)(t0 * 256 + t1) << 32;
                    // Cfix += acc * 2^(f_r + gsh_c), rounded to the fixed-point grid
                    const int sh = fr + gsh[col];
                    long long dlt;
                    if (sh >= 0) dlt = sh < 63 ? acc << sh : 0;
                    else dlt = -sh < 63 ? (acc + (1LL << (-sh - 1))) >> (-sh) : 0;
                    sm.C[b][part * kTcEpiCols + j][r] += dlt;   // written back by the tile's tensor store
                }
            }
            // generic-proxy shared-memory writes become visible to the tensor store (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_arrive(&sm.freed[b]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTcTmemCols);
    }
}

// ------------------------------------------------------------------ W = V^T C on tcgen05 (split over row chunks)
//
// One CTA per (128-column tile of C, chunk of rows). The product is D = C^T V (128 C columns on
// the TMEM lanes x 64 V columns), cut into digit planes: C digits (A operand, plane q) times V
// digits (B operand). The six V planes are stacked along N (row p x 64 + a of a 384-row operand),
// so one MMA multiplies C plane q by V planes p0 .. p0 + w - 1 and accumulates levels q + p0 ..
// q + p0 + w - 1, whose 64-column TMEM blocks are adjacent (levels 0..5 occupy columns 0..383).
// Levels p + q <= 5 are kept: per K step of 16 rows 8 MMAs (N <= 256) cover the 21 digit pairs.
// Level sums are exact in FP32 while below 2^24; a window of 128 rows keeps them below
// 6 x 128 x 2^14 = 1.5 x 2^23, after which the drain warps fold the window into one int64 per
// output, sum_l T_l 2^(8 (5 - l)). That int64 stays below 2^54 sqrt(rows) (Cauchy-Schwarz with
// |N_v| < 2^47 and sum_r N_c(r)^2 < 2^94 from the column-norm scale), so chunks of up to 2^14 rows
// cannot overflow it.
// Roles (704 threads):
//   warp 0 (one thread)  copies: per K-block of 32 rows the raw int64 C rows (two 16-row x 128-
//                        column tensor boxes, 128-byte swizzle) and the block's V digits (one 24 KB
//                        bulk copy; the panel kernel writes them in this K-major core-matrix order);
//   warp 1 (one thread)  the MMAs, two stages of operands;
//   warps 2..5           cut the raw C rows into six bf16 digit planes in shared memory (one C
//                        column per thread, read through the swizzle without bank conflicts);
//   warps 6..21          drain the TMEM level sums every window into int64 registers (one C
//                        column per thread and 16 V columns, four warps on each TMEM lane
//                        quarter) and write the chunk's partial W.
// Every wait is bounded (spin polls and wall time); a role that gives up sets the abort flag and
// the error word; copies and MMAs in flight are still awaited (wall time only) before the CTA frees
// its tensor memory and exits.
constexpr int kVcM = 128;                           // C columns per tile (TMEM lanes)
constexpr int kVcKB = 32;                           // rows per K-block (pipeline stage)
constexpr int kVcWin = 4;                           // K-blocks per exact accumulation window (128 rows)
constexpr int kVcNStack = kDig * kOB;               // 384 rows of the stacked V-digit operand
constexpr int kVcPlaneA = kVcM * kVcKB * 2;         // 8 KB: one C-digit plane of a K-block
constexpr int kVcBBytes = kVcNStack * kVcKB * 2;    // 24 KB: the stacked V digits of a K-block
constexpr int kVcRawBox = 16;                       // rows per raw-C tensor box (128 bytes)
constexpr int kVcRawBytes = kVcM * kVcKB * 8;       // 32 KB of raw C per K-block
constexpr int kVcCutWarps = 4, kVcDrainWarps = 16;
constexpr int kVcDrainCols = 4 * kOB / kVcDrainWarps;   // V columns a drain thread folds (16)
constexpr int kVcThreads = 32 * (2 + kVcCutWarps + kVcDrainWarps);
constexpr int kVcMaxChunk = 1 << 14;                // rows per chunk (int64 accumulator bound)

struct VcSmem {
    unsigned char raw[2][kVcRawBytes];              // 1024-byte aligned (swizzled tensor boxes)
    unsigned char cd[2][kDig][kVcPlaneA];
    unsigned char vd[2][kVcBBytes];
    uint64_t full_raw[2], empty_raw[2], full_cd[2], full_vd[2], empty_op[2], acc_full, acc_empty, drain;
    uint32_t tmem;
    int abort;
};

// 704 threads: 22 warps put 6 on two sub-partitions, whose 16,384 registers then allow 80 a thread
__global__ void __maxnreg__(80)
k_emu_vtc_tc(const __grid_constant__ CUtensorMap rawmap, const unsigned short* VTd, int64_t J0, int nbo, int64_t L,
             int64_t kc, const int* ecol, const int* E, double* Wp, int64_t nprime, long long spin, int* err) {
    extern __shared__ __align__(1024) unsigned char vc_smem_raw[];
    // the 128-byte swizzle of the raw-C boxes needs a 1024-byte aligned destination: the launch
    // gives 1 KB of slack, the structure starts at the first 1024-byte boundary
    const uint32_t base = tc::smem_addr(vc_smem_raw);
    VcSmem& sm = *reinterpret_cast<VcSmem*>(vc_smem_raw + (((base + 1023u) & ~1023u) - base));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t jc = J0 + nbo;
    const int64_t c0 = (int64_t)blockIdx.x * kVcM;
    const int64_t lb = (int64_t)blockIdx.y * kc;
    const int64_t le = lb + kc < L ? lb + kc : L;
    const int nkb = (int)ceil_div_dev(le - lb, kVcKB);
    const int nwin = (nkb + kVcWin - 1) / kVcWin;
    volatile int* abort = &sm.abort;
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&sm.full_raw[b], 1);
            tc::mbar_init(&sm.empty_raw[b], 32 * kVcCutWarps);
            tc::mbar_init(&sm.full_cd[b], 32 * kVcCutWarps);
            tc::mbar_init(&sm.full_vd[b], 1);
            tc::mbar_init(&sm.empty_op[b], 1);
        }
        tc::mbar_init(&sm.acc_full, 1);
        tc::mbar_init(&sm.acc_empty, 32 * kVcDrainWarps);
        tc::mbar_init(&sm.drain, 1);
        sm.abort = 0;
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(&sm.tmem, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    auto fail = [&]() {
        *abort = 1;
        set_error(err, CSLS_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int armed0 = 0, armed1 = 0;   // uses of each stage whose copies were issued (negative: raw only)
            for (int i = 0; i < nkb; ++i) {
                const int st = i & 1, u = i >> 1;
                if (u > 0 && !tc::mbar_wait(&sm.empty_raw[st], (u - 1) & 1, spin, kTcWaitNs, abort)) { fail(); break; }
                const int64_t row = J0 + lb + (int64_t)i * kVcKB;
                tc::mbar_arrive_expect_tx(&sm.full_raw[st], kVcRawBytes);
                tensor_g2s_2d(sm.raw[st], &rawmap, (int)row, (int)(jc + c0), &sm.full_raw[st]);
                tensor_g2s_2d(sm.raw[st] + kVcRawBytes / 2, &rawmap, (int)(row + kVcRawBox), (int)(jc + c0),
                              &sm.full_raw[st]);
                if (u > 0 && !tc::mbar_wait(&sm.empty_op[st], (u - 1) & 1, spin, kTcWaitNs, abort)) {
                    if (st) armed1 = -(u + 1);   // raw copy issued, V copy not
                    else armed0 = -(u + 1);
                    fail();
                    break;
                }
                tc::mbar_arrive_expect_tx(&sm.full_vd[st], kVcBBytes);
                tc::bulk_g2s(sm.vd[st], reinterpret_cast<const unsigned char*>(VTd) + (lb + (int64_t)i * kVcKB) * (kVcNStack * 2),
                             kVcBBytes, &sm.full_vd[st]);
                if (st) armed1 = u + 1;
                else armed0 = u + 1;
            }
            // copies in flight land before the CTA leaves (issued copies always complete)
            for (int st = 0; st < 2; ++st) {
                const int ar = st ? armed1 : armed0;
                const int a = ar < 0 ? -ar : ar;
                if (a == 0) continue;
                tc::mbar_wait(&sm.full_raw[st], (a - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
                if (ar > 0) tc::mbar_wait(&sm.full_vd[st], (a - 1) & 1, kTeardownSpin, kTcWaitNs, nullptr);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            bool issued = false;
            const uint64_t bdA = tc::smem_desc(tc::smem_addr(sm.vd[0]), kVcNStack * 16, 128);
            const uint64_t bdB = tc::smem_desc(tc::smem_addr(sm.vd[1]), kVcNStack * 16, 128);
            const uint64_t adA = tc::smem_desc(tc::smem_addr(sm.cd[0][0]), kVcM * 16, 128);
            const uint64_t adB = tc::smem_desc(tc::smem_addr(sm.cd[1][0]), kVcM * 16, 128);
            for (int i = 0; i < nkb; ++i) {
                const int st = i & 1, u = i >> 1, w = i / kVcWin;
                const bool first = (i % kVcWin) == 0;
                if ((first && w > 0 && !tc::mbar_wait(&sm.acc_empty, (w - 1) & 1, spin, kTcWaitNs, abort)) ||
                    !tc::mbar_wait(&sm.full_cd[st], u & 1, spin, kTcWaitNs, abort) ||
                    !tc::mbar_wait(&sm.full_vd[st], u & 1, spin, kTcWaitNs, abort)) {
                    fail();
                    break;
                }
                tc::fence_after_sync();
#pragma unroll
                for (int k = 0; k < kVcKB / 16; ++k) {
                    const uint64_t ak = (st ? adB : adA) + (uint64_t)((k * 2 * (kVcM * 16)) >> 4);
                    const uint64_t bk = (st ? bdB : bdA) + (uint64_t)((k * 2 * (kVcNStack * 16)) >> 4);
                    const uint32_t z = (first && k == 0) ? 0u : 1u;
                    // (q, p0, w): C plane q times V planes p0 .. p0 + w - 1 -> levels q + p0 ..
#define VC_MMA(q, p0, wdt, acc)                                                                              \
    tc::mma_bf16(tmem + (uint32_t)(kOB * ((q) + (p0))), ak + (uint64_t)(((q) * kVcPlaneA) >> 4),              \
                 bk + (uint64_t)(((p0) * kOB * 16) >> 4), tc::idesc_bf16_f32(kVcM, kOB * (wdt)), (acc))
                    VC_MMA(0, 0, 4, z);
                    VC_MMA(0, 4, 2, z);
                    VC_MMA(1, 0, 4, 1u);
                    VC_MMA(1, 4, 1, 1u);
                    VC_MMA(2, 0, 4, 1u);
                    VC_MMA(3, 0, 3, 1u);
                    VC_MMA(4, 0, 2, 1u);
                    VC_MMA(5, 0, 1, 1u);
#undef VC_MMA
                }
                tc::mma_commit(&sm.empty_op[st]);
                if ((i % kVcWin) == kVcWin - 1 || i == nkb - 1) tc::mma_commit(&sm.acc_full);
                issued = true;
            }
            if (issued) {   // every MMA has completed before the tensor memory is freed (wall-time bound only)
                tc::mma_commit(&sm.drain);
                tc::mbar_wait(&sm.drain, 0, kTeardownSpin, kTcWaitNs, nullptr);
            }
        }
        __syncwarp();
    } else if (warp < 2 + kVcCutWarps) {
        // cutters: thread m owns C column m of the tile
        const int m = threadIdx.x - 64;
        for (int i = 0; i < nkb; ++i) {
            const int st = i & 1, u = i >> 1;
            const bool ok = tc::mbar_wait(&sm.full_raw[st], u & 1, spin, kTcWaitNs, abort) &&
                            (u == 0 || tc::mbar_wait(&sm.empty_op[st], (u - 1) & 1, spin, kTcWaitNs, abort));
            if (!ok) {
                fail();
                break;
            }
#pragma unroll 1
            for (int kg = 0; kg < kVcKB / 8; ++kg) {
                // rows 8 kg .. 8 kg + 7: box kg / 2, 16-byte chunks 4 (kg % 2) .. + 3 of row m (swizzled)
                const unsigned char* box = sm.raw[st] + (kg >> 1) * (kVcRawBytes / 2) + m * 128;
                long long cv[8];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int chunk = (4 * (kg & 1) + h) ^ (m & 7);
                    const longlong2 t = *reinterpret_cast<const longlong2*>(box + chunk * 16);
                    cv[2 * h] = t.x;
                    cv[2 * h + 1] = t.y;
                }
                uint32_t pk[kDig][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    float f0[kDig], f1[kDig];
                    digit_floats_fix(cv[e], f0);
                    digit_floats_fix(cv[e + 1], f1);
#pragma unroll
                    for (int q = 0; q < kDig; ++q) pk[q][e >> 1] = pack_bf16x2(f0[q], f1[q]);
                }
#pragma unroll
                for (int q = 0; q < kDig; ++q)
                    *reinterpret_cast<uint4*>(sm.cd[st][q] + (kg * kVcM + m) * 16) =
                        make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
            }
            // generic-proxy shared-memory writes become visible to the tensor core (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_arrive(&sm.full_cd[st]);
            tc::mbar_arrive(&sm.empty_raw[st]);
        }
    } else {
        // drain: TMEM lanes 32 (warp % 4) .. + 31, V columns 16 grp .. + 15 (four warps on each lane
        // quarter, so their TMEM loads and folds overlap)
        const int quarter = warp & 3, grp = (warp - 2 - kVcCutWarps) >> 2;
        const int m = quarter * 32 + lane;
        long long acc[kVcDrainCols];
#pragma unroll
        for (int a = 0; a < kVcDrainCols; ++a) acc[a] = 0;
        bool ok_all = true;
        for (int w = 0; w < nwin; ++w) {
            bool ok = tc::mbar_wait(&sm.acc_full, w & 1, spin, kTcWaitNs, abort);
            ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld is warp-wide
            if (!ok) {
                fail();
                ok_all = false;
                break;
            }
            tc::fence_after_sync();
            // each level folds into the int64 sums with weight 2^(8 (5 - l)): levels 0 and 1 (at most
            // 2 x 128 x 2^14 = 2^22 per window: magic-number read) add into the high word (weights 2^40
            // and 2^32), levels 2..5 by one 32 x 32 -> 64-bit multiply-add each
            // two levels a TMEM wait (three waits a window)
            const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(kVcDrainCols * grp);
#pragma unroll 1
            for (int l = 0; l <= kLev; l += 2) {
                uint32_t v[kVcDrainCols], u[kVcDrainCols];
                tc::tmem_ld16(tq + (uint32_t)(kOB * l), v);
                tc::tmem_ld16(tq + (uint32_t)(kOB * (l + 1)), u);
                tc::tmem_ld_wait();
                if (l + 2 > kLev) {   // the window's last TMEM reads are done: the MMAs may go on while this folds
                    tc::fence_before_sync();
                    tc::mbar_arrive(&sm.acc_empty);
                }
                if (l == 0) {
#pragma unroll
                    for (int j = 0; j < kVcDrainCols; ++j)
                        acc[j] = add_hi32(acc[j], magic_int(__uint_as_float(v[j])) * 256 + magic_int(__uint_as_float(u[j])));
                } else {
                    const int mul = 1 << (8 * (kLev - l));
#pragma unroll
                    for (int j = 0; j < kVcDrainCols; ++j) {
                        acc[j] = mad_wide_s32(__float2int_rn(__uint_as_float(v[j])), mul, acc[j]);
                        acc[j] = mad_wide_s32(__float2int_rn(__uint_as_float(u[j])), mul >> 8, acc[j]);
                    }
                }
            }
        }
        if (ok_all) {
            // W(a, c) = acc 2^(e_a + E_c - 54) (V digits carry 2^(e_a - 47), C digits 2^(E_c - 47), acc 2^-40)
            const int64_t col = c0 + m;
            double* out = Wp + (int64_t)blockIdx.y * kOB * nprime;
            if (col < nprime) {
                const int ec = E[jc + col];
#pragma unroll
                for (int j = 0; j < kVcDrainCols; ++j) {
                    const int a = kVcDrainCols * grp + j;
                    if (a < nbo) out[(int64_t)a * nprime + col] = ldexp((double)acc[j], ecol[a] + ec - 54);
                }
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
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

// Tensor map of the int64 trailing matrix for the W = V^T C copies: 16-row (128-byte) x 128-column
// boxes with the 128-byte swizzle, so the cutters read a column's 16-byte chunks conflict-free.
static int make_raw_map(CUtensorMap* map, void* A, int64_t lda, int64_t s, int64_t n) {
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
    const cuuint32_t box[2] = {(cuuint32_t)kVcRawBox, (cuuint32_t)kVcM};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, A, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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
    int* ecol;                    // kOB
    int* frow;                    // s
    int* gsh;                     // n: per-column shift of the update products
    unsigned short* Vd;           // kDig * s * kOB (s rounded up to 128)
    unsigned short* VTd;          // kDig * kOB * s
    unsigned short* Wd;           // kDig * n * kOB (n rounded up to 32)
    double* Wp;                   // split-K partials of W (kOB x n per chunk)
    int64_t wp_elems;
    double* Wn;                   // kOB x n
    double* Tb;                   // outer block's T (kOB x kOB)
    double* Ws;                   // the panel block when it does not fit in shared memory (s x kOB)
    unsigned* bar_cnt;            // one grid-barrier counter per outer block (zeroed per factorisation)
};

constexpr int kVcMaxSplit = 16;   // row chunks of W = V^T C (partials kept side by side)
static int64_t emu_wp_elems(int64_t n) { return (int64_t)kVcMaxSplit * kOB * (n + kVcM); }

static EmuScratch emu_carve(Carve& c, int64_t s, int64_t n) {
    const int64_t ldv = round_up(s, kTcM), ldw = round_up(n, kTcN);
    EmuScratch e;
    e.E = c.take<int>((size_t)n);
    e.ecol = c.take<int>(kOB);
    e.frow = c.take<int>((size_t)ldv);
    e.gsh = c.take<int>((size_t)ldw);
    e.Vd = c.take<unsigned short>((size_t)(kDig * ldv * kOB));
    e.VTd = c.take<unsigned short>((size_t)(kDig * ldv * kOB));
    e.Wd = c.take<unsigned short>((size_t)(kDig * ldw * kOB));
    e.wp_elems = emu_wp_elems(n);
    e.Wp = c.take<double>((size_t)e.wp_elems);
    e.Wn = c.take<double>((size_t)(kOB * (n + kOB)));
    e.Tb = c.take<double>(kOB * kOB);
    e.Ws = c.take<double>((size_t)(round_up(s, 32) * kOB));
    e.bar_cnt = c.take<unsigned>((size_t)ceil_div(n, kOB) + 1);
    return e;
}

// doubles of the panel's exchange buffer: per-step slots (two buffers), owner values, the Gram
// partials of every CTA and their reduction
int64_t obpanel_partial_elems(int sms) {
    const int64_t gram = kOB * (kOB - 1) / 2 + kOB;
    return (int64_t)sms * (2 * kOB + gram) + 2 * (kOB + 1) + gram + 64;
}

size_t qr_emu_scratch_bytes(int64_t s, int64_t n) {
    Carve c{nullptr, 0, 0, true};
    emu_carve(c, s, n);
    return c.off;
}

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
    CUtensorMap rawmap;
    CSLS_TRY(make_raw_map(&rawmap, A, lda, s, n));
    CSLS_TRY(raise_smem_limit((const void*)k_emu_vtc_tc, (int)(sizeof(VcSmem) + 1024)));
    CSLS_TRY(raise_smem_limit((const void*)k_emu_update_tc, (int)sizeof(TcUpdSmem)));
    CSLS_TRY(raise_smem_limit((const void*)k_wreduce_ob, (int)kWrSmem));
    const int sms = device_sm_count();
    CSLS_CUDA(cudaMemsetAsync(q.bar, 0, sizeof(GridBarrier), st));
    CSLS_CUDA(cudaMemsetAsync(e.bar_cnt, 0, sizeof(unsigned) * (size_t)(ceil_div(n, kOB) + 1), st));
    k_col_exponent<<<(unsigned)std::min<int64_t>(n, 65535), 256, 0, st>>>(A, lda, s, n, e.E);
    CSLS_CUDA(cudaGetLastError());
    dim3 fg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(s, 1024), 64)), (unsigned)std::min<int64_t>(n, 65535));
    k_to_fixed<<<fg, 256, 0, st>>>(A, lda, s, n, e.E);
    CSLS_CUDA(cudaGetLastError());
    int64_t nl = 2;
    const size_t ob_cap = kObSmemCap;
    CSLS_TRY(raise_smem_limit((const void*)k_obpanel<true>, (int)ob_cap));
    for (int64_t J0 = 0; J0 < n; J0 += kOB) {
        const int nbo = (int)(n - J0 < kOB ? n - J0 : kOB);
        const int64_t L = s - J0;
        const int64_t ldvp = round_up(L, kTcM);   // digit planes use the current block height
        // the outer block: fixed point -> binary64, Householder factorisation, T, digits of V
        {
            // CTA 0 holds no rows, CTA 1 the block's nd diagonal rows, G - 2 CTAs share the other rows
            const int64_t nd = std::min<int64_t>(nbo, L), rest = L - nd;
            int G = 2;
            int64_t chunk = nd;
            if (rest > 0) {
                const int Gr = (int)std::min<int64_t>(sms - 2, std::max<int64_t>(1, ceil_div(rest, 128)));
                chunk = ceil_div(rest, Gr);
                G = (int)ceil_div(rest, chunk) + 2;
            }
            const size_t smem = (size_t)ob_ldw(std::max(chunk, nd)) * nbo * sizeof(double);
            const bool in_smem = smem <= ob_cap;
            int64_t J0v = J0, ldav = lda, sv = s, ldvpv = ldvp;
            int nbov = nbo;
            long long spinv = spin;
            double* tau = q.tau;
            double* part = q.partials;
            unsigned* bar = e.bar_cnt + (J0 / kOB);   // a zeroed counter slot per outer block
            void* args[] = {&A, &ldav, &sv, &J0v, &nbov, &chunk, (void*)&e.E, &tau, (void*)&e.Tb, (void*)&e.Vd,
                            (void*)&e.VTd, &ldvpv, (void*)&e.frow, (void*)&e.ecol, &part, &bar, &spinv, &err,
                            (void*)&e.Ws};
            // algorithmic FP64 work: Householder factorisation of the L x nbo block (2 nbo^2 (L - nbo / 3))
            // and the strict upper Gram matrix of V for T (sum over b of 2 b (L - b))
            const double fb = (double)nbo, fL = (double)L;
            const double panel_flop = 2.0 * fb * fb * (fL - fb / 3.0) + fL * fb * (fb - 1.0) -
                                      (fb - 1.0) * fb * (2.0 * fb - 1.0) / 3.0;
            const int tk = kt_begin(kFamPanel, st);
            if (in_smem)
                CSLS_CUDA(cudaLaunchCooperativeKernel((const void*)k_obpanel<true>, dim3(G), dim3(kObThreads), args,
                                                      smem, st));
            else
                CSLS_CUDA(cudaLaunchCooperativeKernel((const void*)k_obpanel<false>, dim3(G), dim3(kObThreads), args,
                                                      0, st));
            kt_end(tk, panel_flop, st);
            nl += 1;
        }
        const int64_t nprime = n - J0 - nbo;
        if (nprime <= 0) continue;
        // W = V^T C over row chunks: the split that minimises waves x rows per CTA (plus a fixed
        // cost of about two K-blocks per CTA), with chunks of at most kVcMaxChunk rows
        const int64_t ntn = ceil_div(nprime, kVcM);
        int64_t ks = 1, best = INT64_MAX;
        for (int64_t k = 1; k <= kVcMaxSplit; ++k) {
            const int64_t kcb = round_up(ceil_div(L, k), kVcKB);
            if (kcb > kVcMaxChunk) continue;
            const int64_t cost = ceil_div(ntn * ceil_div(L, kcb), sms) * (kcb / kVcKB + 2);
            if (cost < best) { best = cost; ks = k; }
        }
        const int64_t kc = round_up(ceil_div(L, ks), kVcKB);
        ks = ceil_div(L, kc);
        if (kc > kVcMaxChunk || ks > kVcMaxSplit) return CSLS_ERR_ARG;   // rows beyond the accumulator bound
        const double prod_flop = 2.0 * (double)L * (double)nprime * (double)nbo;
        int tk = kt_begin(kFamVtc, st);
        k_emu_vtc_tc<<<dim3((unsigned)ntn, (unsigned)ks), kVcThreads, sizeof(VcSmem) + 1024, st>>>(
            rawmap, e.VTd, J0, nbo, L, kc, e.ecol, e.E, e.Wp, nprime, spin, err);
        CSLS_CUDA(cudaGetLastError());
        kt_end(tk, prod_flop, st);
        k_wreduce_ob<<<(unsigned)ceil_div(nprime, kWrCols), 256, kWrSmem, st>>>(e.Wp, (int)ks, e.Tb, nbo, e.Wn, nprime);
        CSLS_CUDA(cudaGetLastError());
        // digits of Wn, then the exact update
        const int64_t ldwp = round_up(nprime, kTcN);
        k_wdigits<<<(unsigned)std::max<int64_t>(1, ceil_div(ldwp, 128)), 128, 0, st>>>(e.Wn, nbo, nprime, ldwp, e.Wd,
                                                                                        e.E, J0 + nbo, e.gsh);
        CSLS_CUDA(cudaGetLastError());
        // a trailing block exists only right of a full 64-column outer block: the update's
        // products always run over K = 64
        if (nbo != kOB) return CSLS_ERR_ARG;
        tk = kt_begin(kFamUpdate, st);
        const int64_t nrt = ceil_div(L, kTcM), nct = ceil_div(nprime, kTcN);
        const int cpt = tc_update_cpt(nrt, nct, sms);
        k_emu_update_tc<<<dim3((unsigned)ceil_div(nct, cpt), (unsigned)nrt), kTcThreads, sizeof(TcUpdSmem), st>>>(
            cmap, reinterpret_cast<long long*>(A), lda, s, J0, nbo, e.Vd, e.frow, e.Wd, e.gsh, nprime, cpt, spin, err);
        CSLS_CUDA(cudaGetLastError());
        kt_end(tk, prod_flop, st);
        nl += 4;
    }
    if (launches) *launches += nl;
    return CSLS_OK;
}

}  // namespace csls

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

#include "csls_internal.cuh"

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

__device__ __forceinline__ void cut_digits(long long N, int (&d)[kDig]) {
#pragma unroll
    for (int q = kDig - 1; q >= 1; --q) {
        const int r = (int)(((N + 128) & 255) - 128);
        d[q] = r;
        N = (N - r) >> 8;
    }
    d[0] = (int)N;
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

// ------------------------------------------------------------------ per-panel digit kernels

// Masked Householder vector entry: 0 above the diagonal, 1 on it, stored tail below.
__device__ __forceinline__ double vmask(const double* A, int64_t lda, int64_t r, int64_t j0, int a) {
    const int64_t d = j0 + a;
    return r < d ? 0.0 : (r == d ? 1.0 : A[r + d * lda]);
}

// Column maxima of V (for the V^T C digits), as ordered bit patterns (|x| >= 0).
__global__ void __launch_bounds__(256) k_vcolmax(const double* A, int64_t lda, int64_t s, int64_t j0, int nbw,
                                                 unsigned long long* colmax) {
    __shared__ unsigned long long red[kPanel];
    if (threadIdx.x < kPanel) red[threadIdx.x] = 0ULL;
    __syncthreads();
    const int a = threadIdx.x & 31;
    unsigned long long best = 0ULL;
    if (a < nbw) {
        for (int64_t r = j0 + blockIdx.x * 8 + (threadIdx.x >> 5); r < s; r += (int64_t)gridDim.x * 8) {
            const unsigned long long b = __double_as_longlong(fabs(vmask(A, lda, r, j0, a)));
            best = b > best ? b : best;
        }
        atomicMax(&red[a], best);
    }
    __syncthreads();
    if (threadIdx.x < nbw) atomicMax(&colmax[threadIdx.x], red[threadIdx.x]);
}

// Digits of V: per-row scale for C += V Wn (Vd[p][r][a], a contiguous) and per-column
// scale for V^T C (VTd[p][a][r], r contiguous). Rows are local row indices r - j0.
__global__ void __launch_bounds__(256) k_vdigits(const double* A, int64_t lda, int64_t s, int64_t j0, int nbw,
                                                 const unsigned long long* colmax, int64_t ldv,
                                                 unsigned short* Vd, unsigned short* VTd, int* frow, int* ecol) {
    const int64_t L = s - j0;
    if (blockIdx.x == 0 && threadIdx.x < kPanel)
        ecol[threadIdx.x] = threadIdx.x < nbw ? exp_of(__longlong_as_double((long long)colmax[threadIdx.x])) : 0;
    for (int64_t lr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lr < ldv; lr += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = j0 + lr;
        double v[kPanel];
        double mx = 0.0;
#pragma unroll
        for (int a = 0; a < kPanel; ++a) {
            v[a] = (lr < L && a < nbw) ? vmask(A, lda, r, j0, a) : 0.0;
            mx = fmax(mx, fabs(v[a]));
        }
        const int f = exp_of(mx);
        frow[lr] = f;
#pragma unroll
        for (int a = 0; a < kPanel; ++a) {
            int d[kDig];
            digits_f64(v[a], f, d);
            const int ea = a < nbw ? exp_of(__longlong_as_double((long long)colmax[a])) : 0;
            int dt[kDig];
            digits_f64(v[a], ea, dt);
#pragma unroll
            for (int p = 0; p < kDig; ++p) {
                Vd[((int64_t)p * ldv + lr) * kPanel + a] = bf16_of_int(d[p]);
                VTd[((int64_t)p * kPanel + a) * ldv + lr] = bf16_of_int(dt[p]);
            }
        }
    }
}

// Digits of Wn (kPanel x nprime, row-major): per-column scale; Wd[p][c][a].
__global__ void k_wdigits(const double* Wn, int64_t nprime, int64_t ldw, unsigned short* Wd, int* gcol) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ldw; c += (int64_t)gridDim.x * blockDim.x) {
        double w[kPanel];
        double mx = 0.0;
#pragma unroll
        for (int a = 0; a < kPanel; ++a) {
            w[a] = c < nprime ? Wn[(int64_t)a * nprime + c] : 0.0;
            mx = fmax(mx, fabs(w[a]));
        }
        const int g = exp_of(mx);
        gcol[c] = g;
#pragma unroll
        for (int a = 0; a < kPanel; ++a) {
            int d[kDig];
            digits_f64(w[a], g, d);
#pragma unroll
            for (int p = 0; p < kDig; ++p) Wd[((int64_t)p * ldw + c) * kPanel + a] = bf16_of_int(d[p]);
        }
    }
}

// ------------------------------------------------------------------ W = V^T C  (split over row chunks)

constexpr int kVtcCols = 64;
constexpr int kVtcPad = 8;                     // bf16 elements of padding per k-row
constexpr int kVtcLdk = kVtcStep + kVtcPad;    // 40

struct VtcSmem {
    unsigned short As[2][kDig][kPanel][kVtcLdk];   // V^T digits, two pipeline stages: [p][a][k]
    long long Craw[2][kVtcCols][kVtcStep];        // raw fixed-point C rows, two stages: [c][k]
    unsigned short Bs[kDig][kVtcCols][kVtcLdk];    // C digits of the current step: [q][c][k]
};

// Wp[chunk](a, c) for c in the column tile: sum over the chunk's rows of V(r, a) C(r, c).
// Two-stage cp.async pipeline: the V^T digits and raw C rows of step k + 1 are in flight
// while step k is cut into digits and multiplied.
__global__ void __launch_bounds__(kEmuThreads, 2)
k_emu_vtc(const long long* Cfix, int64_t lda, int64_t s, int64_t n, int64_t j0, int nbw, int64_t kc,
          const unsigned short* VTd, int64_t ldv, const int* ecol, const int* E, double* Wp, int64_t nprime) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VtcSmem& sm = *reinterpret_cast<VtcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int64_t jc = j0 + nbw;
    const int64_t c0 = (int64_t)blockIdx.x * kVtcCols;
    const int64_t L = s - j0;
    const int64_t lb = (int64_t)blockIdx.y * kc;               // local row range [lb, le)
    const int64_t le = lb + kc < L ? lb + kc : L;
    const int mi = warp & 1, nt = warp >> 1;                   // warp: a in mi*16.., cols nt*16..
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
        for (int idx = tid; idx < kDig * kPanel * 4; idx += kEmuThreads) {
            const int ch = idx & 3, a = (idx >> 2) % kPanel, p = (idx >> 2) / kPanel;
            const int64_t lr = k0 + ch * 8;
            const bool ok = lr < ldv;
            const unsigned short* src = VTd + ((int64_t)p * kPanel + a) * ldv + (ok ? lr : 0);
            cp_async16(&sm.As[stage][p][a][ch * 8], src, ok ? 16 : 0);
        }
        // raw C: per column 32 rows = 16 chunks of two int64
        for (int idx = tid; idx < kVtcCols * (kVtcStep / 2); idx += kEmuThreads) {
            const int ch = idx % (kVtcStep / 2), c = idx / (kVtcStep / 2);
            const int64_t lr = k0 + 2 * ch, gc = jc + c0 + c;
            const int rows = (gc < n) ? (int)(le - lr < 0 ? 0 : (le - lr > 2 ? 2 : le - lr)) : 0;
            const long long* src = Cfix + (rows > 0 ? (j0 + lr) + gc * lda : 0);
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
        // cut this step's C entries into digits (each thread: one column, 8 rows)
        {
            const int c = tid >> 2, kq = (tid & 3) * 8;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                int d[kDig];
                digits_fix(sm.Craw[stage][c][kq + e], d);
#pragma unroll
                for (int q = 0; q < kDig; ++q) sm.Bs[q][c][kq + e] = bf16_of_int(d[q]);
            }
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
    double* out = Wp + (int64_t)blockIdx.y * kPanel * nprime;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int a = mi * 16 + g + (h >> 1) * 8;
            const int64_t col = c0 + nt * 16 + j * 8 + 2 * t + (h & 1);
            if (col < nprime && a < nbw) {
                const int sc = ecol[a] + E[jc + col] - 14;
                const double v = ldexp((double)hi[j][h], -16) + ldexp((double)lo[j][h], -40);
                out[(int64_t)a * nprime + col] = ldexp(v, sc);
            }
        }
}

// ------------------------------------------------------------------ C += V Wn  (exact integer update)

constexpr int kUpdRows = 64, kUpdCols = 64, kUpdPad = 8, kUpdLdk = kPanel + kUpdPad;   // 40

struct UpdSmem {
    unsigned short Vs[kDig][kUpdRows][kUpdLdk];   // [p][r][a]
    unsigned short Ws[kDig][kUpdCols][kUpdLdk];   // [q][c][a]
    int frow[kUpdRows];
    int gcol[kUpdCols];
    int ecol[kUpdCols];
};

__global__ void __launch_bounds__(kEmuThreads, 3)
k_emu_update(long long* Cfix, int64_t lda, int64_t s, int64_t n, int64_t j0, int nbw, const unsigned short* Vd,
             int64_t ldv, const int* frow, const unsigned short* Wd, int64_t ldw, const int* gcol, const int* E,
             int64_t nprime) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    UpdSmem& sm = *reinterpret_cast<UpdSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int64_t jc = j0 + nbw;
    const int64_t L = s - j0;
    const int64_t rb = (int64_t)blockIdx.x * kUpdRows;   // local row of tile row 0
    const int64_t cb = (int64_t)blockIdx.y * kUpdCols;   // trailing column of tile col 0
    const int wm = warp & 1, wn = warp >> 1;             // warp tile: rows wm*32..+32, cols wn*16..+16
    // issue the loads of this warp's C entries first; they are only needed after the products
    long long cval[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int64_t lr = rb + wm * 32 + i * 16 + g + (h >> 1) * 8;
                const int64_t col = cb + wn * 16 + j * 8 + 2 * t + (h & 1);
                cval[i][j][h] = (lr < L && col < nprime) ? Cfix[(j0 + lr) + (jc + col) * lda] : 0LL;
            }
    // digit tiles: each row of 32 bf16 is 4 chunks of 16 B
    for (int idx = tid; idx < kDig * kUpdRows * 4; idx += kEmuThreads) {
        const int ch = idx & 3, r = (idx >> 2) % kUpdRows, p = (idx >> 2) / kUpdRows;
        const int64_t lr = rb + r;
        const bool ok = lr < L;
        cp_async16(&sm.Vs[p][r][ch * 8], Vd + ((int64_t)p * ldv + (ok ? lr : 0)) * kPanel + ch * 8, ok ? 16 : 0);
    }
    for (int idx = tid; idx < kDig * kUpdCols * 4; idx += kEmuThreads) {
        const int ch = idx & 3, c = (idx >> 2) % kUpdCols, q = (idx >> 2) / kUpdCols;
        const int64_t col = cb + c;
        const bool ok = col < nprime;
        cp_async16(&sm.Ws[q][c][ch * 8], Wd + ((int64_t)q * ldw + (ok ? col : 0)) * kPanel + ch * 8, ok ? 16 : 0);
    }
    cp_async_commit();
    for (int i = tid; i < kUpdRows; i += kEmuThreads) sm.frow[i] = rb + i < L ? frow[rb + i] : 0;
    for (int i = tid; i < kUpdCols; i += kEmuThreads) {
        sm.gcol[i] = cb + i < nprime ? gcol[cb + i] : 0;
        sm.ecol[i] = cb + i < nprime ? E[jc + cb + i] : 0;
    }
    cp_async_wait<0>();
    __syncthreads();
    long long acc64[2][2][4];
#pragma unroll 1
    for (int l = 0; l <= kLev; ++l) {
        float acc[2][2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) acc[i][j][h] = kMagic;
        for (int p = 0; p <= l; ++p) {
            const int q = l - p;
#pragma unroll
            for (int ks = 0; ks < kPanel; ks += 16) {
                uint32_t af[2][4], bq[4];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    ldsm_x4(af[i], &sm.Vs[p][wm * 32 + i * 16 + (lane & 15)][ks + (lane >> 4) * 8]);
                ldsm_x4(bq, &sm.Ws[q][wn * 16 + (lane & 7) + ((lane >> 4) & 1) * 8][ks + ((lane >> 3) & 1) * 8]);
                const uint32_t bfr[2][2] = {{bq[0], bq[1]}, {bq[2], bq[3]}};
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) hmma(acc[i][j], af[i], bfr[j]);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const long long v = (long long)magic_to_int(acc[i][j][h]);
                    acc64[i][j][h] = l == 0 ? v : (acc64[i][j][h] << 8) + v;
                }
    }
    // Cfix += acc64 * 2^(f_r + g_c - 14 - 8 kLev + 62 - E_c), rounded to the fixed-point grid
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = wm * 32 + i * 16 + g + (h >> 1) * 8;
                const int c = wn * 16 + j * 8 + 2 * t + (h & 1);
                const int64_t lr = rb + r, col = cb + c;
                if (lr < L && col < nprime) {
                    const int sh = sm.frow[r] + sm.gcol[c] - 14 - 8 * kLev + kFixBits - sm.ecol[c];
                    const long long v = acc64[i][j][h];
                    long long dlt;
                    if (v == 0) dlt = 0;
                    else if (sh >= 0) dlt = sh < 63 ? v << sh : 0;
                    else dlt = -sh < 63 ? (v + (1LL << (-sh - 1))) >> (-sh) : 0;
                    Cfix[(j0 + lr) + (jc + col) * lda] = cval[i][j][h] + dlt;
                }
            }
}

// ------------------------------------------------------------------ scratch and driver

struct EmuScratch {
    int* E;                       // n column exponents
    unsigned long long* colmax;   // kPanel
    int* ecol;                    // kPanel
    int* frow;                    // s
    int* gcol;                    // n
    unsigned short* Vd;           // kDig * s * kPanel
    unsigned short* VTd;          // kDig * kPanel * s
    unsigned short* Wd;           // kDig * n * kPanel
};

size_t qr_emu_scratch_bytes(int64_t s, int64_t n) {
    Carve c{nullptr, 0, 0, true};
    const int64_t ldv = round_up(s, 8), ldw = round_up(n, 8);
    c.take<int>((size_t)n);
    c.take<unsigned long long>(kPanel);
    c.take<int>(kPanel);
    c.take<int>((size_t)ldv);
    c.take<int>((size_t)ldw);
    c.take<unsigned short>((size_t)(kDig * ldv * kPanel));
    c.take<unsigned short>((size_t)(kDig * ldv * kPanel));
    c.take<unsigned short>((size_t)(kDig * ldw * kPanel));
    return c.off;
}

static EmuScratch emu_carve(Carve& c, int64_t s, int64_t n) {
    const int64_t ldv = round_up(s, 8), ldw = round_up(n, 8);
    EmuScratch e;
    e.E = c.take<int>((size_t)n);
    e.colmax = c.take<unsigned long long>(kPanel);
    e.ecol = c.take<int>(kPanel);
    e.frow = c.take<int>((size_t)ldv);
    e.gcol = c.take<int>((size_t)ldw);
    e.Vd = c.take<unsigned short>((size_t)(kDig * ldv * kPanel));
    e.VTd = c.take<unsigned short>((size_t)(kDig * ldv * kPanel));
    e.Wd = c.take<unsigned short>((size_t)(kDig * ldw * kPanel));
    return e;
}

int qr_panel_launch_f64(double* A, int64_t lda, int64_t s, int64_t j0, int nbw, const QrScratch& q, int* err,
                        long long spin, cudaStream_t st);
int qr_wreduce_launch_f64(const QrScratch& q, int ks, int nbw, int64_t nprime, cudaStream_t st);

int qr_factor_f64_emu(double* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, void* emu_work,
                      size_t emu_bytes, int* err, long long spin, cudaStream_t st, int64_t* launches) {
    if (s < n || n <= 0) return CSLS_ERR_ARG;
    if (emu_bytes < qr_emu_scratch_bytes(s, n)) return CSLS_ERR_WORKSPACE;
    Carve c{(char*)emu_work, 0, emu_bytes, false};
    EmuScratch e = emu_carve(c, s, n);
    const int64_t ldv = round_up(s, 8), ldw = round_up(n, 8);
    static bool attr = false;
    if (!attr) {
        CSLS_CUDA(cudaFuncSetAttribute(k_emu_vtc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(VtcSmem)));
        CSLS_CUDA(cudaFuncSetAttribute(k_emu_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(UpdSmem)));
        attr = true;
    }
    const int sms = device_sm_count();
    CSLS_CUDA(cudaMemsetAsync(q.bar, 0, sizeof(GridBarrier), st));
    k_col_exponent<<<(unsigned)std::min<int64_t>(n, 65535), 256, 0, st>>>(A, lda, s, n, e.E);
    CSLS_CUDA(cudaGetLastError());
    dim3 fg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(s, 1024), 64)), (unsigned)std::min<int64_t>(n, 65535));
    k_to_fixed<<<fg, 256, 0, st>>>(A, lda, s, n, e.E);
    CSLS_CUDA(cudaGetLastError());
    int64_t nl = 2;
    for (int64_t j0 = 0; j0 < n; j0 += kPanel) {
        const int nbw = (int)(n - j0 < kPanel ? n - j0 : kPanel);
        const int64_t L = s - j0;
        dim3 pg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 256), 256)), (unsigned)nbw);
        k_panel_to_f64<<<pg, 256, 0, st>>>(A, lda, s, j0, nbw, e.E);
        CSLS_CUDA(cudaGetLastError());
        if (j0 > 0) {
            dim3 tg((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(j0, 256), 64)), (unsigned)nbw);
            k_panel_top_to_f64<<<tg, 256, 0, st>>>(A, lda, j0, nbw, e.E);
            CSLS_CUDA(cudaGetLastError());
        }
        {
            const int tk = kt_begin(kFamPanel, st);
            CSLS_TRY(qr_panel_launch_f64(A, lda, s, j0, nbw, q, err, spin, st));
            kt_end(tk, 0.0, st);
        }
        nl += 3;
        const int64_t nprime = n - j0 - nbw;
        if (nprime <= 0) continue;
        // digits of V
        CSLS_CUDA(cudaMemsetAsync(e.colmax, 0, sizeof(unsigned long long) * kPanel, st));
        k_vcolmax<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 8), (int64_t)sms * 4)), 256, 0, st>>>(
            A, lda, s, j0, nbw, e.colmax);
        CSLS_CUDA(cudaGetLastError());
        const int64_t ldvp = round_up(L, 8);   // digit planes use the current panel height
        k_vdigits<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ldvp, 256), (int64_t)sms * 8)), 256, 0, st>>>(
            A, lda, s, j0, nbw, e.colmax, ldvp, e.Vd, e.VTd, e.frow, e.ecol);
        CSLS_CUDA(cudaGetLastError());
        // W = V^T C over row chunks
        const int64_t ntn = ceil_div(nprime, kVtcCols);
        int64_t ks = ceil_div(8LL * sms, ntn);
        const int64_t maxks = ceil_div(L, kVtcStep);
        if (ks > maxks) ks = maxks;
        if (ks < 1) ks = 1;
        while (ks > 1 && ks * kPanel * ntn * kVtcCols > q.wp_elems) --ks;
        const int64_t kc = round_up(ceil_div(L, ks), kVtcStep);
        ks = ceil_div(L, kc);
        const double prod_flop = 2.0 * (double)L * (double)nprime * (double)nbw;
        int tk = kt_begin(kFamVtc, st);
        k_emu_vtc<<<dim3((unsigned)ntn, (unsigned)ks), kEmuThreads, sizeof(VtcSmem), st>>>(
            reinterpret_cast<const long long*>(A), lda, s, n, j0, nbw, kc, e.VTd, ldvp, e.ecol, e.E, q.Wp, nprime);
        CSLS_CUDA(cudaGetLastError());
        kt_end(tk, prod_flop, st);
        CSLS_TRY(qr_wreduce_launch_f64(q, (int)ks, nbw, nprime, st));
        // digits of Wn, then the exact update
        const int64_t ldwp = round_up(nprime, 8);
        k_wdigits<<<(unsigned)std::max<int64_t>(1, ceil_div(ldwp, 256)), 256, 0, st>>>(q.Wn, nprime, ldwp, e.Wd, e.gcol);
        CSLS_CUDA(cudaGetLastError());
        tk = kt_begin(kFamUpdate, st);
        k_emu_update<<<dim3((unsigned)ceil_div(L, kUpdRows), (unsigned)ceil_div(nprime, kUpdCols)), kEmuThreads,
                       sizeof(UpdSmem), st>>>(reinterpret_cast<long long*>(A), lda, s, n, j0, nbw, e.Vd, ldvp,
                                              e.frow, e.Wd, ldwp, e.gcol, e.E, nprime);
        CSLS_CUDA(cudaGetLastError());
        kt_end(tk, prod_flop, st);
        nl += 6;
    }
    if (launches) *launches += nl;
    return CSLS_OK;
}

}  // namespace csls

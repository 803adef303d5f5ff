// Blocked Householder QR of the dense s x n sketch (Algorithm 1 step 3).
//
// Right-looking, panel width kPanel (32), compact WY representation
// H_1 ... H_b = I - V T V^T:
//   1. panel factorisation (cooperative kernel, all SMs): the panel's rows are
//      split across CTAs and kept in shared memory; each column needs two
//      grid-wide reductions (the norm, then v^T A for the remaining panel
//      columns), done with fixed-order partial sums so results are
//      deterministic; the same kernel forms T from V^T V;
//   2. W = V^T C, split over row chunks                  (FP64: DMMA m16n8k16)
//   3. Wn = -(T^T sum_chunks W)                           (small)
//   4. C += V Wn, the rank-32 update of the trailing matrix (FP64: DMMA m16n8k16)
// Steps 2 and 4 carry all but O(s n kPanel) of the 2 s n^2 - 2/3 n^3 flops. On
// GB300 the legacy FP64 MMA (mma.sync .f64, m16n8k16) runs about twice as fast
// as FP64 FMA, so it is the FP64 tensor path here; tcgen05 has no f64 kind.
// The binary32 variant uses the same structure with FP32 FMA tiles.
#include "csls_internal.cuh"

namespace csls {

constexpr int kPanelThreads = 256;
// per-CTA slots in the panel partials array
constexpr int kPartStride = 2 + kPanel + kPanel * kPanel;

template <class T>
__device__ __forceinline__ T vval(const T* W, int64_t ld, int a, int r, int64_t grow, int64_t j0) {
    // Householder vector a at local row r (global row grow): 0 above, 1 on, stored tail below the diagonal.
    const int64_t d = j0 + a;
    return grow < d ? T(0) : (grow == d ? T(1) : W[a * ld + r]);
}

template <class T, bool SMEM>
__global__ void __launch_bounds__(kPanelThreads)
k_panel(T* A, int64_t lda, int64_t s, int64_t j0, int nbw, int64_t chunk, T* tau, T* Tmat, T* part,
        GridBarrier* bar, long long spin, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[kPanelThreads / 32];
    __shared__ T coef[4];             // tau, scal, beta, sigma-flag
    __shared__ T wk[kPanel];
    __shared__ T gram[kPanel * kPanel];
    __shared__ T tl[kPanel * kPanel];

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int64_t r0 = j0 + (int64_t)g * chunk;
    const int64_t r1 = r0 + chunk < s ? r0 + chunk : s;
    const int nloc = r1 > r0 ? (int)(r1 - r0) : 0;
    T* W;
    int64_t ld;
    if (SMEM) {
        W = reinterpret_cast<T*>(smem_raw);
        ld = chunk;
        for (int c = 0; c < nbw; ++c)
            for (int r = tid; r < nloc; r += kPanelThreads) W[c * ld + r] = A[(r0 + r) + (j0 + c) * lda];
        __syncthreads();
    } else {
        W = A + r0 + j0 * lda;
        ld = lda;
    }
    T* part_norm = part;                 // G
    T* part_alpha = part + G;            // 1
    T* part_w = part + G + 1;            // G * kPanel
    T* part_gram = part + G + 1 + (int64_t)G * kPanel;   // G * kPanel^2

    for (int c = 0; c < nbw; ++c) {
        const int64_t j = j0 + c;
        // (a) partial ||A(j+1:s, j)||^2 and the diagonal entry alpha
        T acc = T(0);
        for (int r = tid; r < nloc; r += kPanelThreads) {
            if (r0 + r > j) {
                T x = W[c * ld + r];
                acc += x * x;
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            T t = T(0);
            for (int w = 0; w < kPanelThreads / 32; ++w) t += red[w];
            part_norm[g] = t;
            if (j >= r0 && j < r1) part_alpha[0] = W[c * ld + (j - r0)];
        }
        if (!grid_sync(bar, G, spin, err)) return;
        // (b) reflector: every CTA reduces the partials in the same fixed tree order (all threads
        // load, so the G partials cost one round trip instead of G dependent ones)
        T sq = T(0);
        for (int q = tid; q < G; q += kPanelThreads) sq += __ldcg(part_norm + q);
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if ((tid & 31) == 0) red[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            T sigma = T(0);
            for (int w = 0; w < kPanelThreads / 32; ++w) sigma += red[w];
            T alpha = __ldcg(part_alpha);
            if (sigma == T(0)) {
                coef[0] = T(0); coef[1] = T(1); coef[2] = alpha; coef[3] = T(0);
            } else {
                T nrm = sqrt(alpha * alpha + sigma);
                T beta = alpha >= T(0) ? -nrm : nrm;
                coef[0] = (beta - alpha) / beta;
                coef[1] = T(1) / (alpha - beta);
                coef[2] = beta;
                coef[3] = T(1);
            }
            if (g == 0) tau[j] = coef[0];
        }
        __syncthreads();
        const T tau_c = coef[0];
        if (coef[3] != T(0)) {
            const T scal = coef[1];
            for (int r = tid; r < nloc; r += kPanelThreads) {
                const int64_t grow = r0 + r;
                if (grow > j) W[c * ld + r] *= scal;
                else if (grow == j) W[c * ld + r] = coef[2];
            }
        }
        __syncthreads();
        if (c == nbw - 1) break;
        // (c) partial w_k = v^T A(j:s, k) for the remaining panel columns
        const int warp = tid >> 5, lane = tid & 31;
        for (int k = c + 1 + warp; k < nbw; k += kPanelThreads / 32) {
            T a2 = T(0);
            for (int r = lane; r < nloc; r += 32) {
                const int64_t grow = r0 + r;
                if (grow >= j) {
                    T v = grow == j ? T(1) : W[c * ld + r];
                    a2 += v * W[k * ld + r];
                }
            }
            for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            if (lane == 0) part_w[(int64_t)g * kPanel + k] = a2;
        }
        if (!grid_sync(bar, G, spin, err)) return;
        // (d) w_k = tau sum_g partials (8 threads per column, fixed order); A(j:s, k) -= w_k v
        {
            const int k = tid >> 3, sub = tid & 7;
            T t = T(0);
            if (k < nbw && k > c)
                for (int q = sub; q < G; q += 8) t += __ldcg(part_w + (int64_t)q * kPanel + k);
            t += __shfl_xor_sync(0xffffffffu, t, 4);
            t += __shfl_xor_sync(0xffffffffu, t, 2);
            t += __shfl_xor_sync(0xffffffffu, t, 1);
            if (sub == 0 && k < nbw && k > c) wk[k] = tau_c * t;
        }
        __syncthreads();
        const int ncols = nbw - c - 1;
        for (int idx = tid; idx < nloc * ncols; idx += kPanelThreads) {
            const int r = idx % nloc, k = c + 1 + idx / nloc;
            const int64_t grow = r0 + r;
            if (grow >= j) {
                T v = grow == j ? T(1) : W[c * ld + r];
                W[k * ld + r] -= wk[k] * v;
            }
        }
        __syncthreads();
    }
    // Gram matrix V^T V (upper triangle) for T
    for (int p = tid; p < nbw * nbw; p += kPanelThreads) {
        const int a = p % nbw, b = p / nbw;
        T acc = T(0);
        if (a <= b) {
            for (int r = 0; r < nloc; ++r) {
                const int64_t grow = r0 + r;
                acc += vval(W, ld, a, r, grow, j0) * vval(W, ld, b, r, grow, j0);
            }
        }
        part_gram[(int64_t)g * kPanel * kPanel + a + b * kPanel] = acc;
    }
    if (SMEM) {
        for (int c = 0; c < nbw; ++c)
            for (int r = tid; r < nloc; r += kPanelThreads) A[(r0 + r) + (j0 + c) * lda] = W[c * ld + r];
    }
    if (!grid_sync(bar, G, spin, err)) return;
    // reduce the Gram partials across the grid: each warp of each CTA owns entries of V^T V and
    // sums their G partials with its 32 lanes in a fixed order; one more barrier, then CTA 0 forms T
    T* gram_red = part_gram + (int64_t)G * kPanel * kPanel;   // kPanel^2
    {
        const int warp = tid >> 5, lane = tid & 31;
        for (int e = g + warp * G; e < kPanel * kPanel; e += G * (kPanelThreads / 32)) {
            const int a = e % kPanel, b = e / kPanel;
            T t = T(0);
            if (a < nbw && b < nbw && a <= b)
                for (int q = lane; q < G; q += 32) t += __ldcg(part_gram + (int64_t)q * kPanel * kPanel + e);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) gram_red[e] = t;
        }
    }
    if (!grid_sync(bar, G, spin, err)) return;
    if (g != 0) return;
    for (int p = tid; p < kPanel * kPanel; p += kPanelThreads) {
        gram[p] = __ldcg(gram_red + p);
        tl[p] = T(0);
    }
    __syncthreads();
    // T(i,i) = tau_i ; T(0:i, i) = -tau_i T(0:i, 0:i) (V(:,0:i)^T v_i)
    for (int i = 0; i < nbw; ++i) {
        const T ti = tau[j0 + i];
        if (tid < i) {
            T acc = T(0);
            for (int b = tid; b < i; ++b) acc += tl[tid + b * kPanel] * gram[b + i * kPanel];
            tl[tid + i * kPanel] = -ti * acc;
        }
        if (tid == i) tl[i + i * kPanel] = ti;
        __syncthreads();
    }
    for (int p = tid; p < kPanel * kPanel; p += kPanelThreads) Tmat[p] = tl[p];
}

// ------------------------------------------------------------------ DMMA (FP64 tensor) helpers

__device__ __forceinline__ void dmma16816(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
        "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
          "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

constexpr int kUpdM = 64, kUpdN = 64, kPadV = 4, kPadW = 4;
constexpr int kUpdM32 = 128;

// C(j0:s, jc:n) += V Wn ; V is the masked panel (s - j0) x nbw, Wn is kPanel x nprime (row-major, ld nprime).
__global__ void __launch_bounds__(256) k_update_f64(double* A, int64_t lda, int64_t s, int64_t n, int64_t j0,
                                                    int nbw, const double* Wn, int64_t nprime) {
    __shared__ double Vs[kPanel][kUpdM + kPadV];
    __shared__ double Ws[kPanel][kUpdN + kPadW];
    const int tid = threadIdx.x;
    const int64_t jc = j0 + nbw;
    const int64_t rbase = j0 + (int64_t)blockIdx.x * kUpdM;   // global row of tile row 0
    const int64_t cbase = (int64_t)blockIdx.y * kUpdN;        // trailing column of tile col 0
    for (int idx = tid; idx < kPanel * kUpdM; idx += 256) {
        const int r = idx % kUpdM, k = idx / kUpdM;
        const int64_t grow = rbase + r;
        double v = 0.0;
        if (k < nbw && grow < s) {
            const int64_t d = j0 + k;
            v = grow < d ? 0.0 : (grow == d ? 1.0 : A[grow + d * lda]);
        }
        Vs[k][r] = v;
    }
    for (int idx = tid; idx < kPanel * kUpdN; idx += 256) {
        const int c = idx % kUpdN, k = idx / kUpdN;
        const int64_t col = cbase + c;
        Ws[k][c] = (k < nbw && col < nprime) ? Wn[(int64_t)k * nprime + col] : 0.0;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const int wm = warp & 1, wn = warp >> 1;    // warp tile: rows wm*32..+32, cols wn*16..+16
    double acc[2][2][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) {
            const int rr = wm * 32 + mi * 16 + gq;
            const int cc = wn * 16 + ni * 8 + 2 * tq;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int64_t grow = rbase + rr + (h >> 1) * 8;
                const int64_t gcol = jc + cbase + cc + (h & 1);
                acc[mi][ni][h] = (grow < s && gcol < n) ? A[grow + gcol * lda] : 0.0;
            }
        }
#pragma unroll
    for (int kk = 0; kk < kPanel; kk += 16) {
        double af[2][8], bf[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int i = 0; i < 8; ++i) af[mi][i] = Vs[kk + tq + 4 * (i >> 1)][wm * 32 + mi * 16 + gq + 8 * (i & 1)];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
            for (int i = 0; i < 4; ++i) bf[ni][i] = Ws[kk + tq + 4 * i][wn * 16 + ni * 8 + gq];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 2; ++ni) dmma16816(acc[mi][ni], af[mi], bf[ni]);
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) {
            const int rr = wm * 32 + mi * 16 + gq;
            const int cc = wn * 16 + ni * 8 + 2 * tq;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int64_t grow = rbase + rr + (h >> 1) * 8;
                const int64_t gcol = jc + cbase + cc + (h & 1);
                if (grow < s && gcol < n) A[grow + gcol * lda] = acc[mi][ni][h];
            }
        }
}

constexpr int kVtcRows = 32, kVtcN = 64;

// Wp[ks](a, c) = sum over rows of chunk ks of V(r, a) C(r, c), a < kPanel, c < nprime.
__global__ void __launch_bounds__(256) k_vtc_f64(const double* A, int64_t lda, int64_t s, int64_t n, int64_t j0,
                                                 int nbw, int64_t kc, double* Wp, int64_t nprime) {
    __shared__ double Vs[kVtcRows][kPanel + kPadV];
    __shared__ double Cs[kVtcRows][kVtcN + kPadW];
    const int tid = threadIdx.x;
    const int64_t jc = j0 + nbw;
    const int64_t cbase = (int64_t)blockIdx.x * kVtcN;
    const int64_t rb = j0 + (int64_t)blockIdx.y * kc;
    const int64_t re = rb + kc < s ? rb + kc : s;
    const int warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const int mi = warp & 1, nb2 = (warp >> 1) * 16;   // warp: a rows mi*16..+16, cols nb2..nb2+16
    double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    for (int64_t r0 = rb; r0 < re; r0 += kVtcRows) {
        for (int idx = tid; idx < kVtcRows * kPanel; idx += 256) {
            const int r = idx % kVtcRows, a = idx / kVtcRows;
            const int64_t grow = r0 + r;
            double v = 0.0;
            if (a < nbw && grow < re) {
                const int64_t d = j0 + a;
                v = grow < d ? 0.0 : (grow == d ? 1.0 : A[grow + d * lda]);
            }
            Vs[r][a] = v;
        }
        for (int idx = tid; idx < kVtcRows * kVtcN; idx += 256) {
            const int r = idx % kVtcRows, c = idx / kVtcRows;
            const int64_t grow = r0 + r, gcol = jc + cbase + c;
            Cs[r][c] = (grow < re && gcol < n) ? A[grow + gcol * lda] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kVtcRows; kk += 16) {
            double af[8], bf[2][4];
#pragma unroll
            for (int i = 0; i < 8; ++i) af[i] = Vs[kk + tq + 4 * (i >> 1)][mi * 16 + gq + 8 * (i & 1)];
#pragma unroll
            for (int ni = 0; ni < 2; ++ni)
#pragma unroll
                for (int i = 0; i < 4; ++i) bf[ni][i] = Cs[kk + tq + 4 * i][nb2 + ni * 8 + gq];
            dmma16816(acc[0], af, bf[0]);
            dmma16816(acc[1], af, bf[1]);
        }
        __syncthreads();
    }
    double* out = Wp + (int64_t)blockIdx.y * kPanel * nprime;
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int a = mi * 16 + gq + (h >> 1) * 8;
            const int64_t col = cbase + nb2 + ni * 8 + 2 * tq + (h & 1);
            if (col < nprime) out[(int64_t)a * nprime + col] = acc[ni][h];
        }
}

// ------------------------------------------------------------------ FP32 SIMT tiles (binary32 variant)

__global__ void __launch_bounds__(256) k_update_f32(float* A, int64_t lda, int64_t s, int64_t n, int64_t j0, int nbw,
                                                    const float* Wn, int64_t nprime) {
    __shared__ float Vs[kPanel][kUpdM32 + 4];
    __shared__ float Ws[kPanel][kUpdN + 4];
    const int tid = threadIdx.x;
    const int64_t jc = j0 + nbw;
    const int64_t rbase = j0 + (int64_t)blockIdx.x * kUpdM32;
    const int64_t cbase = (int64_t)blockIdx.y * kUpdN;
    for (int idx = tid; idx < kPanel * kUpdM32; idx += 256) {
        const int r = idx % kUpdM32, k = idx / kUpdM32;
        const int64_t grow = rbase + r;
        float v = 0.0f;
        if (k < nbw && grow < s) {
            const int64_t d = j0 + k;
            v = grow < d ? 0.0f : (grow == d ? 1.0f : A[grow + d * lda]);
        }
        Vs[k][r] = v;
    }
    for (int idx = tid; idx < kPanel * kUpdN; idx += 256) {
        const int c = idx % kUpdN, k = idx / kUpdN;
        const int64_t col = cbase + c;
        Ws[k][c] = (k < nbw && col < nprime) ? Wn[(int64_t)k * nprime + col] : 0.0f;
    }
    __syncthreads();
    const int tr = tid & 15, tc = tid >> 4;   // rows tr + 16 i (i < 8), cols tc * 4 + j (j < 4)
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int64_t grow = rbase + tr + 16 * i, gcol = jc + cbase + tc * 4 + jj;
            acc[i][jj] = (grow < s && gcol < n) ? A[grow + gcol * lda] : 0.0f;
        }
#pragma unroll 4
    for (int k = 0; k < kPanel; ++k) {
        float a[8], b[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = Vs[k][tr + 16 * i];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) b[jj] = Ws[k][tc * 4 + jj];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(a[i], b[jj], acc[i][jj]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int64_t grow = rbase + tr + 16 * i, gcol = jc + cbase + tc * 4 + jj;
            if (grow < s && gcol < n) A[grow + gcol * lda] = acc[i][jj];
        }
}

__global__ void __launch_bounds__(256) k_vtc_f32(const float* A, int64_t lda, int64_t s, int64_t n, int64_t j0,
                                                 int nbw, int64_t kc, float* Wp, int64_t nprime) {
    __shared__ float Vs[kVtcRows][kPanel + 1];
    __shared__ float Cs[kVtcRows][kVtcN + 1];
    const int tid = threadIdx.x;
    const int64_t jc = j0 + nbw;
    const int64_t cbase = (int64_t)blockIdx.x * kVtcN;
    const int64_t rb = j0 + (int64_t)blockIdx.y * kc;
    const int64_t re = rb + kc < s ? rb + kc : s;
    const int a = tid & 31, cq = (tid >> 5) * 8;   // output (a, cq..cq+8)
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t r0 = rb; r0 < re; r0 += kVtcRows) {
        for (int idx = tid; idx < kVtcRows * kPanel; idx += 256) {
            const int r = idx % kVtcRows, aa = idx / kVtcRows;
            const int64_t grow = r0 + r;
            float v = 0.0f;
            if (aa < nbw && grow < re) {
                const int64_t d = j0 + aa;
                v = grow < d ? 0.0f : (grow == d ? 1.0f : A[grow + d * lda]);
            }
            Vs[r][aa] = v;
        }
        for (int idx = tid; idx < kVtcRows * kVtcN; idx += 256) {
            const int r = idx % kVtcRows, c = idx / kVtcRows;
            const int64_t grow = r0 + r, gcol = jc + cbase + c;
            Cs[r][c] = (grow < re && gcol < n) ? A[grow + gcol * lda] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kVtcRows; ++r) {
            const float v = Vs[r][a];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[jj] = fmaf(v, Cs[r][cq + jj], acc[jj]);
        }
        __syncthreads();
    }
    float* out = Wp + (int64_t)blockIdx.y * kPanel * nprime;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const int64_t col = cbase + cq + jj;
        if (col < nprime) out[(int64_t)a * nprime + col] = acc[jj];
    }
}

// Wp[0](b, c) = sum_ks Wp[ks](b, c) for every entry (b < nbw), a warp per entry, fixed order.
template <class T>
__global__ void __launch_bounds__(256) k_psum(T* Wp, int KS, int nbw, int64_t nprime) {
    const int lane = threadIdx.x & 31;
    const int64_t entries = (int64_t)nbw * nprime;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < entries; e += nw) {
        const int64_t bb = e / nprime, c = e % nprime;
        T t = T(0);
        for (int q = lane; q < KS; q += 32) t += Wp[((int64_t)q * kPanel + bb) * nprime + c];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) Wp[bb * nprime + c] = t;
    }
}

// Wn(a, c) = -sum_{b <= a} T(b, a) sum_ks Wp[ks](b, c). A CTA owns 32 columns: one thread per
// (b, c) entry sums its partials (coalesced along c), then one per (a, c) forms -T^T W.
constexpr int kWrCols = 32;

template <class T>
__global__ void __launch_bounds__(256) k_wreduce(const T* Wp, int KS, const T* Tmat, int nbw, T* Wn, int64_t nprime) {
    __shared__ T Ts[kPanel * kPanel];
    __shared__ T Ws[kPanel * kWrCols];
    const int64_t c0 = (int64_t)blockIdx.x * kWrCols;
    for (int p = threadIdx.x; p < kPanel * kPanel; p += blockDim.x) Ts[p] = Tmat[p];
    for (int i = threadIdx.x; i < kPanel * kWrCols; i += blockDim.x) {
        const int bb = i / kWrCols, cl = i % kWrCols;
        const int64_t c = c0 + cl;
        T t = T(0);
        if (bb < nbw && c < nprime)
            for (int q = 0; q < KS; ++q) t += Wp[((int64_t)q * kPanel + bb) * nprime + c];
        Ws[i] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPanel * kWrCols; i += blockDim.x) {
        const int a = i / kWrCols, cl = i % kWrCols;
        const int64_t c = c0 + cl;
        if (c >= nprime) continue;
        T t = T(0);
        for (int bb = 0; bb <= a; ++bb) t += Ts[bb + a * kPanel] * Ws[bb * kWrCols + cl];
        Wn[(int64_t)a * nprime + c] = a < nbw ? -t : T(0);
    }
}

// ------------------------------------------------------------------ R extraction and diagonal blocks

template <class T>
__global__ void k_extract_r(const T* A, int64_t lda, int64_t n, T* R) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            T v = T(0);
            if (i <= j) {
                v = A[i + j * lda];
                if (A[i + i * lda] < T(0)) v = -v;
            }
            R[i + j * n] = v;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(1024) k_rdiag_stats(const T* R, int64_t n, double* stats) {
    __shared__ double mn[1024], mx[1024], bad[1024];
    double a = __longlong_as_double(0x7ff0000000000000LL), b = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double d = fabs((double)R[i + i * n]);
        if (!(d > 0.0) || !isfinite(d)) c += 1.0;
        if (isfinite(d)) { a = d < a ? d : a; b = d > b ? d : b; }
    }
    mn[threadIdx.x] = a; mx[threadIdx.x] = b; bad[threadIdx.x] = c;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + o]);
            mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + o]);
            bad[threadIdx.x] += bad[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { stats[0] = mn[0]; stats[1] = mx[0]; stats[2] = bad[0]; }
}

// Inverse of each 64 x 64 diagonal block of upper-triangular R (identity-padded past n).
// Thread t forms column t of the inverse by back substitution on R_bb x = e_t.
template <class T>
__global__ void __launch_bounds__(kTrsvBlock) k_diag_inverse(const T* R, int64_t n, double* Dinv) {
    __shared__ double Rb[kTrsvBlock][kTrsvBlock + 1];
    const int64_t b0 = (int64_t)blockIdx.x * kTrsvBlock;
    const int bs = (int)(n - b0 < kTrsvBlock ? n - b0 : kTrsvBlock);
    const int t = threadIdx.x;
    for (int i = 0; i < kTrsvBlock; ++i) {
        double v = 0.0;
        if (i < bs && t < bs) v = (double)R[(b0 + i) + (b0 + t) * n];
        else if (i == t) v = 1.0;
        Rb[i][t] = v;
    }
    __syncthreads();
    double x[kTrsvBlock];
    for (int i = kTrsvBlock - 1; i >= 0; --i) {
        double acc = 0.0;
        if (i <= t) {
            acc = (i == t) ? 1.0 : 0.0;
            for (int k = i + 1; k <= t; ++k) acc -= Rb[i][k] * x[k];
            acc /= Rb[i][i];
        }
        x[i] = acc;
    }
    double* out = Dinv + (int64_t)blockIdx.x * kTrsvBlock * kTrsvBlock;
    for (int i = 0; i < kTrsvBlock; ++i) out[i + t * kTrsvBlock] = x[i];
}

// ------------------------------------------------------------------ host side

static int panel_grid(int64_t L) {
    int64_t g = ceil_div(L, 128);
    int sms = device_sm_count();
    if (g > sms) g = sms;
    return (int)(g < 1 ? 1 : g);
}

static int64_t wp_capacity(int64_t n) {
    int64_t a = (int64_t)kPanel * (n + kVtcN);
    int64_t b = (int64_t)kPanel * kVtcN * (8LL * device_sm_count() + 8);
    return a > b ? a : b;
}

size_t qr_scratch_bytes(int64_t s, int64_t n, int elem_bytes) {
    Carve c{nullptr, 0, 0, true};
    qr_scratch_carve(c, s, n, elem_bytes);
    return c.off;
}

QrScratch qr_scratch_carve(Carve& c, int64_t s, int64_t n, int elem_bytes) {
    (void)s;
    QrScratch q;
    const size_t e = elem_bytes == 8 ? 1 : 2;   // carve in doubles; floats use half
    q.tau = c.take<double>((size_t)n / e + 1);
    q.T = c.take<double>(kPanel * kPanel);
    q.part_elems = (int64_t)device_sm_count() * kPartStride + 8 + kPanel * kPanel;
    if (obpanel_partial_elems(device_sm_count()) > q.part_elems) q.part_elems = obpanel_partial_elems(device_sm_count());
    q.partials = c.take<double>((size_t)q.part_elems);
    q.wp_elems = wp_capacity(n);
    q.Wp = c.take<double>((size_t)q.wp_elems);
    q.Wn = c.take<double>((size_t)kPanel * (size_t)(n + kVtcN));
    q.bar = c.take<GridBarrier>(1);
    return q;
}

// Apply the panel at columns [j0, j0 + nbw) (V below its diagonal, T in Tm) to columns
// [j0 + nbw, n): W = V^T C (split over row chunks), Wn = -T^T W, C += V Wn.
template <class T>
static int trailing_update(T* A, int64_t lda, int64_t s, int64_t n, int64_t j0, int nbw, const QrScratch& q,
                           const T* Tm, cudaStream_t st, bool timed = true) {
    const int64_t L = s - j0;
    const int64_t nprime = n - j0 - nbw;
    if (nprime <= 0) return CSLS_OK;
    T* Wp = reinterpret_cast<T*>(q.Wp);
    T* Wn = reinterpret_cast<T*>(q.Wn);
    const int64_t ntn = ceil_div(nprime, kVtcN);
    int64_t ks = ceil_div(4LL * device_sm_count(), ntn);
    const int64_t maxks = ceil_div(L, kVtcRows);
    if (ks > maxks) ks = maxks;
    if (ks < 1) ks = 1;
    while (ks > 1 && ks * kPanel * ntn * kVtcN > q.wp_elems * (int64_t)(8 / sizeof(T))) --ks;
    const int64_t kc = round_up(ceil_div(L, ks), kVtcRows);
    ks = ceil_div(L, kc);
    const double prod_flop = 2.0 * (double)L * (double)nprime * (double)nbw;
    int tk = timed ? kt_begin(kFamVtc, st) : -1;
    if (sizeof(T) == 8)
        k_vtc_f64<<<dim3((unsigned)ntn, (unsigned)ks), 256, 0, st>>>((const double*)A, lda, s, n, j0, nbw, kc,
                                                                     (double*)Wp, nprime);
    else
        k_vtc_f32<<<dim3((unsigned)ntn, (unsigned)ks), 256, 0, st>>>((const float*)A, lda, s, n, j0, nbw, kc,
                                                                     (float*)Wp, nprime);
    CSLS_CUDA(cudaGetLastError());
    kt_end(tk, prod_flop, st);
    int ksr = (int)ks;
    if (ks > 8) {
        // many row chunks (narrow trailing blocks): sum the partials of each entry with a warp first,
        // in place into chunk 0, so that the T^T product below reads one partial per entry
        const int64_t entries = (int64_t)nbw * nprime;
        const int g = (int)std::min<int64_t>(ceil_div(entries * 32, 256), (int64_t)device_sm_count() * 8);
        k_psum<T><<<g, 256, 0, st>>>(Wp, (int)ks, nbw, nprime);
        CSLS_CUDA(cudaGetLastError());
        ksr = 1;
    }
    k_wreduce<T><<<(unsigned)ceil_div(nprime, kWrCols), 256, 0, st>>>(Wp, ksr, Tm, nbw, Wn, nprime);
    CSLS_CUDA(cudaGetLastError());
    dim3 ug((unsigned)ceil_div(L, kUpdM), (unsigned)ceil_div(nprime, kUpdN));
    tk = timed ? kt_begin(kFamUpdate, st) : -1;
    if (sizeof(T) == 8)
        k_update_f64<<<ug, 256, 0, st>>>((double*)A, lda, s, n, j0, nbw, (const double*)Wn, nprime);
    else
        k_update_f32<<<dim3((unsigned)ceil_div(L, kUpdM32), ug.y), 256, 0, st>>>((float*)A, lda, s, n, j0, nbw,
                                                                                (const float*)Wn, nprime);
    CSLS_CUDA(cudaGetLastError());
    kt_end(tk, prod_flop, st);
    return CSLS_OK;
}

template <class T>
static int qr_factor_impl(T* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, int* err, long long spin,
                          cudaStream_t st, int64_t* launches) {
    if (s < n || n <= 0) return CSLS_ERR_ARG;
    CSLS_CUDA(cudaMemsetAsync(q.bar, 0, sizeof(GridBarrier), st));
    T* tau = reinterpret_cast<T*>(q.tau);
    T* Tm = reinterpret_cast<T*>(q.T);
    T* part = reinterpret_cast<T*>(q.partials);
    const size_t smem_cap = 200 * 1024;
    CSLS_TRY(raise_smem_limit((const void*)k_panel<T, true>, (int)smem_cap));
    int64_t nl = 0;
    for (int64_t j0 = 0; j0 < n; j0 += kPanel) {
        const int nbw = (int)(n - j0 < kPanel ? n - j0 : kPanel);
        const int64_t L = s - j0;
        int G = panel_grid(L);
        int64_t chunk = ceil_div(L, G);
        size_t smem = (size_t)chunk * nbw * sizeof(T);
        const bool use_smem = smem <= smem_cap;
        long long spin_ll = spin;
        void* args[] = {&A, (void*)&lda, (void*)&s, (void*)&j0, (void*)&nbw, (void*)&chunk, &tau, &Tm, &part,
                        (void*)&q.bar, &spin_ll, &err};
        cudaError_t ce;
        const int tkp = kt_begin(kFamPanel, st);
        if (use_smem)
            ce = cudaLaunchCooperativeKernel((const void*)k_panel<T, true>, dim3(G), dim3(kPanelThreads), args, smem, st);
        else
            ce = cudaLaunchCooperativeKernel((const void*)k_panel<T, false>, dim3(G), dim3(kPanelThreads), args, 0, st);
        CSLS_CUDA(ce);
        kt_end(tkp, 0.0, st);
        ++nl;
        if (n - j0 - nbw <= 0) continue;
        CSLS_TRY(trailing_update<T>(A, lda, s, n, j0, nbw, q, Tm, st));
        nl += 3;
    }
    if (launches) *launches += nl;
    return CSLS_OK;
}

int qr_trailing_update_f64(double* A, int64_t lda, int64_t s, int64_t n_end, int64_t j0, int nbw, const QrScratch& q,
                           cudaStream_t st) {
    return trailing_update<double>(A, lda, s, n_end, j0, nbw, q, q.T, st, false);
}

int qr_panel_launch_f64(double* A, int64_t lda, int64_t s, int64_t j0, int nbw, const QrScratch& q, int* err,
                        long long spin, cudaStream_t st) {
    const size_t smem_cap = 200 * 1024;
    CSLS_TRY(raise_smem_limit((const void*)k_panel<double, true>, (int)smem_cap));
    const int64_t L = s - j0;
    int G = panel_grid(L);
    int64_t chunk = ceil_div(L, G);
    size_t smem = (size_t)chunk * nbw * sizeof(double);
    double* tau = q.tau;
    double* Tm = q.T;
    double* part = q.partials;
    long long spin_ll = spin;
    void* args[] = {&A, (void*)&lda, (void*)&s, (void*)&j0, (void*)&nbw, (void*)&chunk, &tau, &Tm, &part,
                    (void*)&q.bar, &spin_ll, &err};
    if (smem <= smem_cap)
        CSLS_CUDA(cudaLaunchCooperativeKernel((const void*)k_panel<double, true>, dim3(G), dim3(kPanelThreads), args,
                                              smem, st));
    else
        CSLS_CUDA(cudaLaunchCooperativeKernel((const void*)k_panel<double, false>, dim3(G), dim3(kPanelThreads), args,
                                              0, st));
    return CSLS_OK;
}

int qr_factor_f64(double* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, int* err, long long spin,
                  cudaStream_t st, int64_t* launches) {
    return qr_factor_impl<double>(A, lda, s, n, q, err, spin, st, launches);
}
int qr_factor_f32(float* A, int64_t lda, int64_t s, int64_t n, const QrScratch& q, int* err, long long spin,
                  cudaStream_t st, int64_t* launches) {
    return qr_factor_impl<float>(A, lda, s, n, q, err, spin, st, launches);
}

template <class T>
static int extract_impl(const T* A, int64_t lda, int64_t n, T* R, double* stats, cudaStream_t st) {
    dim3 g((unsigned)ceil_div(n, 256), (unsigned)(n < 65535 ? n : 65535));
    k_extract_r<T><<<g, 256, 0, st>>>(A, lda, n, R);
    CSLS_CUDA(cudaGetLastError());
    k_rdiag_stats<T><<<1, 1024, 0, st>>>(R, n, stats);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}
// z(i) = sign(A_ii) A(i, n), i < n: column n of the factored augmented sketch [SA, Sb] holds
// Q^T S b in its first n rows; the sign follows the row flips that make R's diagonal
// non-negative.
template <class T>
__global__ void k_extract_qtb(const T* A, int64_t lda, int64_t n, double* z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)A[i + n * lda];
        z[i] = A[i + i * lda] < T(0) ? -v : v;
    }
}

int qr_extract_qtb_f64(const double* A, int64_t lda, int64_t n, double* z, cudaStream_t st) {
    k_extract_qtb<double><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1024)), 256, 0, st>>>(
        A, lda, n, z);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}
int qr_extract_qtb_f32(const float* A, int64_t lda, int64_t n, double* z, cudaStream_t st) {
    k_extract_qtb<float><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1024)), 256, 0, st>>>(
        A, lda, n, z);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

int qr_extract_r_f64(const double* A, int64_t lda, int64_t n, double* R, double* stats, cudaStream_t st) {
    return extract_impl<double>(A, lda, n, R, stats, st);
}
int qr_extract_r_f32(const float* A, int64_t lda, int64_t n, float* R, double* stats, cudaStream_t st) {
    return extract_impl<float>(A, lda, n, R, stats, st);
}

int diag_block_inverses_f64(const double* R, int64_t n, double* Dinv, cudaStream_t st) {
    k_diag_inverse<double><<<(unsigned)ceil_div(n, kTrsvBlock), kTrsvBlock, 0, st>>>(R, n, Dinv);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}
int diag_block_inverses_f32(const float* R, int64_t n, double* Dinv, cudaStream_t st) {
    k_diag_inverse<float><<<(unsigned)ceil_div(n, kTrsvBlock), kTrsvBlock, 0, st>>>(R, n, Dinv);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

}  // namespace csls

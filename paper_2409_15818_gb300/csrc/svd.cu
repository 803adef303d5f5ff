// One-sided Jacobi SVD of R (Hestenes; Demmel and Veselic 1992) for the
// CSSVDP preconditioner (Algorithm 2 step 3): SA = Q R, so SA and R share Sigma
// and V. Column pairs of G = R are orthogonalised by plane rotations in the
// round-robin (circle) order: each step rotates n/2 disjoint pairs, one CTA per
// pair, accumulating the same rotations into V. Sweeps repeat until no pair
// needs a rotation. Then P = V_r Sigma_r^{-1} keeps sigma_i > rcond sigma_1.
#include <algorithm>
#include <cmath>
#include <vector>

#include "csls_internal.cuh"

namespace csls {

constexpr int kJacThreads = 256;

// One plane rotation of the column pair with index pidx in round-robin step `step` (all threads
// of the CTA take part; shared scratch is passed in).
__device__ __forceinline__ void jacobi_pair(double* G, double* V, int64_t n, int64_t N, int64_t step, int64_t pidx,
                                            double tol, double floor_c, unsigned* rotations, double (*red)[kJacThreads / 32],
                                            double* cs_s, int* skip_s) {
    int64_t a, b;
    if (pidx == 0) {
        a = step % (N - 1);
        b = N - 1;
    } else {
        a = (step + pidx) % (N - 1);
        b = (step - pidx + (N - 1)) % (N - 1);
    }
    if (a > b) { int64_t t = a; a = b; b = t; }
    if (b >= n) return;   // padding column (uniform across the CTA)
    double* ga = G + a * n;
    double* gb = G + b * n;
    double saa = 0.0, sbb = 0.0, sab = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kJacThreads) {
        const double x = ga[i], y = gb[i];
        saa += x * x; sbb += y * y; sab += x * y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        saa += __shfl_xor_sync(0xffffffffu, saa, o);
        sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
        sab += __shfl_xor_sync(0xffffffffu, sab, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = saa; red[1][threadIdx.x >> 5] = sbb; red[2][threadIdx.x >> 5] = sab;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0, C = 0.0;
        for (int w = 0; w < kJacThreads / 32; ++w) { A += red[0][w]; B += red[1][w]; C += red[2][w]; }
        // no rotation when the pair is already orthogonal to working accuracy, when its inner product
        // is below the floor, or when one column's squared norm is (that column is truncated later; the
        // numerically zero columns of a rank-deficient R would otherwise keep rotating on noise)
        if (C == 0.0 || fabs(C) <= tol * sqrt(A * B) || fabs(C) <= floor_c || fmin(A, B) <= floor_c) {
            *skip_s = 1;
        } else {
            *skip_s = 0;
            const double zeta = (B - A) / (2.0 * C);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            cs_s[0] = c;
            cs_s[1] = c * t;
            atomicAdd(rotations, 1u);
        }
    }
    __syncthreads();
    const int skip = *skip_s;
    const double c = cs_s[0], s = cs_s[1];
    __syncthreads();   // the shared scratch is reused by the CTA's next pair
    if (skip) return;
    double* va = V + a * n;
    double* vb = V + b * n;
    for (int64_t i = threadIdx.x; i < n; i += kJacThreads) {
        const double x = ga[i], y = gb[i];
        ga[i] = c * x - s * y;
        gb[i] = s * x + c * y;
        const double p = va[i], q = vb[i];
        va[i] = c * p - s * q;
        vb[i] = s * p + c * q;
    }
}

// A whole sweep in one cooperative launch: the N - 1 round-robin steps are separated by grid
// barriers; a CTA takes pairs blockIdx.x, blockIdx.x + gridDim.x, ... of each step.
__global__ void __launch_bounds__(kJacThreads)
k_jacobi_sweep(double* G, double* V, int64_t n, int64_t N, double tol, double floor_c, unsigned* rotations,
               GridBarrier* bar, long long spin, int* err) {
    __shared__ double red[3][kJacThreads / 32];
    __shared__ double cs_s[2];
    __shared__ int skip_s;
    for (int64_t step = 0; step < N - 1; ++step) {
        for (int64_t pidx = blockIdx.x; pidx < N / 2; pidx += gridDim.x)
            jacobi_pair(G, V, n, N, step, pidx, tol, floor_c, rotations, red, cs_s, &skip_s);
        if (!grid_sync(bar, gridDim.x, spin, err)) return;
    }
}

__global__ void k_copy_init(const double* R, double* G, double* V, int64_t n) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        G[idx] = R[idx];
        V[idx] = (idx % n == idx / n) ? 1.0 : 0.0;
    }
}

__global__ void __launch_bounds__(kJacThreads) k_col_norms(const double* G, int64_t n, double* sigma) {
    __shared__ double red[kJacThreads / 32];
    const double* g = G + (int64_t)blockIdx.x * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kJacThreads) s += g[i] * g[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kJacThreads / 32; ++w) t += red[w];
        sigma[blockIdx.x] = sqrt(t);
    }
}

__global__ void k_form_p(const double* V, const double* sigma, const int* order, int64_t n, int64_t r, double* P,
                         double* sigma_sorted) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * r;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx % n, k = idx / n;
        const int src = order[k];
        P[i + k * n] = V[i + (int64_t)src * n] / sigma[src];
        if (i == 0) sigma_sorted[k] = sigma[src];
    }
}

int svd_precond(const double* R, int64_t n, double rcond, double* G, double* V, double* sigma, double* P, int* order,
                int64_t* r_out, GridBarrier* bar, long long spin, int* err, cudaStream_t st, int64_t* launches) {
    const int64_t N = n + (n & 1);
    k_copy_init<<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 65535), 256, 0, st>>>(R, G, V, n);
    CSLS_CUDA(cudaGetLastError());
    // rotations counter lives in the first word of `order` until the ordering is written
    unsigned* rot = reinterpret_cast<unsigned*>(order);
    // a pair counts as orthogonal once |g_a^T g_b| <= sqrt(n) u ||g_a|| ||g_b|| (the convergence test of
    // LAPACK's one-sided Jacobi): tighter than the rounding of the dot products themselves, sweeps would
    // keep rotating pairs on noise
    const double tol = std::max(1e-15, std::sqrt((double)n) * 1.1102230246251565e-16);
    // rounding floor of the inner products: n u^2 ||R||_F^2 (P is scratch until it is formed)
    k_col_norms<<<(unsigned)n, kJacThreads, 0, st>>>(G, n, P);
    CSLS_CUDA(cudaGetLastError());
    std::vector<double> cn((size_t)n);
    CSLS_CUDA(cudaMemcpyAsync(cn.data(), P, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    double frob2 = 0.0;
    for (double v : cn) frob2 += v * v;
    // below (1e-2 rcond)^2 ||R||_F^2 an inner product is noise of columns that end up truncated, or turns
    // a column at the truncation edge by less than 1e-4 rad: such pairs are left alone, so the sweeps of a
    // rank-deficient R converge instead of rotating its numerically zero columns on rounding noise
    const double u = 1.1102230246251565e-16;
    const double floor_c = std::max((double)n * u * u, 1e-4 * rcond * rcond) * frob2;
    int64_t nl = 1;
    int per_sm = 0;
    CSLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_sweep, kJacThreads, 0));
    const int64_t resident = (int64_t)std::max(per_sm, 1) * device_sm_count();
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(N / 2, resident));
    CSLS_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st));
    for (int sweep = 0; sweep < 60 && N >= 2; ++sweep) {
        CSLS_CUDA(cudaMemsetAsync(rot, 0, sizeof(unsigned), st));
        void* args[] = {&G, (void*)&V, (void*)&n, (void*)&N, (void*)&tol, (void*)&floor_c, (void*)&rot, (void*)&bar,
                        (void*)&spin, (void*)&err};
        CSLS_CUDA(cudaLaunchCooperativeKernel((const void*)k_jacobi_sweep, dim3(grid), dim3(kJacThreads), args, 0, st));
        nl += 1;
        unsigned h_rot = 0;
        int h_err = 0;
        CSLS_CUDA(cudaMemcpyAsync(&h_rot, rot, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CSLS_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CSLS_CUDA(cudaStreamSynchronize(st));
        if (h_err) return CSLS_OK;   // the caller reads the error word
        if (h_rot == 0) break;
    }
    // sigma_j = ||G_j||, sorted descending on the host (n values)
    double* sig_raw = P;   // scratch: P is rewritten below
    k_col_norms<<<(unsigned)n, kJacThreads, 0, st>>>(G, n, sig_raw);
    CSLS_CUDA(cudaGetLastError());
    std::vector<double> hs((size_t)n);
    CSLS_CUDA(cudaMemcpyAsync(hs.data(), sig_raw, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    std::vector<int> ord((size_t)n);
    for (int64_t i = 0; i < n; ++i) ord[(size_t)i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return hs[(size_t)x] > hs[(size_t)y]; });
    int64_t r = 0;
    const double s1 = n > 0 ? hs[(size_t)ord[0]] : 0.0;
    while (r < n && hs[(size_t)ord[(size_t)r]] > rcond * s1) ++r;
    // sigma (device) <- raw norms, order (device) <- permutation; P <- V_r Sigma_r^{-1}
    CSLS_CUDA(cudaMemcpyAsync(sigma, hs.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaMemcpyAsync(order, ord.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    if (r > 0) {
        k_form_p<<<(unsigned)std::min<int64_t>(ceil_div(n * r, 256), 65535), 256, 0, st>>>(V, sigma, order, n, r, P,
                                                                                             G);
        CSLS_CUDA(cudaGetLastError());
        // sorted singular values end up in G[0..r) ; copy them to sigma
        CSLS_CUDA(cudaMemcpyAsync(sigma, G, sizeof(double) * (size_t)r, cudaMemcpyDeviceToDevice, st));
    }
    *r_out = r;
    if (launches) *launches += nl + 2;
    return CSLS_OK;
}

}  // namespace csls

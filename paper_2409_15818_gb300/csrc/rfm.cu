// Assembly of the random-feature-method least-squares rows on the GPU (Section 2.1 and
// Appendix B): the step before the solve, so that a PDE problem reaches the solver as a few
// megabytes of geometry and feature parameters instead of a host-built CSR matrix.
//
// Box i carries J features phi_ij(x) = tanh(k_ij . l_i(x) + c_ij), l_i the affine map of the
// box onto [-1, 1]^d (half-widths r_d). Each row is described by its kind, box, neighbour box,
// face axis and the local point t of the collocation point:
//   kind 0  -Laplace u at t:          2 tanh(z) (1 - tanh(z)^2) sum_d k_d^2 / r_d^2
//   kind 1  u at t (boundary value):  tanh(z)
//   kind 2  u(box) - u(nbox) across the face t[axis] = +1 of box (C0)
//   kind 3  the same for d u / d x_axis (C1): (1 - tanh(z)^2) k_axis / r_axis
// Interface rows hold the box's J columns then the neighbour's J (with the neighbour's local
// point t[axis] = -1); columns are box-major (column = box J + feature).
#include <algorithm>

#include "csls_internal.cuh"

namespace csls {

__global__ void k_rfm_widths(const csls_rfm_row* rows, int64_t nrows, int J, int* widths) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x)
        widths[i] = rows[i].kind >= 2 ? 2 * J : J;
}

// Sum of the row widths (the nnz of the assembled matrix); integer atomics, so the total does not
// depend on the order in which the warps add.
__global__ void k_rfm_count(const csls_rfm_row* rows, int64_t nrows, int J, unsigned long long* total) {
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x)
        acc += rows[i].kind >= 2 ? 2 * J : J;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

template <int DIM>
__device__ __forceinline__ double feature_z(const double* k, const double* c, int64_t f, const double* t) {
    double z = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) z = fma(t[d], k[f * DIM + d], z);
    return z + c[f];
}

template <int DIM>
__global__ void __launch_bounds__(256) k_rfm_rows(const csls_rfm_row* rows, int64_t nrows, int J, const double* k,
                                                  const double* c, double r0, double r1, double r2,
                                                  const int64_t* row_ptr, int32_t* col, double* val) {
    const double rr[3] = {r0, r1, r2};
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nrows; i += nw) {
        const csls_rfm_row rw = rows[i];
        const int64_t base = row_ptr[i];
        double t[DIM], tn[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            t[d] = rw.t[d];
            tn[d] = (rw.kind >= 2 && d == rw.axis) ? -1.0 : rw.t[d];
        }
        double lap = 0.0, sa = 0.0;
        for (int j = lane; j < J; j += 32) {
            const int64_t f = (int64_t)rw.box * J + j;
            const double th = tanh(feature_z<DIM>(k, c, f, t));
            double v;
            if (rw.kind == 0) {
                lap = 0.0;
#pragma unroll
                for (int d = 0; d < DIM; ++d) lap += k[f * DIM + d] * k[f * DIM + d] * (1.0 / (rr[d] * rr[d]));
                v = 2.0 * th * (1.0 - th * th) * lap;
            } else if (rw.kind == 3) {
                sa = k[f * DIM + rw.axis] / rr[rw.axis];
                v = (1.0 - th * th) * sa;
            } else {
                v = th;
            }
            col[base + j] = (int32_t)f;
            val[base + j] = v;
            if (rw.kind >= 2) {
                const int64_t fn = (int64_t)rw.nbox * J + j;
                const double thn = tanh(feature_z<DIM>(k, c, fn, tn));
                const double vn = rw.kind == 3 ? (1.0 - thn * thn) * (k[fn * DIM + rw.axis] / rr[rw.axis]) : thn;
                col[base + J + j] = (int32_t)fn;
                val[base + J + j] = -vn;
            }
        }
    }
}

}  // namespace csls

using namespace csls;

int csls_rfm_assemble_workspace(int64_t nrows, size_t* bytes) {
    if (nrows <= 0 || !bytes) return CSLS_ERR_ARG;
    *bytes = (size_t)round_up(nrows * 4, 256);
    return CSLS_OK;
}

int csls_rfm_nnz(int64_t nrows, const csls_rfm_row* rows, int64_t J, void* work, size_t work_bytes,
                 int64_t* nnz, csls_stream_t stream) {
    if (nrows <= 0 || !rows || J <= 0 || J > 65536 || !nnz) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_rfm_assemble_workspace(nrows, &need));
    if (!work || work_bytes < need || ((uintptr_t)work & 255) != 0) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* total = (unsigned long long*)work;
    CSLS_CUDA(cudaMemsetAsync(total, 0, sizeof(*total), st));
    const int64_t cap = (int64_t)device_sm_count() * 8;
    const int g = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(nrows, 256)), cap);
    k_rfm_count<<<g, 256, 0, st>>>(rows, nrows, (int)J, total);
    CSLS_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    CSLS_CUDA(cudaMemcpyAsync(&h, total, sizeof(h), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    *nnz = (int64_t)h;
    return CSLS_OK;
}

int csls_rfm_assemble(int dim, const double* r_half, int64_t J, const double* k, const double* c, int64_t nrows,
                      const csls_rfm_row* rows, int64_t* row_ptr, int32_t* col, double* val, void* work,
                      size_t work_bytes, csls_stream_t stream) {
    if ((dim != 2 && dim != 3) || !r_half || J <= 0 || J > 65536 || !k || !c || nrows <= 0 || !rows || !row_ptr ||
        !col || !val)
        return CSLS_ERR_ARG;
    for (int d = 0; d < dim; ++d)
        if (!(r_half[d] > 0.0)) return CSLS_ERR_ARG;
    size_t need = 0;
    CSLS_TRY(csls_rfm_assemble_workspace(nrows, &need));
    if (!work || work_bytes < need || ((uintptr_t)work & 255) != 0) return CSLS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int* widths = (int*)work;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    const int gw = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(nrows, 256)), cap);
    k_rfm_widths<<<gw, 256, 0, st>>>(rows, nrows, (int)J, widths);
    CSLS_CUDA(cudaGetLastError());
    CSLS_TRY(scan_counts(widths, row_ptr, nrows, st));
    const int gr = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(nrows * 32, 256)), cap);
    const double r2 = dim == 3 ? r_half[2] : 1.0;
    if (dim == 2)
        k_rfm_rows<2><<<gr, 256, 0, st>>>(rows, nrows, (int)J, k, c, r_half[0], r_half[1], r2, row_ptr, col, val);
    else
        k_rfm_rows<3><<<gr, 256, 0, st>>>(rows, nrows, (int)J, k, c, r_half[0], r_half[1], r2, row_ptr, col, val);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

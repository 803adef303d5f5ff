// Count sketch SA = Phi D A (Definition 2.3; Algorithm 1 step 2).
//
// Design: rows are bucketed by h(i) with a counting sort (histogram, scan,
// scatter, per-bucket sort into ascending row order), then one warp owns one
// bucket and streams that bucket's rows in ascending order, adding d(i) * A[i, :]
// into row h(i) of the dense column-major SA. Different warps never write the
// same row of SA and lanes of a warp never write the same entry within one row
// (CSR columns are distinct), so there are no floating-point atomics and every
// entry is summed in ascending row order -- the result is bit-reproducible.
#include "csls_internal.cuh"

namespace csls {

// Round-to-nearest addition that the compiler may not contract or reorder.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

__device__ __forceinline__ void hash_row(uint64_t seed, int64_t i, uint32_t s, uint32_t* bucket, bool* neg) {
    uint64_t z = splitmix_mix(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
    *bucket = (uint32_t)(((z >> 32) * (uint64_t)s) >> 32);
    *neg = (z & 1ULL) != 0;
}

__global__ void k_hash_count(int64_t m, uint32_t s, uint64_t seed, int* counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b;
        bool neg;
        hash_row(seed, i, s, &b, &neg);
        atomicAdd(&counts[b], 1);
    }
}

__global__ void k_hash_scatter(int64_t m, uint32_t s, uint64_t seed, const int64_t* offsets, int* cursor,
                               int32_t* list) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b;
        bool neg;
        hash_row(seed, i, s, &b, &neg);
        int pos = atomicAdd(&cursor[b], 1);
        list[offsets[b] + pos] = (int32_t)i;
    }
}

template <class T>
__global__ void k_zero_cols(T* SA, int64_t s, int64_t n, int64_t ld) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        T* colp = SA + j * ld;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
            colp[i] = T(0);
    }
}

// Contiguous zero fill with 16-byte stores (ld == s and 16-byte aligned base).
__global__ void k_zero_vec(double2* p, int64_t count2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count2; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_double2(0.0, 0.0);
}

template <class T>
__global__ void __launch_bounds__(256) k_segsum(const int64_t* offsets, const int32_t* list, const int64_t* row_ptr,
                                                const int32_t* col, const double* val, int64_t s, uint64_t seed,
                                                T* SA, int64_t ld) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < s; k += nwarps) {
        T* dst_row = SA + k;
        for (int64_t e = offsets[k]; e < offsets[k + 1]; ++e) {
            const int64_t i = list[e];
            uint32_t b;
            bool neg;
            hash_row(seed, i, (uint32_t)s, &b, &neg);
            for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
                T a = (T)val[p];
                if (neg) a = -a;
                T* dst = dst_row + (int64_t)col[p] * ld;
                *dst = add_rn(*dst, a);
            }
            __syncwarp();   // orders this row's updates before the next row's (same warp)
        }
    }
}

size_t sketch_scratch_bytes(int64_t m, int64_t s) {
    Carve c{nullptr, 0, 0, true};
    sketch_scratch_carve(c, m, s);
    return c.off;
}

SketchScratch sketch_scratch_carve(Carve& c, int64_t m, int64_t s) {
    SketchScratch sc;
    sc.counts = c.take<int>((size_t)s);
    sc.offsets = c.take<int64_t>((size_t)s + 1);
    sc.cursor = c.take<int>((size_t)s);
    sc.list = c.take<int32_t>((size_t)(m > 0 ? m : 1));
    return sc;
}

static int grid_cap(int64_t work, int threads) {
    int64_t g = ceil_div(work, threads);
    int64_t cap = (int64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// S b for a dense m-vector b from the bucket lists of the last sketch_run (same seed and s):
// out[k] = sum over the rows i hashed to bucket k, in ascending order, of d(i) b(i), rounded
// to T after each addition (one thread per bucket; every bucket is written, empty ones as 0).
template <class T>
__global__ void __launch_bounds__(256) k_sketch_vec(const int64_t* offsets, const int32_t* list, const double* b,
                                                    int64_t s, uint64_t seed, T* out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s; k += (int64_t)gridDim.x * blockDim.x) {
        T acc = T(0);
        for (int64_t e = offsets[k]; e < offsets[k + 1]; ++e) {
            const int64_t i = list[e];
            uint32_t bk;
            bool neg;
            hash_row(seed, i, (uint32_t)s, &bk, &neg);
            T a = (T)b[i];
            if (neg) a = -a;
            acc = add_rn(acc, a);
        }
        out[k] = acc;
    }
}

int sketch_vec_run(const SketchScratch& sc, const double* b, int64_t s, uint64_t seed, int prec, void* out,
                   cudaStream_t st, int64_t* launches) {
    const int blocks = grid_cap(s, 256);
    if (prec == CSLS_PREC_F32)
        k_sketch_vec<float><<<blocks, 256, 0, st>>>(sc.offsets, sc.list, b, s, seed, (float*)out);
    else
        k_sketch_vec<double><<<blocks, 256, 0, st>>>(sc.offsets, sc.list, b, s, seed, (double*)out);
    CSLS_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
    return CSLS_OK;
}

int sketch_run(const csls_csr* A, int64_t s, uint64_t seed, int prec, void* SA, int64_t ld, const SketchScratch& sc,
               int* err, cudaStream_t st, int64_t* launches) {
    (void)err;
    const int64_t m = A->m, n = A->n;
    CSLS_CUDA(cudaMemsetAsync(sc.counts, 0, sizeof(int) * (size_t)s, st));
    CSLS_CUDA(cudaMemsetAsync(sc.cursor, 0, sizeof(int) * (size_t)s, st));
    k_hash_count<<<grid_cap(m, 256), 256, 0, st>>>(m, (uint32_t)s, seed, sc.counts);
    CSLS_CUDA(cudaGetLastError());
    CSLS_TRY(scan_counts(sc.counts, sc.offsets, s, st));
    k_hash_scatter<<<grid_cap(m, 256), 256, 0, st>>>(m, (uint32_t)s, seed, sc.offsets, sc.cursor, sc.list);
    CSLS_CUDA(cudaGetLastError());
    // Bucket sizes are Poisson(m/s), but nothing bounds the longest one on the host side, so
    // all three sort stages are launched (each returns at once for segments outside its size
    // range): every bucket ends up in ascending row order whatever its length.
    CSLS_TRY(segmented_sort(sc.list, nullptr, sc.offsets, s, m, st));
    const int esz = prec == CSLS_PREC_F64 ? 8 : 4;
    if (ld == s && esz == 8 && ((uintptr_t)SA % 16) == 0 && (s * n) % 2 == 0) {
        k_zero_vec<<<grid_cap(s * n / 2, 256), 256, 0, st>>>((double2*)SA, s * n / 2);
    } else if (esz == 8) {
        dim3 g((unsigned)ceil_div(s, 256 * 4) > 0 ? (unsigned)ceil_div(s, 256 * 4) : 1u,
               (unsigned)(n < 65535 ? (n > 0 ? n : 1) : 65535));
        k_zero_cols<double><<<g, 256, 0, st>>>((double*)SA, s, n, ld);
    } else {
        dim3 g((unsigned)ceil_div(s, 256 * 4) > 0 ? (unsigned)ceil_div(s, 256 * 4) : 1u,
               (unsigned)(n < 65535 ? (n > 0 ? n : 1) : 65535));
        k_zero_cols<float><<<g, 256, 0, st>>>((float*)SA, s, n, ld);
    }
    CSLS_CUDA(cudaGetLastError());
    const int sum_blocks = grid_cap(s * 32, 256);
    if (esz == 8)
        k_segsum<double><<<sum_blocks, 256, 0, st>>>(sc.offsets, sc.list, A->row_ptr, A->col, A->val, s, seed,
                                                     (double*)SA, ld);
    else
        k_segsum<float><<<sum_blocks, 256, 0, st>>>(sc.offsets, sc.list, A->row_ptr, A->col, A->val, s, seed,
                                                    (float*)SA, ld);
    CSLS_CUDA(cudaGetLastError());
    if (launches) *launches += 8;
    return CSLS_OK;
}

}  // namespace csls

// ======================================================================= no-allocation variant
//
// csls_sketch_noalloc runs csls_sketch with a fixed, library-owned scratch area
// instead of a caller workspace. The area is a file-scope __device__ array, so
// every GPU that loads the library holds these bytes until the process exits.
// Host code cannot use the array's name as a device address; its address is
// looked up once per device with cudaGetSymbolAddress (with that device current)
// on the first call made on that device.

#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_sketch_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

int noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CSLS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CSLS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sketch_scratch) != cudaSuccess || !p) return CSLS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CSLS_OK;
}

}  // namespace

extern "C" int csls_sketch_noalloc(const csls_csr* A, int64_t s, uint64_t seed, int prec, void* SA, int64_t ld,
                                   csls_stream_t stream) {
    if (!A || s <= 0 || s > 2147483647LL) return CSLS_ERR_ARG;
    size_t need = 0;
    const int rc = csls_sketch_workspace(A, s, &need);
    if (rc != CSLS_OK) return rc;
    if (need > kNoAllocScratchBytes) return CSLS_ERR_WORKSPACE;   // beyond the static maximum
    void* scratch = nullptr;
    const int sc = noalloc_scratch(&scratch);
    if (sc != CSLS_OK) return sc;
    // csls_sketch clears every scratch entry that must start at zero.
    return csls_sketch(A, s, seed, prec, SA, ld, scratch, kNoAllocScratchBytes, stream);
}

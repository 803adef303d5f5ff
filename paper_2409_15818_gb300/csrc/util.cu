// Scans, segmented sorts, CSR validation and the transposed copy of A.
#include <climits>
#include <cstdio>

#include <vector>

#include <mutex>
#include <set>
#include <utility>

#include "csls_internal.cuh"

namespace csls {

namespace {
thread_local char g_last_cuda_error[256] = "";
}  // namespace

void note_cuda_error(cudaError_t e, const char* where) {
    const char* file = where;
    for (const char* p = where; *p; ++p)
        if (*p == '/') file = p + 1;
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s (%s) at %s", cudaGetErrorName(e),
             cudaGetErrorString(e), file);
}

const char* last_cuda_error() { return g_last_cuda_error; }

namespace {
constexpr int kMaxDev = 64;
std::mutex g_dev_mu;
int g_sm_count[kMaxDev] = {};
std::set<std::pair<const void*, int>> g_smem_attr_done;   // (kernel, device) pairs already raised
}  // namespace

int device_sm_count() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (g_sm_count[dev] == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
        g_sm_count[dev] = v > 0 ? v : 1;
    }
    return g_sm_count[dev];
}

int raise_smem_limit(const void* kernel, int bytes) {
    int dev = 0;
    CSLS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_dev_mu);
    const auto key = std::make_pair(kernel, dev);
    if (g_smem_attr_done.count(key)) return CSLS_OK;
    CSLS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    g_smem_attr_done.insert(key);
    return CSLS_OK;
}

// ------------------------------------------------------------------ per-family kernel timing

namespace {
struct KtSpan {
    cudaEvent_t a, b;
    int fam;
    double flop;
};
struct KtState {
    bool on = false;
    std::vector<KtSpan> spans;
};
thread_local KtState kt_state;
}  // namespace

void kt_install(bool on) {
    kt_state.on = on;
    kt_state.spans.clear();
}

int kt_begin(int fam, cudaStream_t st) {
    if (!kt_state.on) return -1;
    KtSpan sp{nullptr, nullptr, fam, 0.0};
    if (cudaEventCreate(&sp.a) != cudaSuccess || cudaEventCreate(&sp.b) != cudaSuccess) return -1;
    cudaEventRecord(sp.a, st);
    kt_state.spans.push_back(sp);
    return (int)kt_state.spans.size() - 1;
}

void kt_end(int token, double flop, cudaStream_t st) {
    if (token < 0 || token >= (int)kt_state.spans.size()) return;
    KtSpan& sp = kt_state.spans[(size_t)token];
    sp.flop = flop;
    cudaEventRecord(sp.b, st);
}

void kt_collect(double ms[3], int64_t launches[3], double flop[3]) {
    for (int f = 0; f < 3; ++f) { ms[f] = 0.0; launches[f] = 0; flop[f] = 0.0; }
    for (KtSpan& sp : kt_state.spans) {
        float t = 0.f;
        if (sp.a && sp.b && cudaEventElapsedTime(&t, sp.a, sp.b) == cudaSuccess && sp.fam >= 0 && sp.fam < 3) {
            ms[sp.fam] += t;
            launches[sp.fam] += 1;
            flop[sp.fam] += sp.flop;
        }
        if (sp.a) cudaEventDestroy(sp.a);
        if (sp.b) cudaEventDestroy(sp.b);
    }
    kt_install(false);
}

// ------------------------------------------------------------------ exclusive scan (one block)

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_counts(const int* in, int64_t* out, int64_t len) {
    __shared__ int64_t sums[kScanThreads];
    const int t = threadIdx.x;
    const int64_t chunk = (len + kScanThreads - 1) / kScanThreads;
    const int64_t beg = (int64_t)t * chunk;
    const int64_t end = beg + chunk < len ? beg + chunk : len;
    int64_t s = 0;
    for (int64_t i = beg; i < end; ++i) s += in[i];
    sums[t] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {   // inclusive Hillis-Steele
        int64_t v = t >= o ? sums[t - o] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int64_t run = sums[t] - s;
    for (int64_t i = beg; i < end; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (t == kScanThreads - 1) out[len] = sums[t];
}

int scan_counts(const int* counts, int64_t* out, int64_t len, cudaStream_t st) {
    k_scan_counts<<<1, kScanThreads, 0, st>>>(counts, out, len);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

// ------------------------------------------------------------------ segmented sort

constexpr int kSmallSeg = 32;
constexpr int kCtaSeg = 4096;
constexpr int kSortThreads = 512;

__global__ void k_sort_small(int32_t* keys, int32_t* pay, const int64_t* off, int64_t nseg) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nseg) return;
    int64_t b = off[k], e = off[k + 1];
    if (e - b > kSmallSeg || e - b < 2) return;
    for (int64_t i = b + 1; i < e; ++i) {     // insertion sort
        int32_t key = keys[i];
        int32_t p = pay ? pay[i] : 0;
        int64_t j = i - 1;
        while (j >= b && keys[j] > key) {
            keys[j + 1] = keys[j];
            if (pay) pay[j + 1] = pay[j];
            --j;
        }
        keys[j + 1] = key;
        if (pay) pay[j + 1] = p;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_cta(int32_t* keys, int32_t* pay, const int64_t* off) {
    __shared__ int32_t sk[kCtaSeg];
    __shared__ int32_t sp[kCtaSeg];
    const int64_t b = off[blockIdx.x], e = off[blockIdx.x + 1];
    const int len = (int)(e - b);
    if (len <= kSmallSeg || len > kCtaSeg) return;
    int np = 1;
    while (np < len) np <<= 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        sk[i] = i < len ? keys[b + i] : INT_MAX;
        sp[i] = (i < len && pay) ? pay[b + i] : 0;
    }
    __syncthreads();
    for (int size = 2; size <= np; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                int j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    int32_t a = sk[i], c = sk[j];
                    if ((a > c) == up) {
                        sk[i] = c; sk[j] = a;
                        int32_t t = sp[i]; sp[i] = sp[j]; sp[j] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        keys[b + i] = sk[i];
        if (pay) pay[b + i] = sp[i];
    }
}

// Odd-even transposition sort in global memory for rare long segments.
__global__ void __launch_bounds__(kSortThreads) k_sort_big(int32_t* keys, int32_t* pay, const int64_t* off) {
    const int64_t b = off[blockIdx.x], e = off[blockIdx.x + 1];
    const int64_t len = e - b;
    if (len <= kCtaSeg) return;
    for (int64_t phase = 0; phase < len; ++phase) {
        for (int64_t i = (phase & 1) + 2 * (int64_t)threadIdx.x; i + 1 < len; i += 2 * (int64_t)blockDim.x) {
            int32_t a = keys[b + i], c = keys[b + i + 1];
            if (a > c) {
                keys[b + i] = c; keys[b + i + 1] = a;
                if (pay) { int32_t t = pay[b + i]; pay[b + i] = pay[b + i + 1]; pay[b + i + 1] = t; }
            }
        }
        __syncthreads();
    }
}

// max_hint must bound the longest segment from above (stages for longer segments are skipped).
int segmented_sort(int32_t* keys, int32_t* payload, const int64_t* off, int64_t nseg, int64_t max_hint,
                   cudaStream_t st) {
    if (nseg <= 0) return CSLS_OK;
    k_sort_small<<<(unsigned)ceil_div(nseg, 256), 256, 0, st>>>(keys, payload, off, nseg);
    CSLS_CUDA(cudaGetLastError());
    if (max_hint > kSmallSeg) {
        for (int64_t s0 = 0; s0 < nseg; s0 += 2147483647LL) {
            unsigned g = (unsigned)(nseg - s0 < 2147483647LL ? nseg - s0 : 2147483647LL);
            k_sort_cta<<<g, kSortThreads, 0, st>>>(keys, payload, off + s0);
            CSLS_CUDA(cudaGetLastError());
            if (max_hint > kCtaSeg) {
                k_sort_big<<<g, kSortThreads, 0, st>>>(keys, payload, off + s0);
                CSLS_CUDA(cudaGetLastError());
            }
        }
    }
    return CSLS_OK;
}

// ------------------------------------------------------------------ transposed CSR

__global__ void k_col_count(const int32_t* col, int64_t nnz, int64_t n, int* counts, int* err) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t j = col[p];
        if (j < 0 || j >= n) { set_error(err, CSLS_ERR_ARG); continue; }
        atomicAdd(&counts[j], 1);
    }
}

__global__ void k_scatter_t(const int64_t* row_ptr, const int32_t* col, int64_t m, int64_t n,
                            const int64_t* rpt, int* cursor, int32_t* colt, int32_t* perm) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
            int32_t j = col[p];
            if (j < 0 || j >= n) continue;
            int pos = atomicAdd(&cursor[j], 1);
            colt[rpt[j] + pos] = (int32_t)i;
            perm[rpt[j] + pos] = (int32_t)p;
        }
    }
}

__global__ void k_gather_vals(const double* val, const int32_t* perm, double* valt, int64_t nnz) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        valt[q] = val[perm[q]];
}

__global__ void k_max_seg(const int64_t* off, int64_t nseg, int* out) {
    int best = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nseg;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = off[k + 1] - off[k];
        int v = l > INT_MAX ? INT_MAX : (int)l;
        best = v > best ? v : best;
    }
    atomicMax(out, best);
}

static int grid_for(int64_t work, int threads) {
    int64_t g = ceil_div(work, threads);
    int64_t cap = (int64_t)device_sm_count() * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

int transpose_build(const csls_csr* A, Transpose& T, int* counts, int* cursor, int* err, cudaStream_t st,
                    int64_t* launches) {
    const int64_t n = A->n, m = A->m, nnz = A->nnz;
    CSLS_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)n, st));
    CSLS_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)n, st));
    if (nnz > 0) {
        k_col_count<<<grid_for(nnz, 256), 256, 0, st>>>(A->col, nnz, n, counts, err);
        CSLS_CUDA(cudaGetLastError());
    }
    CSLS_TRY(scan_counts(counts, T.row_ptr, n, st));
    if (nnz > 0) {
        k_scatter_t<<<grid_for(m * 32, 256), 256, 0, st>>>(A->row_ptr, A->col, m, n, T.row_ptr, cursor, T.col,
                                                            T.perm);
        CSLS_CUDA(cudaGetLastError());
    }
    // longest column decides which sort kernels run (one small device->host copy)
    CSLS_CUDA(cudaMemsetAsync(counts, 0, sizeof(int), st));
    k_max_seg<<<grid_for(n, 256), 256, 0, st>>>(T.row_ptr, n, counts);
    CSLS_CUDA(cudaGetLastError());
    int maxlen = 0;
    CSLS_CUDA(cudaMemcpyAsync(&maxlen, counts, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSLS_CUDA(cudaStreamSynchronize(st));
    CSLS_TRY(segmented_sort(T.col, T.perm, T.row_ptr, n, maxlen, st));
    CSLS_TRY(transpose_gather_values(A, T, st));
    if (launches) *launches += 7;
    return CSLS_OK;
}

int transpose_gather_values(const csls_csr* A, const Transpose& T, cudaStream_t st) {
    if (A->nnz == 0) return CSLS_OK;
    k_gather_vals<<<grid_for(A->nnz, 256), 256, 0, st>>>(A->val, T.perm, T.val, A->nnz);
    CSLS_CUDA(cudaGetLastError());
    return CSLS_OK;
}

}  // namespace csls

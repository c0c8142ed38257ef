// Runtime pieces of the C ABI: errors, the allocator hook, CSR upload + validation,
// and a device exclusive scan used by the index build.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace knn {

// ---------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

knn_status fail(knn_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------------
// allocator hook
// ---------------------------------------------------------------------------------
static std::mutex g_alloc_mu;
static knn_alloc_fn g_alloc = nullptr;
static knn_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

void* dev_alloc(size_t bytes, cudaStream_t stream) {
    knn_alloc_fn a;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
    }
    if (a) return a(bytes, (void*)stream, ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t stream) {
    if (!p) return;
    knn_free_fn f;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (f) {
        f(p, bytes, (void*)stream, ctx);
        return;
    }
    cudaFreeAsync(p, stream);
}

// ---------------------------------------------------------------------------------
// CSR validation kernels
// ---------------------------------------------------------------------------------
enum : uint32_t {
    BAD_INDPTR = 1u,
    BAD_DIM = 2u,
    BAD_ORDER = 4u,
    BAD_WEIGHT = 8u,
};

struct CsrCheck {
    uint32_t flags;
    int32_t max_nnz;
    uint32_t max_w_bits;                // float bits of the largest weight
    unsigned long long max_sum_bits;   // double bits of the largest row sum
    unsigned long long max_sq_bits;    // double bits of the largest sum of squared weights
};

__global__ void k_check_indptr(const int64_t* __restrict__ indptr, int64_t n, int64_t nnz,
                               CsrCheck* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > n) return;
    int64_t v = indptr[i];
    bool bad = v < 0 || v > nnz;
    if (i == 0 && v != 0) bad = true;
    if (i == n && v != nnz) bad = true;
    if (i < n && indptr[i + 1] < v) bad = true;
    if (bad) atomicOr(&out->flags, BAD_INDPTR);
}

template <class W>
__device__ inline bool weight_ok(W w);
template <>
__device__ inline bool weight_ok<uint8_t>(uint8_t w) { return w != 0; }
template <>
__device__ inline bool weight_ok<float>(float w) { return w > 0.0f && isfinite(w); }

// one warp per row
template <class W>
__global__ void k_check_rows(const int64_t* __restrict__ indptr, const int32_t* __restrict__ idx,
                             const W* __restrict__ val, int64_t n, int32_t dim, CsrCheck* out) {
    int lane = threadIdx.x & 31;
    int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (; row < n; row += nwarps) {
        int64_t a = indptr[row], b = indptr[row + 1];
        uint32_t flags = 0;
        float wmax = 0.0f;
        double sum = 0.0, sq = 0.0;
        for (int64_t j = a + lane; j < b; j += 32) {
            int32_t d = idx[j];
            if (d < 0 || d >= dim) flags |= BAD_DIM;
            if (j > a && idx[j - 1] >= d) flags |= BAD_ORDER;
            W w = val[j];
            if (!weight_ok<W>(w)) flags |= BAD_WEIGHT;
            float wf = (float)w;
            if (wf > wmax) wmax = wf;
            sum += (double)wf;
            sq += (double)wf * (double)wf;
        }
        for (int o = 16; o > 0; o >>= 1) {
            flags |= __shfl_xor_sync(0xffffffffu, flags, o);
            wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
        }
        if (lane == 0) {
            if (flags) atomicOr(&out->flags, flags);
            atomicMax(&out->max_nnz, (int32_t)(b - a));
            if (wmax == wmax && wmax > 0.0f) atomicMax(&out->max_w_bits, __float_as_uint(wmax));
            if (sum > 0.0 && sum < 1e300)
                atomicMax(&out->max_sum_bits, (unsigned long long)__double_as_longlong(sum));
            if (sq > 0.0 && sq < 1e300)
                atomicMax(&out->max_sq_bits, (unsigned long long)__double_as_longlong(sq));
        }
    }
}

knn_status prepare_csr(const knn_csr* in, cudaStream_t stream, Buffers& bufs, bool validate,
                       bool need_stats, DevCSR* out) {
    if (!in) return fail(KNN_EINVAL, "CSR pointer is NULL");
    if (in->n_rows < 0) return fail(KNN_EINVAL, "n_rows < 0");
    if (in->dim < 1) return fail(KNN_EINVAL, "dim must be >= 1");
    if (in->dtype != KNN_U8 && in->dtype != KNN_F32) return fail(KNN_EINVAL, "unknown dtype");
    if (!in->indptr) return fail(KNN_EINVAL, "indptr is NULL");
    int64_t n = in->n_rows;
    int64_t first = 0, nnz = 0;
    if (in->on_device) {
        int64_t ends[2];
        KNN_CUDA_TRY(cudaMemcpyAsync(&ends[0], in->indptr, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
        KNN_CUDA_TRY(cudaMemcpyAsync(&ends[1], in->indptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
        KNN_CUDA_TRY(cudaStreamSynchronize(stream));
        first = ends[0];
        nnz = ends[1];
    } else {
        first = in->indptr[0];
        nnz = in->indptr[n];
    }
    if (first != 0) return fail(KNN_EINVAL, "indptr[0] must be 0");
    if (nnz < 0) return fail(KNN_EINVAL, "indptr[n_rows] < 0");
    if (nnz > (int64_t)INT32_MAX) return fail(KNN_EUNSUPPORTED, "more than 2^31-1 features");
    if (nnz > 0 && (!in->indices || !in->values)) return fail(KNN_EINVAL, "indices/values are NULL");
    size_t wsz = in->dtype == KNN_U8 ? 1 : 4;

    out->n_rows = n;
    out->nnz = nnz;
    out->dim = in->dim;
    out->dtype = in->dtype;
    if (in->on_device) {
        out->indptr = in->indptr;
        out->indices = in->indices;
        out->values = in->values;
    } else {
        int64_t* ip = nullptr;
        int32_t* ix = nullptr;
        uint8_t* vv = nullptr;
        KNN_TRY(bufs.get(&ip, (size_t)n + 1));
        KNN_TRY(bufs.get(&ix, (size_t)nnz));
        KNN_TRY(bufs.get(&vv, (size_t)nnz * wsz));
        KNN_CUDA_TRY(cudaMemcpyAsync(ip, in->indptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, stream));
        if (nnz) {
            KNN_CUDA_TRY(cudaMemcpyAsync(ix, in->indices, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, stream));
            KNN_CUDA_TRY(cudaMemcpyAsync(vv, in->values, wsz * nnz, cudaMemcpyHostToDevice, stream));
        }
        out->indptr = ip;
        out->indices = ix;
        out->values = vv;
    }
    if (!validate && !need_stats) return KNN_OK;

    CsrCheck* chk = nullptr;
    KNN_TRY(bufs.get(&chk, 1));
    KNN_CUDA_TRY(cudaMemsetAsync(chk, 0, sizeof(CsrCheck), stream));
    if (validate) {
        k_check_indptr<<<launch_blocks(n + 1, 256), 256, 0, stream>>>(out->indptr, n, nnz, chk);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
        CsrCheck h;
        KNN_CUDA_TRY(cudaMemcpyAsync(&h, chk, sizeof(h), cudaMemcpyDeviceToHost, stream));
        KNN_CUDA_TRY(cudaStreamSynchronize(stream));
        if (h.flags & BAD_INDPTR) return fail(KNN_EINVAL, "indptr is not a non-decreasing sequence from 0 to nnz");
    }
    if (n > 0) {
        int blocks = launch_blocks(n * 32, 256, 152 * 64);
        if (in->dtype == KNN_U8)
            k_check_rows<uint8_t><<<blocks, 256, 0, stream>>>(out->indptr, out->indices,
                                                             (const uint8_t*)out->values, n, in->dim, chk);
        else
            k_check_rows<float><<<blocks, 256, 0, stream>>>(out->indptr, out->indices,
                                                           (const float*)out->values, n, in->dim, chk);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    CsrCheck h;
    KNN_CUDA_TRY(cudaMemcpyAsync(&h, chk, sizeof(h), cudaMemcpyDeviceToHost, stream));
    KNN_CUDA_TRY(cudaStreamSynchronize(stream));
    if (validate) {
        if (h.flags & BAD_DIM) return fail(KNN_EINVAL, "a feature dimension is outside [0, dim)");
        if (h.flags & BAD_ORDER) return fail(KNN_EINVAL, "features of a row are not strictly ascending");
        if (h.flags & BAD_WEIGHT) return fail(KNN_EINVAL, "a weight is not > 0 (or not finite)");
    }
    out->max_row_nnz = h.max_nnz;
    float mw;
    memcpy(&mw, &h.max_w_bits, 4);
    out->max_w = mw;
    double ms;
    memcpy(&ms, &h.max_sum_bits, 8);
    out->max_row_sum = ms;
    double mq;
    memcpy(&mq, &h.max_sq_bits, 8);
    out->max_row_norm = std::sqrt(mq) * (1.0 + 1e-9);   // rounded up: a bound for every row
    return KNN_OK;
}

// Validation and row statistics of a CSR already on the device, with the check record
// in caller-provided device memory (at least 256 bytes, any contents) instead of an
// allocation.  Used by the allocation-free join; synchronises the stream.
knn_status check_device_csr_into(const knn_csr* in, void* scratch, bool validate, cudaStream_t stream,
                                 DevCSR* out) {
    if (!in) return fail(KNN_EINVAL, "CSR pointer is NULL");
    if (!in->on_device) return fail(KNN_EINVAL, "this call needs R in device memory (on_device = 1)");
    if (in->n_rows < 0) return fail(KNN_EINVAL, "n_rows < 0");
    if (in->dim < 1) return fail(KNN_EINVAL, "dim must be >= 1");
    if (in->dtype != KNN_U8 && in->dtype != KNN_F32) return fail(KNN_EINVAL, "unknown dtype");
    if (!in->indptr) return fail(KNN_EINVAL, "indptr is NULL");
    static_assert(sizeof(CsrCheck) <= 256, "check record must fit the scratch header");
    const int64_t n = in->n_rows;
    int64_t ends[2];
    KNN_CUDA_TRY(cudaMemcpyAsync(&ends[0], in->indptr, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    KNN_CUDA_TRY(cudaMemcpyAsync(&ends[1], in->indptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    KNN_CUDA_TRY(cudaStreamSynchronize(stream));
    if (ends[0] != 0) return fail(KNN_EINVAL, "indptr[0] must be 0");
    const int64_t nnz = ends[1];
    if (nnz < 0) return fail(KNN_EINVAL, "indptr[n_rows] < 0");
    if (nnz > (int64_t)INT32_MAX) return fail(KNN_EUNSUPPORTED, "more than 2^31-1 features");
    if (nnz > 0 && (!in->indices || !in->values)) return fail(KNN_EINVAL, "indices/values are NULL");
    out->n_rows = n;
    out->nnz = nnz;
    out->dim = in->dim;
    out->dtype = in->dtype;
    out->indptr = in->indptr;
    out->indices = in->indices;
    out->values = in->values;
    CsrCheck* chk = (CsrCheck*)scratch;
    KNN_CUDA_TRY(cudaMemsetAsync(chk, 0, sizeof(CsrCheck), stream));   // the record starts at zero
    CsrCheck h;
    if (validate) {
        k_check_indptr<<<launch_blocks(n + 1, 256), 256, 0, stream>>>(in->indptr, n, nnz, chk);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
        KNN_CUDA_TRY(cudaMemcpyAsync(&h, chk, sizeof(h), cudaMemcpyDeviceToHost, stream));
        KNN_CUDA_TRY(cudaStreamSynchronize(stream));
        if (h.flags & BAD_INDPTR) return fail(KNN_EINVAL, "indptr is not a non-decreasing sequence from 0 to nnz");
    }
    if (n > 0) {
        int blocks = launch_blocks(n * 32, 256, 152 * 64);
        if (in->dtype == KNN_U8)
            k_check_rows<uint8_t><<<blocks, 256, 0, stream>>>(in->indptr, in->indices, (const uint8_t*)in->values,
                                                             n, in->dim, chk);
        else
            k_check_rows<float><<<blocks, 256, 0, stream>>>(in->indptr, in->indices, (const float*)in->values, n,
                                                           in->dim, chk);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    KNN_CUDA_TRY(cudaMemcpyAsync(&h, chk, sizeof(h), cudaMemcpyDeviceToHost, stream));
    KNN_CUDA_TRY(cudaStreamSynchronize(stream));
    if (validate) {
        if (h.flags & BAD_DIM) return fail(KNN_EINVAL, "a feature dimension is outside [0, dim)");
        if (h.flags & BAD_ORDER) return fail(KNN_EINVAL, "features of a row are not strictly ascending");
        if (h.flags & BAD_WEIGHT) return fail(KNN_EINVAL, "a weight is not > 0 (or not finite)");
    }
    out->max_row_nnz = h.max_nnz;
    float mw;
    memcpy(&mw, &h.max_w_bits, 4);
    out->max_w = mw;
    double ms;
    memcpy(&ms, &h.max_sum_bits, 8);
    out->max_row_sum = ms;
    double mq;
    memcpy(&mq, &h.max_sq_bits, 8);
    out->max_row_norm = std::sqrt(mq) * (1.0 + 1e-9);   // rounded up: a bound for every row
    return KNN_OK;
}

// ---------------------------------------------------------------------------------
// exclusive scan of u32
// ---------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_scan_tile_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
    __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t t = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t j = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (j < n) t += in[j];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) s += warp_tot[w];
        sums[blockIdx.x] = s;
    }
}

// Each thread owns SCAN_ITEMS consecutive elements of the tile.
__global__ void k_scan_tile_apply(const uint32_t* in, uint32_t* out, int64_t n,
                                  const uint32_t* __restrict__ tile_off) {
    __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t j = base + i;
        v[i] = j < n ? in[j] : 0u;
        t += v[i];
    }
    // inclusive scan of thread totals across the block
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = t;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += warp_tot[w];
    uint32_t run = tile_off[blockIdx.x] + wpre + x - t;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t j = base + i;
        if (j < n) out[j] = run;
        run += v[i];
    }
    if (base <= n - 1 && base + SCAN_ITEMS >= n) out[n] = run;  // thread holding the last element
}

knn_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t stream,
                              Buffers& bufs) {
    if (n <= 0) {
        KNN_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint32_t), stream));
        return KNN_OK;
    }
    int64_t tiles = ceil_div(n, SCAN_TILE);
    uint32_t* sums = nullptr;
    uint32_t* offs = nullptr;
    KNN_TRY(bufs.get(&sums, (size_t)tiles));
    KNN_TRY(bufs.get(&offs, (size_t)tiles + 1));
    k_scan_tile_sums<<<(unsigned)tiles, SCAN_THREADS, 0, stream>>>(in, n, sums);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    if (tiles == 1) {
        KNN_CUDA_TRY(cudaMemsetAsync(offs, 0, sizeof(uint32_t), stream));
    } else {
        KNN_TRY(exclusive_scan_u32(sums, offs, tiles, stream, bufs));
    }
    k_scan_tile_apply<<<(unsigned)tiles, SCAN_THREADS, 0, stream>>>(in, out, n, offs);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    return KNN_OK;
}

}  // namespace knn

// ---------------------------------------------------------------------------------
// exported runtime entry points
// ---------------------------------------------------------------------------------
extern "C" knn_status knn_set_allocator(knn_alloc_fn alloc, knn_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return knn::fail(KNN_EINVAL, "allocator and release must both be set or both be NULL");
    std::lock_guard<std::mutex> lk(knn::g_alloc_mu);
    knn::g_alloc = alloc;
    knn::g_free = release;
    knn::g_alloc_ctx = ctx;
    return KNN_OK;
}

extern "C" const char* knn_last_error(void) { return knn::g_last_error.c_str(); }

extern "C" const char* knn_version(void) { return "knnjoin-gb300 0.1 (sm_103a)"; }

extern "C" int64_t knn_kernel_launch_count(void) { return knn::g_launches.load(); }

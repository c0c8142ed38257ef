// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/knn_join.h"

namespace knn {

// ---------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
knn_status fail(knn_status st, const char* fmt, ...);

// counts kernel launches (knn_kernel_launch_count)
void count_launch(int n = 1);

#define KNN_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::knn::fail(KNN_ECUDA, "%s failed: %s (%s:%d)", #expr,               \
                               cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

#define KNN_TRY(expr)                                                                   \
    do {                                                                                \
        knn_status s_ = (expr);                                                         \
        if (s_ != KNN_OK) return s_;                                                    \
    } while (0)

// ---------------------------------------------------------------------------------
// device memory through the installed allocator
// ---------------------------------------------------------------------------------
void* dev_alloc(size_t bytes, cudaStream_t stream);
void dev_free(void* p, size_t bytes, cudaStream_t stream);

// A set of buffers released together (RAII for temporaries of one call).
struct Buffers {
    cudaStream_t stream = nullptr;
    std::vector<std::pair<void*, size_t>> items;
    explicit Buffers(cudaStream_t s) : stream(s) {}
    Buffers(const Buffers&) = delete;
    Buffers& operator=(const Buffers&) = delete;
    template <class T>
    knn_status get(T** out, size_t count) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        void* p = dev_alloc(bytes, stream);
        if (!p) return fail(KNN_ENOMEM, "device allocation of %zu bytes failed", bytes);
        items.emplace_back(p, bytes);
        *out = static_cast<T*>(p);
        return KNN_OK;
    }
    size_t total() const {
        size_t t = 0;
        for (auto& it : items) t += it.second;
        return t;
    }
    void release() {
        for (auto& it : items) dev_free(it.first, it.second, stream);
        items.clear();
    }
    // hands ownership of every buffer to `other`
    void move_to(Buffers& other) {
        for (auto& it : items) other.items.push_back(it);
        items.clear();
    }
    ~Buffers() { release(); }
};

// ---------------------------------------------------------------------------------
// a CSR on the device (uploaded or borrowed) after validation
// ---------------------------------------------------------------------------------
struct DevCSR {
    int64_t n_rows = 0, nnz = 0;
    int32_t dim = 0;
    knn_dtype dtype = KNN_U8;
    const int64_t* indptr = nullptr;
    const int32_t* indices = nullptr;
    const void* values = nullptr;
    int32_t max_row_nnz = 0;
    double max_w = 0.0;        // largest weight
    double max_row_sum = 0.0;  // largest sum of a row's weights
    double max_row_norm = 0.0; // largest L2 norm of a row (rounded up)
};

// Uploads (if on host) and validates a CSR; buffers it allocates go to `bufs`.
// `need_stats` fills max_row_nnz / max_w / max_row_sum (synchronises the stream).
knn_status prepare_csr(const knn_csr* in, cudaStream_t stream, Buffers& bufs, bool validate,
                       bool need_stats, DevCSR* out);

// Same checks and statistics for a device CSR, with the check record placed in the
// given device scratch (>= 256 bytes) instead of an allocation.
knn_status check_device_csr_into(const knn_csr* in, void* scratch, bool validate, cudaStream_t stream,
                                 DevCSR* out);

// ---------------------------------------------------------------------------------
// the index (owned device buffers + layout parameters)
// ---------------------------------------------------------------------------------
}  // namespace knn

struct knn_index {
    int64_t n_rows = 0, nnz = 0, n_postings = 0;   // n_postings: nnz + list padding
    int32_t dim = 0, block_size = 0, n_blocks = 0, n_levels = 0, block_shift = 0;
    knn_dtype dtype = KNN_U8;
    int32_t max_row_nnz = 0;
    double max_w = 0.0, max_row_sum = 0.0, max_row_norm = 0.0;
    float levels[KNN_MAX_LEVELS] = {};  // ladder of bound thresholds, levels[0] == 0
    // device arrays
    uint32_t* binoff = nullptr;  // [n_blocks * dim * n_levels + 1] posting-bin offsets
    void* postings = nullptr;    // [n_postings] u32 (lid | w<<24) for u8; uint2 {lid, w} for f32;
                                 // every (S block, d) list padded to whole 16-byte chunks
    int64_t* s_indptr = nullptr; // [n_rows + 1]
    int32_t* sp_d = nullptr;     // [nnz] features of each s in cut order (dimension)
    void* sp_w = nullptr;        // [nnz] weights in the same order (u8 or f32)
    uint16_t* n_unidx = nullptr; // [n_levels * n_rows] unindexed prefix length per level
    uint32_t* ubound = nullptr;  // [n_levels * n_rows] weight sum of that prefix (u32 or f32 bits)
    cudaStream_t stream = nullptr;
    knn::Buffers* bufs = nullptr;
    // after knn_index_to_host: the arrays above live in pinned, mapped host memory
    std::vector<void*> host_arrays;
    size_t host_bytes = 0;
};

namespace knn {

// ---------------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------------
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int launch_blocks(int64_t work, int per_block, int64_t cap = (1LL << 31) - 1) {
    int64_t b = ceil_div(work, per_block);
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// Predicted k-th scores (device float[n_rows]) of a device CSR with the model.
knn_status model_predict_tau(const knn_model* md, const DevCSR& r, float tau_scale, float* tau, cudaStream_t s,
                             Buffers& tmp);
// The model's calibrated prediction multiplier (1 until knn_threshold_model_calibrate).
float model_tau_scale(const knn_model* md);
// KNN_ETIMEOUT if a model GEMM gave up a bounded wait since the last check (the caller
// has synchronised the stream), else KNN_OK.
knn_status model_check();

// Exclusive scan of u32 counts (n elements) into out[0..n], out[n] = total.
// The total must stay below 2^32 (checked by the caller).  Works in place.
knn_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t stream,
                              Buffers& bufs);

}  // namespace knn

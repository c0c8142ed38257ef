// Learned-threshold join with verify-and-fallback.
//
// 1. tau = exp(MLP(sketch(r))) x the model's calibrated multiplier per query row (or
//    caller-given thresholds);
// 2. knn_join with tau as each row's inclusive start threshold: a row keeps only the s
//    with score >= tau, and the Section 4.4 cut starts from tau instead of 0;
// 3. a row that ends with k entries has its exact top-k (every s with score >= tau was
//    surfaced, so the k best of them are the k best overall); the rows that found fewer
//    than k are gathered on the device and joined again with the plain threshold, and
//    their results are scattered back.
// The result is therefore always the exact top-k; the plain join is both the fallback
// and the check of the prediction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace knn {

__global__ void k_fallback_rows(const int32_t* __restrict__ n_found, int64_t n, int32_t k, int64_t* __restrict__ list,
                                unsigned long long* __restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && n_found[i] < k) list[atomicAdd(count, 1ull)] = i;
}

__global__ void k_row_lengths(const int64_t* __restrict__ indptr, const int64_t* __restrict__ list, int64_t m,
                              uint32_t* __restrict__ len) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < m) len[j] = (uint32_t)(indptr[list[j] + 1] - indptr[list[j]]);
}

__global__ void k_u32_to_i64(const uint32_t* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int64_t)in[i];
}

template <class W>
__global__ void k_gather_rows(const int64_t* __restrict__ indptr, const int32_t* __restrict__ idx,
                              const W* __restrict__ val, const int64_t* __restrict__ list, int64_t m,
                              const int64_t* __restrict__ sub_indptr, int32_t* __restrict__ sub_idx,
                              W* __restrict__ sub_val) {
    int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (j >= m) return;
    int64_t a = indptr[list[j]], n = indptr[list[j] + 1] - a, o = sub_indptr[j];
    for (int64_t q = lane; q < n; q += 32) {
        sub_idx[o + q] = idx[a + q];
        sub_val[o + q] = val[a + q];
    }
}

__global__ void k_scatter_rows(const int64_t* __restrict__ list, int64_t m, int32_t k, const int32_t* __restrict__ sub_ids,
                               const uint32_t* __restrict__ sub_sc, int32_t* __restrict__ ids, uint32_t* __restrict__ sc) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= m * k) return;
    int64_t j = t / k, q = t % k;
    ids[list[j] * k + q] = sub_ids[t];
    sc[list[j] * k + q] = sub_sc[t];
}

}  // namespace knn

using namespace knn;

extern "C" knn_status knn_join_learned(const knn_index* ix, const knn_model* md, const knn_csr* R, int32_t k,
                                       const knn_learned_opts* lopts, int32_t* out_ids, void* out_scores,
                                       knn_learned_stats* stats, void* stream_) {
    cudaStream_t s = (cudaStream_t)stream_;
    if (!ix || !R) return fail(KNN_EINVAL, "NULL argument");
    knn_learned_opts o = {};
    if (lopts) o = *lopts;
    if (!md && !o.tau) return fail(KNN_EINVAL, "a model or caller thresholds (tau) are needed");
    if (k < 1) return fail(KNN_EINVAL, "k must be >= 1");
    if (k > KNN_MAX_K) return fail(KNN_EUNSUPPORTED, "k > %d", KNN_MAX_K);
    if (R->dim != ix->dim || R->dtype != ix->dtype) return fail(KNN_EINVAL, "R does not match the index");
    Buffers tmp(s);
    DevCSR r;
    KNN_TRY(prepare_csr(R, s, tmp, !o.join.skip_validation, false, &r));
    if (stats) memset(stats, 0, sizeof(*stats));
    if (r.n_rows == 0) return KNN_OK;
    if (!out_ids || !out_scores) return fail(KNN_EINVAL, "outputs are NULL");
    const knn_csr Rd = {r.n_rows, r.dim, r.dtype, r.indptr, r.indices, r.values, 1};

    int32_t* d_ids = out_ids;
    uint32_t* d_sc = (uint32_t*)out_scores;
    if (o.join.outputs_on_host) {
        KNN_TRY(tmp.get(&d_ids, (size_t)r.n_rows * k));
        KNN_TRY(tmp.get(&d_sc, (size_t)r.n_rows * k));
    }
    // 1. start thresholds
    float* tau = (float*)o.tau;
    if (!tau) {
        KNN_TRY(tmp.get(&tau, (size_t)r.n_rows));
        KNN_TRY(model_predict_tau(md, r, o.tau_scale > 0.0f ? o.tau_scale : model_tau_scale(md), tau, s, tmp));
        KNN_CUDA_TRY(cudaStreamSynchronize(s));
        KNN_TRY(model_check());
    }
    // 2. the join from those thresholds
    int32_t* found = nullptr;
    KNN_TRY(tmp.get(&found, (size_t)r.n_rows));
    knn_join_opts jo = o.join;
    jo.init_threshold = tau;
    jo.n_found = found;
    jo.outputs_on_host = 0;
    jo.skip_validation = 1;
    KNN_TRY(knn_join(ix, &Rd, k, &jo, d_ids, d_sc, s));
    // 3. verify: rows with fewer than k entries are joined again without a threshold
    int64_t* list = nullptr;
    unsigned long long* cnt = nullptr;
    KNN_TRY(tmp.get(&list, (size_t)r.n_rows));
    KNN_TRY(tmp.get(&cnt, 1));
    KNN_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    k_fallback_rows<<<launch_blocks(r.n_rows, 256), 256, 0, s>>>(found, r.n_rows, k, list, cnt);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    unsigned long long h_cnt = 0;
    KNN_CUDA_TRY(cudaMemcpyAsync(&h_cnt, cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, s));
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t m = (int64_t)h_cnt;
    if (m > 0) {
        uint32_t* len = nullptr;
        int64_t* sub_indptr = nullptr;
        KNN_TRY(tmp.get(&len, (size_t)m + 1));
        KNN_TRY(tmp.get(&sub_indptr, (size_t)m + 1));
        k_row_lengths<<<launch_blocks(m, 256), 256, 0, s>>>(r.indptr, list, m, len);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
        KNN_TRY(exclusive_scan_u32(len, len, m, s, tmp));
        k_u32_to_i64<<<launch_blocks(m + 1, 256), 256, 0, s>>>(len, m + 1, sub_indptr);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
        int64_t sub_nnz = 0;
        KNN_CUDA_TRY(cudaMemcpyAsync(&sub_nnz, sub_indptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KNN_CUDA_TRY(cudaStreamSynchronize(s));
        int32_t* sub_idx = nullptr;
        uint8_t* sub_val = nullptr;
        const size_t wsz = r.dtype == KNN_U8 ? 1 : 4;
        KNN_TRY(tmp.get(&sub_idx, (size_t)sub_nnz));
        KNN_TRY(tmp.get(&sub_val, (size_t)sub_nnz * wsz));
        if (r.dtype == KNN_U8)
            k_gather_rows<uint8_t><<<launch_blocks(m * 32, 256), 256, 0, s>>>(
                r.indptr, r.indices, (const uint8_t*)r.values, list, m, sub_indptr, sub_idx, sub_val);
        else
            k_gather_rows<float><<<launch_blocks(m * 32, 256), 256, 0, s>>>(
                r.indptr, r.indices, (const float*)r.values, list, m, sub_indptr, sub_idx, (float*)sub_val);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
        const knn_csr Rs = {m, r.dim, r.dtype, sub_indptr, sub_idx, sub_val, 1};
        int32_t* s_ids = nullptr;
        uint32_t* s_sc = nullptr;
        KNN_TRY(tmp.get(&s_ids, (size_t)m * k));
        KNN_TRY(tmp.get(&s_sc, (size_t)m * k));
        knn_join_opts po = o.join;
        po.init_threshold = nullptr;
        po.n_found = nullptr;
        po.outputs_on_host = 0;
        po.skip_validation = 1;
        KNN_TRY(knn_join(ix, &Rs, k, &po, s_ids, s_sc, s));
        k_scatter_rows<<<launch_blocks(m * k, 256), 256, 0, s>>>(list, m, k, s_ids, s_sc, d_ids, d_sc);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    if (o.join.outputs_on_host) {
        KNN_CUDA_TRY(cudaMemcpyAsync(out_ids, d_ids, sizeof(int32_t) * r.n_rows * k, cudaMemcpyDeviceToHost, s));
        KNN_CUDA_TRY(cudaMemcpyAsync(out_scores, d_sc, sizeof(uint32_t) * r.n_rows * k, cudaMemcpyDeviceToHost, s));
    }
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    if (stats) {
        stats->rows = r.n_rows;
        stats->fallback_rows = m;
    }
    return KNN_OK;
}

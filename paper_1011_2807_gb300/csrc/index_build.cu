// Index build: the inverted lists of S (Section 4.3, Create_Inverted_List_IIB of
// Algorithm 3), split into S blocks, with the threshold cut of Section 4.4
// (Create_Inverted_List_IIIB of Algorithm 4) precomputed for a ladder of thresholds.
//
// Algorithm 4 walks the features of s in a dimension order, adds maxWeight_d * w to a
// bound t, and indexes the features from the one where t exceeds MinPruneScore on.
// The index is built before any R is known, so this build
//   * fixes one dimension order pi for all queries (descending document frequency in
//     S, ties by ascending d; Theorem 1 holds for any order),
//   * keeps the R-dependent factor out of the bound: with M >= every weight of the
//     query, t(j) <= M * tS(j), where tS(j) is the sum of s's weights over its first
//     j+1 features in pi order,
//   * precomputes, for each level value L_l of a ladder (L_0 = 0 < L_1 < ...), which
//     features a query whose threshold theta satisfies M * L_l < theta may leave
//     unindexed: exactly those with tS(j) <= L_l (a prefix of s in pi order).
// A posting's bucket is the highest level at which it is still indexed,
// max{l : tS(j) > L_l}.  Each (S block, d) list is stored bucket-descending, so the
// part of the list indexed at level l is a prefix, and binoff gives its end.
//
// Layout in HBM (all device arrays owned by the index):
//   binoff   u32 [n_blocks * dim * n_levels + 1]: bin (b, d, n_levels-1-bucket) start
//   postings u32 (lid | w << 24) for uint8, uint2 {lid, float bits} for float32; each
//            (S block, d) list padded to whole 16-byte chunks with (lid 0, weight 0)
//   s_indptr / sp_d / sp_w: S in CSR with each row's features in pi order
//   n_unidx  u16 [n_levels][|S|]: unindexed prefix length of s at level l
//   ubound   u32 [n_levels][|S|]: tS of that prefix (u32 for uint8, float bits rounded up)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace knn {

__global__ void k_df(const int32_t* __restrict__ idx, int64_t nnz, uint32_t* __restrict__ df) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < nnz; i += stride) atomicAdd(&df[idx[i]], 1u);
}

// rank[d] = number of dimensions ahead of d in (df desc, d asc) order
__global__ void k_rank(const uint32_t* __restrict__ df, int32_t dim, int32_t* __restrict__ rank) {
    __shared__ uint32_t tile[1024];
    int32_t d = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t f = d < dim ? df[d] : 0u;
    int32_t r = 0;
    for (int32_t t0 = 0; t0 < dim; t0 += 1024) {
        __syncthreads();
        for (int32_t i = threadIdx.x; i < 1024; i += blockDim.x)
            tile[i] = t0 + i < dim ? df[t0 + i] : 0u;
        __syncthreads();
        int32_t lim = min(1024, dim - t0);
        for (int32_t i = 0; i < lim; i++) {
            uint32_t g = tile[i];
            int32_t e = t0 + i;
            r += (g > f) || (g == f && e < d);
        }
    }
    if (d < dim) rank[d] = r;
}

template <class W>
struct WTraits;
template <>
struct WTraits<uint8_t> {
    using Sum = uint32_t;
    __device__ static uint32_t bound_bits(uint32_t t) { return t; }
};
template <>
struct WTraits<float> {
    using Sum = double;
    // float not below the double value (the bound must not shrink)
    __device__ static uint32_t bound_bits(double t) {
        float f = __double2float_ru(t);
        return __float_as_uint(f);
    }
};

struct CutParams {
    int64_t n_rows;
    int32_t n_levels;
    float levels[KNN_MAX_LEVELS];
};

// one warp per s: pi-order the features, prefix sums tS, buckets, per-level prefix data
template <class W>
__global__ void k_cut_order(const int64_t* __restrict__ indptr, const int32_t* __restrict__ idx,
                            const W* __restrict__ val, const int32_t* __restrict__ rank,
                            CutParams p, int32_t* __restrict__ sp_d, W* __restrict__ sp_w,
                            uint8_t* __restrict__ bucket, uint16_t* __restrict__ n_unidx,
                            uint32_t* __restrict__ ubound) {
    using Sum = typename WTraits<W>::Sum;
    const int lane = threadIdx.x & 31;
    int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (; s < p.n_rows; s += nwarps) {
        const int64_t a = indptr[s], b = indptr[s + 1];
        const int32_t n = (int32_t)(b - a);
        // position of feature j in pi order = number of features of s ranked before it
        for (int32_t j = lane; j < n; j += 32) {
            int32_t rj = rank[idx[a + j]];
            int32_t pos = 0;
            for (int32_t q = 0; q < n; q++) pos += rank[idx[a + q]] < rj;
            sp_d[a + pos] = idx[a + j];
            sp_w[a + pos] = val[a + j];
        }
        __threadfence_block();
        __syncwarp();
        Sum carry = 0;
        uint32_t my_n = 0;      // lane l keeps level l's unindexed count
        Sum my_u = 0;           // ... and its prefix sum
        for (int32_t c = 0; c < n; c += 32) {
            int32_t j = c + lane;
            bool valid = j < n;
            Sum x = valid ? (Sum)sp_w[a + j] : (Sum)0;
            // inclusive warp scan
            for (int o = 1; o < 32; o <<= 1) {
                Sum y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            Sum ts = carry + x;
            carry = __shfl_sync(0xffffffffu, ts, 31);
            int bk = 0;
            for (int l = 1; l < p.n_levels; l++) {
                bool un = valid && (double)ts <= (double)p.levels[l];
                bk += (valid && !un) ? 1 : 0;
                unsigned m = __ballot_sync(0xffffffffu, un);
                int hi = m ? 31 - __clz(m) : 0;
                Sum top = __shfl_sync(0xffffffffu, ts, hi);
                if (lane == l && m) {
                    my_n += __popc(m);
                    my_u = top;
                }
            }
            if (valid) bucket[a + j] = (uint8_t)bk;
        }
        if (lane < p.n_levels) {
            n_unidx[(int64_t)lane * p.n_rows + s] = (uint16_t)min(my_n, 65535u);
            ubound[(int64_t)lane * p.n_rows + s] = WTraits<W>::bound_bits(my_u);
        }
    }
}

struct BinParams {
    int64_t n_rows;
    int32_t dim, n_levels, block_shift;
};

__device__ inline size_t bin_of(const BinParams& p, int64_t s, int32_t d, int bk) {
    size_t blk = (size_t)(s >> p.block_shift);
    return ((blk * (size_t)p.dim + (size_t)d) * (size_t)p.n_levels) + (size_t)(p.n_levels - 1 - bk);
}

__global__ void k_bin_count(const int64_t* __restrict__ indptr, const int32_t* __restrict__ sp_d,
                            const uint8_t* __restrict__ bucket, BinParams p, uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (; s < p.n_rows; s += nwarps) {
        for (int64_t j = indptr[s] + lane; j < indptr[s + 1]; j += 32)
            atomicAdd(&cnt[bin_of(p, s, sp_d[j], bucket[j])], 1u);
    }
}

// Pads every (S block, d) list to a whole number of 16-byte chunks: the padding is
// added to the list's last bin (bucket 0), so lists start on chunk boundaries and the
// whole-list prefix ends on one.  Padding postings are zero (local id 0, weight 0).
__global__ void k_pad_lists(uint32_t* __restrict__ cnt, int64_t n_lists, int32_t n_levels, uint32_t per_chunk) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_lists) return;
    uint32_t* c = cnt + i * n_levels;
    uint32_t t = 0;
    for (int l = 0; l < n_levels; l++) t += c[l];
    c[n_levels - 1] += (per_chunk - t % per_chunk) % per_chunk;
}

template <class W>
__global__ void k_scatter(const int64_t* __restrict__ indptr, const int32_t* __restrict__ sp_d,
                          const W* __restrict__ sp_w, const uint8_t* __restrict__ bucket, BinParams p,
                          uint32_t* __restrict__ cursor, void* __restrict__ postings) {
    const int lane = threadIdx.x & 31;
    int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    const uint32_t lid_mask = (1u << p.block_shift) - 1u;
    for (; s < p.n_rows; s += nwarps) {
        uint32_t lid = (uint32_t)s & lid_mask;
        for (int64_t j = indptr[s] + lane; j < indptr[s + 1]; j += 32) {
            uint32_t pos = atomicAdd(&cursor[bin_of(p, s, sp_d[j], bucket[j])], 1u);
            W w = sp_w[j];
            if constexpr (sizeof(W) == 1) {
                ((uint32_t*)postings)[pos] = lid | ((uint32_t)w << 24);
            } else {
                ((uint2*)postings)[pos] = make_uint2(lid, __float_as_uint((float)w));
            }
        }
    }
}

// Orders the postings of every bin so that the join's add instructions hit different
// shared-memory banks (local id mod 32) where the bin's contents allow.  The join adds
// slot j of 32 consecutive chunks of its concatenated lists with one instruction, and
// where a list sits in that concatenation depends on the query, so any two chunks of a
// list fewer than 32 apart may share an instruction -- the nearer, the likelier.  Chunk
// by chunk and slot by slot, the posting placed is the first of the bin's next
// (up to) 32 chunks' worth whose bank has the least weight among the banks at the same
// slot of the previous W - 1 chunks, a bank at distance t weighing W - t.  Padding
// postings (weight 0, added nowhere that matters) take the least-weighted bank as their
// local id.  Only the order inside a bin changes, so every level's prefix keeps the
// same postings.  One thread per (S block, d) list.
template <class Post, int V>
__device__ __forceinline__ uint32_t post_bank(Post e);
template <>
__device__ __forceinline__ uint32_t post_bank<uint32_t, 4>(uint32_t e) { return e & 31u; }
template <>
__device__ __forceinline__ uint32_t post_bank<uint2, 2>(uint2 e) { return e.x & 31u; }
template <class Post>
__device__ __forceinline__ bool post_is_pad(Post e);
template <>
__device__ __forceinline__ bool post_is_pad<uint32_t>(uint32_t e) { return (e >> 24) == 0u; }
template <>
__device__ __forceinline__ bool post_is_pad<uint2>(uint2 e) { return e.y == 0u; }
__device__ __forceinline__ uint32_t with_lid(uint32_t e, uint32_t lid) { return (e & 0xFFFF0000u) | lid; }
__device__ __forceinline__ uint2 with_lid(uint2 e, uint32_t lid) { return make_uint2(lid, e.y); }

template <class Post, int V>
__global__ void k_arrange(const uint32_t* __restrict__ binoff, int64_t n_lists, int32_t n_levels,
                          Post* __restrict__ post) {
    constexpr int POOL = 32 * V;   // postings considered at once
    constexpr int W = 24;          // chunks whose banks weigh on the next pick
    const int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (li >= n_lists) return;
    const uint32_t* bo = binoff + li * n_levels;
    const uint32_t L0 = bo[0];
    uint8_t ring[V][W];            // ring[j][c % W]: bank at slot j of chunk c (0xFF: none yet)
#pragma unroll
    for (int j = 0; j < V; j++)
        for (int t = 0; t < W; t++) ring[j][t] = 0xFFu;
    Post buf[POOL];
    for (int t = 0; t < n_levels; t++) {
        const uint32_t x = bo[t], y = bo[t + 1];
        for (uint32_t a = x; a < y; a += POOL) {
            const uint32_t b = min(y, a + (uint32_t)POOL);
            int rem = (int)(b - a);
            for (int i = 0; i < rem; i++) buf[i] = post[a + i];
            for (uint32_t q = a; q < b; q++) {
                const int j = (int)(q & (V - 1));
                const uint32_t c = (q - L0) / V;   // chunk of the list (lists start on chunks)
                uint32_t cost[32];
#pragma unroll
                for (int k = 0; k < 32; k++) cost[k] = 0u;
                for (int e = 1; e < W; e++) {
                    if (c < (uint32_t)e) break;
                    const uint32_t bk = ring[j][(c - e) % W];
                    if (bk != 0xFFu) cost[bk] += (uint32_t)(W - e);
                }
                int pick = 0;
                uint32_t best = 0xFFFFFFFFu;
                for (int i = 0; i < rem; i++) {
                    const uint32_t ci = post_is_pad(buf[i]) ? 0u : cost[post_bank<Post, V>(buf[i])];
                    if (ci < best) {
                        best = ci;
                        pick = i;
                        if (ci == 0u) break;
                    }
                }
                Post e = buf[pick];
                buf[pick] = buf[rem - 1];
                rem--;
                if (post_is_pad(e)) {   // padding: the least-weighted bank as its local id
                    uint32_t bk = 0, bc = cost[0];
                    for (uint32_t k = 1; k < 32; k++)
                        if (cost[k] < bc) {
                            bc = cost[k];
                            bk = k;
                        }
                    e = with_lid(e, bk);
                }
                post[q] = e;
                ring[j][c % W] = (uint8_t)post_bank<Post, V>(e);
            }
        }
    }
}

static int ilog2(int64_t v) {
    int r = 0;
    while ((int64_t(1) << r) < v) r++;
    return r;
}

}  // namespace knn

using namespace knn;

extern "C" knn_status knn_join_build_index(const knn_csr* S, const knn_build_opts* opts, void* stream_,
                                           knn_index** out) {
    if (!out) return fail(KNN_EINVAL, "out is NULL");
    *out = nullptr;
    cudaStream_t stream = (cudaStream_t)stream_;
    knn_build_opts o = {};
    if (opts) o = *opts;
    int32_t nl = o.n_levels == 0 ? 16 : o.n_levels;
    if (nl < 1 || nl > KNN_MAX_LEVELS) return fail(KNN_EINVAL, "n_levels must be in [1, %d]", KNN_MAX_LEVELS);
    if (o.block_size != 0) {
        if (o.block_size < 256 || o.block_size > KNN_MAX_BLOCK || (o.block_size & (o.block_size - 1)))
            return fail(KNN_EINVAL, "block_size must be a power of two in [256, %d]", KNN_MAX_BLOCK);
    }

    Buffers tmp(stream);
    DevCSR s;
    KNN_TRY(prepare_csr(S, stream, tmp, true, true, &s));
    if (s.max_row_nnz > 65535) return fail(KNN_EUNSUPPORTED, "an S row has more than 65535 features");

    knn_index* ix = new knn_index();
    ix->bufs = new Buffers(stream);
    ix->stream = stream;
    auto bail = [&](knn_status st) {
        ix->bufs->release();
        delete ix->bufs;
        delete ix;
        return st;
    };
    ix->n_rows = s.n_rows;
    ix->nnz = s.nnz;
    ix->dim = s.dim;
    ix->dtype = s.dtype;
    ix->max_row_nnz = s.max_row_nnz;
    ix->max_w = s.max_w;
    ix->max_row_sum = s.max_row_sum;
    ix->max_row_norm = s.max_row_norm;
    int32_t bs = o.block_size;
    if (bs == 0) {
        bs = 16384;
        int64_t need = std::max<int64_t>(256, int64_t(1) << ilog2(std::max<int64_t>(1, s.n_rows)));
        if (need < bs) bs = (int32_t)need;
    }
    ix->block_size = bs;
    ix->block_shift = ilog2(bs);
    ix->n_blocks = (int32_t)std::max<int64_t>(1, ceil_div(s.n_rows, bs));
    ix->n_levels = nl;
    // ladder: L_0 = 0; L_l = (tmax / 2) * 2^(-(nl - 1 - l) / 2) for l >= 1
    double tmax = s.max_row_sum > 0 ? s.max_row_sum : 1.0;
    ix->levels[0] = 0.0f;
    for (int l = 1; l < nl; l++) ix->levels[l] = (float)(0.5 * tmax * std::pow(2.0, -0.5 * (nl - 1 - l)));

    const size_t wsz = s.dtype == KNN_U8 ? 1 : 4;
    const size_t psz = s.dtype == KNN_U8 ? 4 : 8;
    const size_t nbins = (size_t)ix->n_blocks * (size_t)s.dim * (size_t)nl;
    {   // posting offsets are 32-bit: nnz plus at most (16 / psz - 1) padding postings per list
        const uint64_t lists = (uint64_t)ix->n_blocks * (uint64_t)s.dim;
        const uint64_t pad = (uint64_t)(16 / psz - 1) * std::min<uint64_t>(lists, (uint64_t)s.nnz);
        if ((uint64_t)s.nnz + pad > 0xffffffffull)
            return bail(fail(KNN_EUNSUPPORTED, "S has too many nonzeros for 32-bit posting offsets"));
    }
    uint8_t* spw = nullptr;
    uint8_t* post = nullptr;
    knn_status st;
    if ((st = ix->bufs->get(&ix->binoff, nbins + 1)) != KNN_OK) return bail(st);
    if ((st = ix->bufs->get(&ix->s_indptr, (size_t)s.n_rows + 1)) != KNN_OK) return bail(st);
    if ((st = ix->bufs->get(&ix->sp_d, (size_t)s.nnz)) != KNN_OK) return bail(st);
    if ((st = ix->bufs->get(&spw, (size_t)s.nnz * wsz)) != KNN_OK) return bail(st);
    if ((st = ix->bufs->get(&ix->n_unidx, (size_t)nl * s.n_rows)) != KNN_OK) return bail(st);
    if ((st = ix->bufs->get(&ix->ubound, (size_t)nl * s.n_rows)) != KNN_OK) return bail(st);
    ix->sp_w = spw;

    uint32_t* df = nullptr;
    int32_t* rank = nullptr;
    uint8_t* bucket = nullptr;
    uint32_t* cursor = nullptr;
    if ((st = tmp.get(&df, (size_t)s.dim)) != KNN_OK) return bail(st);
    if ((st = tmp.get(&rank, (size_t)s.dim)) != KNN_OK) return bail(st);
    if ((st = tmp.get(&bucket, (size_t)s.nnz)) != KNN_OK) return bail(st);
    if ((st = tmp.get(&cursor, nbins + 1)) != KNN_OK) return bail(st);

#define BAIL_CUDA(expr)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bail(fail(KNN_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)));             \
    } while (0)

    BAIL_CUDA(cudaMemcpyAsync(ix->s_indptr, s.indptr, sizeof(int64_t) * (s.n_rows + 1),
                              cudaMemcpyDeviceToDevice, stream));
    BAIL_CUDA(cudaMemsetAsync(df, 0, sizeof(uint32_t) * s.dim, stream));
    k_df<<<launch_blocks(s.nnz, 256, 152 * 32), 256, 0, stream>>>(s.indices, s.nnz, df);
    BAIL_CUDA(cudaGetLastError());
    count_launch();
    k_rank<<<launch_blocks(s.dim, 256), 256, 0, stream>>>(df, s.dim, rank);
    BAIL_CUDA(cudaGetLastError());
    count_launch();

    CutParams cp;
    cp.n_rows = s.n_rows;
    cp.n_levels = nl;
    memcpy(cp.levels, ix->levels, sizeof(cp.levels));
    int wblocks = launch_blocks(std::max<int64_t>(1, s.n_rows) * 32, 256, 152 * 64);
    if (s.n_rows) {
        if (s.dtype == KNN_U8)
            k_cut_order<uint8_t><<<wblocks, 256, 0, stream>>>(s.indptr, s.indices, (const uint8_t*)s.values,
                                                             rank, cp, ix->sp_d, (uint8_t*)spw, bucket,
                                                             ix->n_unidx, ix->ubound);
        else
            k_cut_order<float><<<wblocks, 256, 0, stream>>>(s.indptr, s.indices, (const float*)s.values,
                                                           rank, cp, ix->sp_d, (float*)spw, bucket,
                                                           ix->n_unidx, ix->ubound);
        BAIL_CUDA(cudaGetLastError());
        count_launch();
    }
    BinParams bp;
    bp.n_rows = s.n_rows;
    bp.dim = s.dim;
    bp.n_levels = nl;
    bp.block_shift = ix->block_shift;
    BAIL_CUDA(cudaMemsetAsync(ix->binoff, 0, sizeof(uint32_t) * (nbins + 1), stream));
    if (s.n_rows) {
        k_bin_count<<<wblocks, 256, 0, stream>>>(ix->s_indptr, ix->sp_d, bucket, bp, ix->binoff);
        BAIL_CUDA(cudaGetLastError());
        count_launch();
    }
    {
        const int64_t n_lists = (int64_t)ix->n_blocks * s.dim;
        k_pad_lists<<<launch_blocks(n_lists, 256), 256, 0, stream>>>(ix->binoff, n_lists, nl, (uint32_t)(16 / psz));
        BAIL_CUDA(cudaGetLastError());
        count_launch();
    }
    if ((st = exclusive_scan_u32(ix->binoff, ix->binoff, (int64_t)nbins, stream, tmp)) != KNN_OK) return bail(st);
    BAIL_CUDA(cudaMemcpyAsync(cursor, ix->binoff, sizeof(uint32_t) * (nbins + 1), cudaMemcpyDeviceToDevice, stream));
    uint32_t n_post = 0;
    BAIL_CUDA(cudaMemcpyAsync(&n_post, ix->binoff + nbins, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    BAIL_CUDA(cudaStreamSynchronize(stream));
    ix->n_postings = n_post;
    if ((st = ix->bufs->get(&post, (size_t)n_post * psz)) != KNN_OK) return bail(st);
    BAIL_CUDA(cudaMemsetAsync(post, 0, (size_t)n_post * psz, stream));   // padding postings: id 0, weight 0
    ix->postings = post;
    if (s.n_rows) {
        if (s.dtype == KNN_U8)
            k_scatter<uint8_t><<<wblocks, 256, 0, stream>>>(ix->s_indptr, ix->sp_d, (const uint8_t*)spw, bucket,
                                                           bp, cursor, post);
        else
            k_scatter<float><<<wblocks, 256, 0, stream>>>(ix->s_indptr, ix->sp_d, (const float*)spw, bucket,
                                                         bp, cursor, post);
        BAIL_CUDA(cudaGetLastError());
        count_launch();
        const int64_t n_lists = (int64_t)ix->n_blocks * s.dim;
        if (s.dtype == KNN_U8)
            k_arrange<uint32_t, 4><<<launch_blocks(n_lists, 128), 128, 0, stream>>>(ix->binoff, n_lists, nl,
                                                                                     (uint32_t*)post);
        else
            k_arrange<uint2, 2><<<launch_blocks(n_lists, 128), 128, 0, stream>>>(ix->binoff, n_lists, nl,
                                                                                  (uint2*)post);
        BAIL_CUDA(cudaGetLastError());
        count_launch();
    }
    BAIL_CUDA(cudaStreamSynchronize(stream));
#undef BAIL_CUDA
    tmp.release();
    *out = ix;
    return KNN_OK;
}

extern "C" knn_status knn_index_get_info(const knn_index* ix, knn_index_info* info) {
    if (!ix || !info) return fail(KNN_EINVAL, "NULL argument");
    info->n_rows = ix->n_rows;
    info->nnz = ix->nnz;
    info->dim = ix->dim;
    info->block_size = ix->block_size;
    info->n_blocks = ix->n_blocks;
    info->n_levels = ix->n_levels;
    info->dtype = ix->dtype;
    info->max_row_nnz = ix->max_row_nnz;
    info->device_bytes = ix->bufs ? ix->bufs->total() : 0;
    info->host_bytes = ix->host_bytes;
    return KNN_OK;
}

extern "C" knn_status knn_index_to_host(knn_index* ix, void* stream_) {
    if (!ix) return fail(KNN_EINVAL, "NULL argument");
    if (ix->host_bytes) return KNN_OK;
    cudaStream_t s = stream_ ? (cudaStream_t)stream_ : ix->stream;
    const size_t psz = ix->dtype == KNN_U8 ? 4 : 8, wsz = ix->dtype == KNN_U8 ? 1 : 4;
    const size_t nbins = (size_t)ix->n_blocks * (size_t)ix->dim * (size_t)ix->n_levels;
    struct Arr {
        void** ptr;
        size_t bytes;
    } arrs[] = {
        {(void**)&ix->binoff, (nbins + 1) * 4},
        {&ix->postings, (size_t)ix->n_postings * psz},
        {(void**)&ix->s_indptr, ((size_t)ix->n_rows + 1) * 8},
        {(void**)&ix->sp_d, (size_t)ix->nnz * 4},
        {&ix->sp_w, (size_t)ix->nnz * wsz},
        {(void**)&ix->n_unidx, (size_t)ix->n_levels * (size_t)ix->n_rows * 2},
        {(void**)&ix->ubound, (size_t)ix->n_levels * (size_t)ix->n_rows * 4},
    };
    std::vector<void*> host(7, nullptr);
    auto undo = [&](knn_status st) {
        for (void* h : host)
            if (h) cudaFreeHost(h);
        return st;
    };
    size_t total = 0;
    for (int i = 0; i < 7; i++) {
        const size_t bytes = arrs[i].bytes ? arrs[i].bytes : 16;
        if (cudaHostAlloc(&host[i], bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            host[i] = nullptr;
            return undo(fail(KNN_ENOMEM, "pinned host allocation of %zu bytes failed", bytes));
        }
        total += bytes;
        if (arrs[i].bytes) {
            cudaError_t e = cudaMemcpyAsync(host[i], *arrs[i].ptr, arrs[i].bytes, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return undo(fail(KNN_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e)));
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return undo(fail(KNN_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e)));
    // the device addresses of the mapped host arrays (equal to the host addresses with
    // unified addressing); from now on the joins read the index over the host link
    std::vector<void*> dev(7, nullptr);
    for (int i = 0; i < 7; i++) {
        e = cudaHostGetDevicePointer(&dev[i], host[i], 0);
        if (e != cudaSuccess) return undo(fail(KNN_ECUDA, "cudaHostGetDevicePointer: %s", cudaGetErrorString(e)));
    }
    for (int i = 0; i < 7; i++) *arrs[i].ptr = dev[i];
    ix->bufs->release();
    ix->host_arrays = host;
    ix->host_bytes = total;
    return KNN_OK;
}

extern "C" void knn_index_destroy(knn_index* ix) {
    if (!ix) return;
    if (ix->bufs) {
        ix->bufs->release();
        delete ix->bufs;
    }
    for (void* h : ix->host_arrays)
        if (h) cudaFreeHost(h);
    delete ix;
}

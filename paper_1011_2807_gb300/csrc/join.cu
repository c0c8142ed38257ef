// The join: Algorithm 1's loop over S blocks for each query row, with
// Find_Matches_IIB (Algorithm 3) / Find_Matches_IIIB (Algorithm 4) per S block, and the
// KNN candidate set with its pruneScore kept as an exact top-k.
//
// One CTA owns one (query row r, group of consecutive S blocks).  Per S block b:
//   1. threshold: theta = the smallest score that can still enter, i.e. max(floor,
//      score of the current k-th entry + 1 unit: that entry came from an earlier block,
//      so a tie with it loses); the level l is the highest with M * L_l < theta, where
//      M = max weight of r (l = 0 in IIB mode or while no k-th entry exists).  Section 4.4's MinPruneScore for a one-row R block is this
//      row's own pruneScore, and M bounds maxWeight_d(B_r) for every d.
//   2. scan: for each feature (d, r[d]), the prefix of list (b, d) indexed at level l
//      is read with 128-bit loads and r[d] * w is added into a shared-memory
//      accumulator of the block's S vectors (Algorithm 3/4's score map A).
//   3. select: every accumulator entry whose upper bound (partial + M * L_l) reaches
//      theta is checked against its exact unindexed bound, completed with the dot
//      over its unindexed prefix (Algorithm 4's completion step, merged against r's
//      features in shared memory), and pushed when its key beats the k-th entry.
//   4. merge: the pushed keys and the current top-k are bitonic-sorted; the first k
//      stay.  Keys are (score << 32) | ~id, so larger keys are better and ties go to
//      the lower id (the strict "A[s] > pruneScore(r)" of Algorithms 2-4 with S
//      visited in ascending id).
// With several groups per row, the groups publish their k-th key through a per-row
// atomicMax floor (a lower bound on the final k-th key) and a second kernel merges
// the groups' lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace knn {

typedef unsigned long long u64;

constexpr int KMAX = KNN_MAX_K;
constexpr int SORT_CAP = 1024;            // keys in the merge buffer (pushed + current top-k)
constexpr int PUSH_CAP = SORT_CAP - KMAX;  // pushed candidates between merges
constexpr int CQ_CAP = 256;                // entries queued for completion per pass

__device__ __forceinline__ u64 make_key(uint32_t score_bits, uint32_t gid) {
    return ((u64)score_bits << 32) | (u64)(0xFFFFFFFFu - gid);
}
__device__ __forceinline__ uint32_t key_gid(u64 key) { return 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull); }

template <class W>
struct JT;
template <>
struct JT<uint8_t> {
    using Acc = int32_t;
    using Post = uint32_t;
    static constexpr int PER_VEC = 4;  // postings per 16-byte load
    static constexpr bool FIXED_OK = false;   // scores are integers already
    __device__ static uint32_t score_bits(int32_t v) { return (uint32_t)v; }
    __device__ static double score_of_bits(uint32_t b) { return (double)b; }
    __device__ static int32_t value_of_bits(uint32_t b) { return (int32_t)b; }
    // posting = lid | w << 24 (lid < 2^15).  With m = r[d] << 8, the high word of
    // posting * m is w * r[d] exactly: the low part lid * r[d] * 2^8 stays below 2^32.
    using Mul = uint32_t;
    __device__ static int32_t post_lid(uint32_t p) { return (int32_t)(p & 0xFFFFu); }
    __device__ static int32_t post_w(uint32_t p) { return (int32_t)(p >> 24); }
    __device__ static Mul scan_mul(int32_t rw) { return (uint32_t)rw << 8; }
    __device__ static int32_t post_val(uint32_t p, Mul m) { return (int32_t)__umulhi(p, m); }
    __device__ static double ubound(uint32_t b) { return (double)b; }
    __device__ static u64 floor_key(float tau) {
        if (!(tau > 1.0f)) return (u64)1 << 32;
        double c = ceil((double)tau);
        if (c >= 4294967295.0) return (u64)0xFFFFFFFFull << 32;
        return (u64)(uint32_t)c << 32;
    }
    // integer sums are exact: no rounding error to allow for
    __device__ static double gamma(int n) { return 0.0; }
    // bound on the unindexed residual at a level: M * (largest integer weight sum <= L)
    __device__ static double level_bound(double M, float L, double g) { return M * floor((double)L); }
    // smallest partial score whose upper bound (partial + lb) reaches theta
    __device__ static int32_t cheap_min(double theta, double lb) {
        double c = ceil(theta - lb);
        if (c < 1.0) c = 1.0;
        if (c > 2147483647.0) c = 2147483647.0;
        return (int32_t)c;
    }
    __device__ static bool exact_ok(int32_t v, double M, uint32_t ub_bits, double theta, double g) {
        return (double)v + M * (double)ub_bits >= theta;
    }
    template <class S>
    __device__ static void set_cmin(S& st, int32_t c) { st.cmin_i = c; }
    template <class S>
    __device__ static int32_t get_cmin(const S& st) { return st.cmin_i; }
    // Per-block threshold arithmetic in the score's own type (integers), so that the
    // level choice of every block step needs no double-precision instructions.
    using Th = uint32_t;   // int32 scores + 1 fit; a floor of 2^32 - 1 admits nothing
    // Smallest score with which an s of the current S block can still enter: the k-th
    // key came from earlier blocks, whose ids are all smaller, so a tie with its score
    // loses; the floor (a caller threshold or another group's k-th key) admits ties.
    __device__ static Th entry_th(u64 kth, u64 fl) {
        const Th a = kth ? (uint32_t)(kth >> 32) + 1u : 0u;
        return max(a, (uint32_t)(fl >> 32));
    }
    __device__ static double th_value(Th t) { return (double)t; }
    // smallest integer theta with lb < theta (exact) and lb <= margin * theta (the margin
    // only steers the work: its quotient uses the fast reciprocal, which keeps double
    // division and its register cost out of the kernel); saturated at 2^32 - 1, as no
    // int32 score reaches a theta that large
    __device__ static Th level_need(double lb, float margin) {
        const double n = fmax(floor(lb) + 1.0, ceil(lb * (double)__fdividef(1.0f, margin)));
        return n < 4294967295.0 ? (Th)n : 0xFFFFFFFFu;
    }
    __device__ static Th bound_up(double lb) { return lb < 4294967295.0 ? (Th)ceil(lb) : 0xFFFFFFFFu; }
    // cheap_min for an integer theta and the bound rounded up: max(1, theta - lbu)
    __device__ static int32_t cheap_min_th(Th theta, Th lbu) {
        const uint32_t c = theta > lbu ? theta - lbu : 1u;
        return c > 2147483647u ? 2147483647 : (int32_t)max(c, 1u);
    }
    template <class S>
    __device__ static Th& need(S& st, int l) { return st.need_i[l]; }
    template <class S>
    __device__ static Th& lbu(S& st, int l) { return st.lbu_i[l]; }
    template <class S>
    __device__ static Th& theta(S& st) { return st.theta_i; }
};
template <>
struct JT<float> {
    using Acc = float;
    using Post = uint2;
    static constexpr int PER_VEC = 2;
    static constexpr bool FIXED_OK = true;    // the scan may accumulate in fixed point
    __device__ static uint32_t score_bits(float v) { return __float_as_uint(v); }
    __device__ static double score_of_bits(uint32_t b) { return (double)__uint_as_float(b); }
    __device__ static float value_of_bits(uint32_t b) { return __uint_as_float(b); }
    using Mul = float;
    __device__ static int32_t post_lid(uint2 p) { return (int32_t)p.x; }
    __device__ static float post_w(uint2 p) { return __uint_as_float(p.y); }
    __device__ static Mul scan_mul(float rw) { return rw; }
    __device__ static float post_val(uint2 p, Mul m) { return m * __uint_as_float(p.y); }
    __device__ static double ubound(uint32_t b) { return (double)__uint_as_float(b); }
    __device__ static u64 floor_key(float tau) {
        if (!(tau > 0.0f)) return (u64)1 << 32;
        return (u64)__float_as_uint(tau) << 32;
    }
    // Rounding.  A candidate's score is F = fl(v + res): v its fp32 partial (compared as
    // computed, so its own rounding needs no allowance), res the fp32 dot over its
    // unindexed features.  res has at most n = nnz(r) nonzero terms (a feature missing
    // from r adds an exact 0), so for any summation order res <= Q (1 + gamma_n), Q the
    // real residual, with gamma_n = n u / (1 - n u), u = 2^-24 (the standard bound for n
    // roundings of nonnegative terms); a further 2^-40 covers the double arithmetic of
    // the bounds themselves.  The final add gives F <= (v + res)(1 + u).
    static constexpr double SLACK = 1.0 / (1 << 20);   // >= 2u: room for the final add
    __device__ static double gamma(int n) {
        const double nu = (double)(n + 1) * (1.0 / 16777216.0);
        return nu / (1.0 - nu) + 1.0 / 1099511627776.0;
    }
    // bound on the computed residual at a level: M * L * (1 + gamma)
    __device__ static double level_bound(double M, float L, double g) { return M * (double)L * (1.0 + g); }
    // a partial v below this cannot give F >= theta: v < theta (1 - SLACK) - lb implies
    // (v + lb)(1 + u) < theta
    __device__ static float cheap_min(double theta, double lb) {
        double c = theta * (1.0 - SLACK) - lb;
        float f = c > 0.0 ? __double2float_rd(c) : 0.0f;
        return fmaxf(f, 1.40129846e-45f);   // candidates are always > 0
    }
    // F can reach theta: (v + M ub)(1 + gamma) >= theta, with gamma >= u also covering the
    // final add
    __device__ static bool exact_ok(float v, double M, uint32_t ub_bits, double theta, double g) {
        return ((double)v + M * (double)__uint_as_float(ub_bits)) * (1.0 + g) >= theta;
    }
    template <class S>
    __device__ static void set_cmin(S& st, float c) { st.cmin_f = c; }
    template <class S>
    __device__ static float get_cmin(const S& st) { return st.cmin_f; }
    // Per-block threshold arithmetic in float, rounded so that the level test and the
    // candidate cut stay on the safe side of their double-precision definitions.
    using Th = float;
    // as for integers, with the next float above the k-th score (scores are finite and > 0)
    __device__ static Th entry_th(u64 kth, u64 fl) {
        const float a = kth ? __uint_as_float((uint32_t)(kth >> 32) + 1u) : 0.0f;
        return fmaxf(a, __uint_as_float((uint32_t)(fl >> 32)));
    }
    __device__ static double th_value(Th t) { return (double)t; }
    // smallest float theta with lb < theta (exact); the margin part as for integers
    __device__ static Th level_need(double lb, float margin) {
        float a = __double2float_ru(lb);   // >= lb >= 0; the next float if equal
        if ((double)a <= lb && a < __int_as_float(0x7f800000)) a = __uint_as_float(__float_as_uint(a) + 1u);
        return fmaxf(a, __double2float_ru(lb * (double)__fdividef(1.0f, margin)));
    }
    __device__ static Th bound_up(double lb) { return __double2float_ru(lb); }
    // cheap_min from the bound rounded up, rounding down: at most its double value
    __device__ static float cheap_min_th(Th theta, Th lbu) {
        const float c = __fsub_rd(__fmul_rd(theta, 1.0f - 1.0f / 1048576.0f), lbu);   // theta (1 - SLACK) - lb
        return fmaxf(c, 1.40129846e-45f);
    }
    template <class S>
    __device__ static Th& need(S& st, int l) { return st.need_f[l]; }
    template <class S>
    __device__ static Th& lbu(S& st, int l) { return st.lbu_f[l]; }
    template <class S>
    __device__ static Th& theta(S& st) { return st.theta_f; }
};

struct JoinParams {
    int64_t n_rows;
    const int64_t* r_indptr;
    const int32_t* r_idx;
    const void* r_val;
    int64_t n_s;
    int32_t dim, n_blocks, n_levels, block_shift;
    const uint32_t* binoff;
    const void* postings;
    const int64_t* s_indptr;
    const int32_t* sp_d;
    const void* sp_w;
    const uint16_t* n_unidx;
    const uint32_t* ubound;
    int64_t u_stride;   // elements between levels of n_unidx / ubound (|S|, or a staged slice's)
    float s_maxnorm;    // largest L2 norm of an S vector, rounded up (float scores: fixed-point scale)
    const int32_t* row_list;   // one group per row: the rows of this launch (NULL: row = CTA index)
    uint8_t* fx_flag;   // float joins in fixed point: per row, set to 1 by the fixed-point launches
                        // when the row must be joined again in fp32; the fp32 re-join launch
                        // joins only the rows set
    float levels[KNN_MAX_LEVELS];
    int32_t k, groups, blocks_per_group, iiib, max_r_nnz;
    int32_t bf;         // brute force: every s scored in full (Algorithm 2), no posting scan
    float level_margin;
    int32_t rden_dim;   // >0: r's uint8 weights are kept densely (rden_dim bytes, a multiple of 16)
    const float* init_thr;
    u64* part_keys;
    int32_t* out_ids;
    void* out_scores;
    int32_t* n_found;
    u64* floor_keys;
    unsigned long long* touched;
    unsigned long long* stats;
    // S-block-synchronous schedule (groups == 1): this launch covers blocks
    // [block_begin, block_end) of every row; rows carry their top-k keys between launches
    int32_t block_begin, block_end, carry_in, carry_out;
    u64* carry;
    int32_t* done;   // batched form: per row, the number of groups finished
};

struct SmemLayout {
    size_t acc, rf_d, rf_w, lbeg, lend, ipre, topk, sort, cq, rden, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemLayout smem_layout(int nb, int max_r_nnz, int rden_bytes = 0) {
    SmemLayout L;
    size_t o = 0;
    L.acc = o;  o = align16(o + (size_t)nb * 4);
    L.rf_d = o; o = align16(o + (size_t)max_r_nnz * 4);
    L.rf_w = o; o = align16(o + (size_t)max_r_nnz * 4);
    L.lbeg = o; o = align16(o + (size_t)max_r_nnz * 8);   // two buffers (this / next S block)
    L.lend = o; o = align16(o + (size_t)max_r_nnz * 8);
    L.ipre = o; o = align16(o + (size_t)(max_r_nnz + 1) * 8);   // two buffers
    L.topk = o; o = align16(o + (size_t)KMAX * 8);
    L.sort = o; o = align16(o + (size_t)SORT_CAP * 8);
    L.cq = o;   o = align16(o + (size_t)CQ_CAP * 8);
    L.rden = o; o = align16(o + (size_t)rden_bytes);
    L.total = o;
    return L;
}

// Descending bitonic sort of buf[0..P), P a power of two, all threads of the CTA.
__device__ void cta_bitonic_desc(u64* buf, int P) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool desc = (lo & size) == 0;
                u64 a = buf[lo], b = buf[hi];
                if ((a < b) == desc) {
                    buf[lo] = b;
                    buf[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

struct CtaState {
    int cnt;        // pushed candidates in the sort buffer
    int size;       // entries in topk
    int level;
    int pending[2]; // candidates still masked (overflow rounds), by S block parity: warp 0
                    // resets the next block's count while others may still read this one
    uint32_t theta_i;  // entry threshold of the current block (integer / float scores)
    float theta_f;
    u64 floor;      // keys below this never qualify
    u64 kth;        // current k-th key (0 while fewer than k)
    double M;       // largest weight of r
    double g;       // relative rounding allowance of a completed score (0 for integers)
    int fx;         // float scores: this row accumulates the scan in fixed point (fx_decide)
    float fx_scale, fx_inv;   // the fixed-point scale (a power of two) and its inverse
    double fx_rsq;  // |r|^2
    double lb;      // residual bound of the current level (0 at level 0)
    float cmin_f;   // smallest partial score worth a look in this block (as float/int)
    int32_t cmin_i;
    double lbnd[KNN_MAX_LEVELS];  // residual bound of every level for this row
    uint32_t need_i[KNN_MAX_LEVELS], lbu_i[KNN_MAX_LEVELS]; // per level: smallest theta that
    float need_f[KNN_MAX_LEVELS], lbu_f[KNN_MAX_LEVELS];    // may use it, bound rounded up
    unsigned long long n_steps, n_merges, n_rounds;  // work counters (thread 0)
    int qcnt;       // entries in the completion queue
    int dq_n;       // candidates deferred to warp 0 (in the completion queue's arrays)
    int dq_level;   // level of the block they came from
    int pred_level; // level the next block's list ranges were prepared for (-1: none)
    int need_prepare;
    int allowed;    // highest level the current threshold allows (the next block's plan)
    // radix select of a candidate threshold (blocks with too many candidates)
    int rs_shift, rs_need, rs_done;
    unsigned rs_prefix, rs_above, rs_key;
    unsigned hist[256];
};

// merge pushed keys with topk; all threads
__device__ void merge_topk(u64* topk, u64* sortbuf, CtaState& st, int k) {
    __syncthreads();
    int cnt = st.cnt;
    if (cnt == 0) return;
    int m = st.size;
    for (int i = threadIdx.x; i < m; i += blockDim.x) sortbuf[cnt + i] = topk[i];
    int n = cnt + m;
    int P = 2;
    while (P < n) P <<= 1;
    for (int i = n + threadIdx.x; i < P; i += blockDim.x) sortbuf[i] = 0ull;
    __syncthreads();
    cta_bitonic_desc(sortbuf, P);
    int keep = min(k, n);
    for (int i = threadIdx.x; i < keep; i += blockDim.x) topk[i] = sortbuf[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        st.size = keep;
        st.cnt = 0;
        st.kth = keep == k ? topk[k - 1] : 0ull;
    }
    __syncthreads();
}

// In-place exclusive scan of data[0..n) by the whole CTA; data[n] = total.
// Each thread owns a contiguous segment; `wtot` holds 32 words of scratch.
__device__ void cta_exclusive_scan(uint32_t* data, int n, uint32_t* wtot) {
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + T - 1) / T;
    const int a = min(n, tid * per), b = min(n, a + per);
    uint32_t s = 0;
    for (int i = a; i < b; i++) s += data[i];
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < (T >> 5) ? wtot[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < (T >> 5)) wtot[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    uint32_t run = (warp ? wtot[warp - 1] : 0u) + x - s;
    for (int i = a; i < b; i++) {
        uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
    if (tid == T - 1) data[n] = wtot[(T >> 5) - 1];
    __syncthreads();
}

// Shared-memory accesses through 32-bit shared addresses (no generic-address checks).
__device__ __forceinline__ void red_add_shared(uint32_t saddr, int32_t v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(saddr), "r"(v));
}
__device__ __forceinline__ void red_add_shared(uint32_t saddr, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(saddr), "f"(v));
}
__device__ __forceinline__ int4 ld_shared_v4(uint32_t saddr) {
    int4 r;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"(saddr));
    return r;
}
__device__ __forceinline__ void st_shared_v4(uint32_t saddr, int4 v) {
    asm volatile("st.shared.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(saddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

template <class W>
__device__ __forceinline__ typename JT<W>::Acc lookup_r(const int32_t* rf_d, const typename JT<W>::Acc* rf_w,
                                                        int n, int32_t d) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (rf_d[mid] < d) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && rf_d[lo] == d) ? rf_w[lo] : (typename JT<W>::Acc)0;
}

// One query row against S blocks [b0, b1) of group g (the whole CTA).
// out_mode: OUT_FINAL writes ids/scores, OUT_CARRY the row's keys to p.carry for the
// next range of S blocks, OUT_GROUP the group's keys to p.part_keys (merged later).
enum { OUT_FINAL = 0, OUT_CARRY = 1, OUT_GROUP = 2 };

// List ranges of r's features in S block bb at level `level`, and the work items: each
// list (starting on a 16-byte chunk) is cut into items of at most CH chunks, and
// ipre[i] is the first item of list i (ipre[rn] = total).  One warp, lists in rounds
// of 32 with a warp scan per round.
template <int V, int CH>
__device__ __forceinline__ void prepare_block_warp(const JoinParams& p, const int32_t* rf_d, int rn, int bb,
                                                   int level, uint32_t* lbeg, uint32_t* lend, uint32_t* ipre,
                                                   int lane) {
    const size_t bbase = (size_t)bb * (size_t)p.dim;
    const int off = p.n_levels - level;
    uint32_t carry = 0;
    for (int i0 = 0; i0 < rn; i0 += 32) {
        const int i = i0 + lane;
        uint32_t it = 0;
        if (i < rn) {
            const size_t base = (bbase + (size_t)rf_d[i]) * (size_t)p.n_levels;
            const uint32_t a = __ldg(p.binoff + base), e = __ldg(p.binoff + base + off);
            lbeg[i] = a;
            lend[i] = e;
            it = ((e - a + V - 1) / V + CH - 1) / CH;
        }
        uint32_t x = it;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (i < rn) ipre[i] = carry + x - it;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) ipre[rn] = carry;
}

// Float joins sum the scan in fixed point: each product r[d] w times a power-of-two
// scale, rounded to an integer, added with an integer shared-memory atomic (2.5x the
// rate of the float one on this GPU), and integer sums do not depend on the order of
// the adds.  The scale keeps every partial below 2^30 -- a score, and any one product,
// is at most |r| max|s| (Cauchy-Schwarz) -- so a partial converted back is off by at
// most n / (2 scale) (n = nnz(r) rounded terms) besides fp32's relative rounding of the
// products and of the conversion.  Nothing else changes: the kernel ranks the converted
// partials like fp32 ones, and every bound of the cut is stated in terms of the
// computed partial.  When a row is done, one unit (1 / scale) must be at most 2^-23 of
// the smallest score it returns: each rounded term then errs by no more than an fp32
// rounding at that magnitude (2^-24 of it), so the fixed-point sum's error bound is no
// larger than that of the fp32 sum it replaces (n 2^-24 relative for n terms).  A row
// that fails, or that has no usable scale, is flagged and joined again in fp32.
template <class S>
__device__ void fx_decide(const JoinParams& p, S& st) {
    st.fx = 0;
    st.fx_scale = 1.0f;
    st.fx_inv = 1.0f;
    if (!(p.s_maxnorm >= 1e-18f) || !(st.fx_rsq > 0.0) || !(st.fx_rsq < 1e300)) return;
    const double ub = sqrt(st.fx_rsq) * (1.0 + 1e-9) * (double)p.s_maxnorm;
    int e;
    frexp(ub, &e);                   // ub < 2^e
    const int es = 30 - e;           // scale 2^es: ub * scale < 2^30
    if (es > 100 || es < -100) return;
    const double scale = ldexp(1.0, es);
    st.fx = 1;
    st.fx_scale = (float)scale;
    st.fx_inv = (float)(1.0 / scale);
}

template <class W, bool COUNT, bool BF, bool FX>
__device__ __forceinline__ void join_row(const JoinParams& p, const int64_t row, const int g, const int b0,
                                         const int b1, const bool carry_in, const int out_mode,
                                         unsigned char* smem) {
    using Acc = typename JT<W>::Acc;
    using Post = typename JT<W>::Post;
    // FX: a fixed-point launch of a float join (fx_decide); otherwise the fp32 (or
    // integer) join, which, when given the fixed-point launches' flags, joins only the
    // rows they flagged
    constexpr bool FXABLE = JT<W>::FIXED_OK && !BF && FX;
    if constexpr (JT<W>::FIXED_OK && !BF && !FX) {
        if (p.fx_flag && !p.fx_flag[row]) return;
    }
    __shared__ CtaState st;
    __shared__ uint32_t red_m[32];
    __shared__ unsigned long long red_u[32];

    const int nb = 1 << p.block_shift;
    const SmemLayout L = smem_layout(nb, p.max_r_nnz, p.rden_dim);
    Acc* acc = (Acc*)(smem + L.acc);
    const uint32_t acc_s = (uint32_t)__cvta_generic_to_shared(acc);
    int32_t* rf_d = (int32_t*)(smem + L.rf_d);
    Acc* rf_w = (Acc*)(smem + L.rf_w);
    uint32_t* lbeg_buf = (uint32_t*)(smem + L.lbeg);
    uint32_t* lend_buf = (uint32_t*)(smem + L.lend);
    uint32_t* ipre_buf = (uint32_t*)(smem + L.ipre);
    uint32_t* cq_gid = (uint32_t*)(smem + L.cq);
    Acc* cq_v = (Acc*)(smem + L.cq + CQ_CAP * 4);
    uint8_t* rden = p.rden_dim ? (uint8_t*)(smem + L.rden) : nullptr;   // r's weights by dimension (uint8)
    u64* topk = (u64*)(smem + L.topk);
    u64* sortbuf = (u64*)(smem + L.sort);

    const int tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
    const int64_t ra = p.r_indptr[row];
    const int rn = (int)(p.r_indptr[row + 1] - ra);

    // load r (ascending d) and its largest weight
    uint32_t mloc = 0u;   // as score bits: weights are > 0, so the bits order like the values
    float rsq = 0.0f;     // sum of squared weights (float rows: the fixed-point scale)
    for (int i = tid; i < rn; i += T) {
        rf_d[i] = p.r_idx[ra + i];
        Acc w = (Acc)((const W*)p.r_val)[ra + i];
        rf_w[i] = w;
        mloc = max(mloc, JT<W>::score_bits(w));
        if (FXABLE) rsq = fmaf((float)w, (float)w, rsq);
    }
    mloc = __reduce_max_sync(0xffffffffu, mloc);
    if (lane == 0) red_m[warp] = mloc;
    if (FXABLE) {
        for (int o = 16; o > 0; o >>= 1) rsq += __shfl_xor_sync(0xffffffffu, rsq, o);
        if (lane == 0) red_u[warp] = (unsigned long long)__float_as_uint(rsq);
    }
    // clear the accumulator (and the dense copy of r)
    for (int i = tid * 4; i < nb; i += T * 4) *(int4*)(acc + i) = make_int4(0, 0, 0, 0);
    if (rden) {
        for (int i = tid * 16; i < p.rden_dim; i += T * 16) *(int4*)(rden + i) = make_int4(0, 0, 0, 0);
        __syncthreads();
        for (int i = tid; i < rn; i += T) rden[rf_d[i]] = (uint8_t)rf_w[i];
    }
    __syncthreads();
    if (warp == 0) {
        const double m = (double)JT<W>::value_of_bits(
            __reduce_max_sync(0xffffffffu, lane < nwarps ? red_m[lane] : 0u));
        const double g = JT<W>::gamma(rn);
        if (lane < p.n_levels) {   // lane l: level l's bound and the thresholds derived from it
            const double lb = lane ? JT<W>::level_bound(m, p.levels[lane], g) : 0.0;
            st.lbnd[lane] = lb;
            JT<W>::need(st, lane) = JT<W>::level_need(lb, p.level_margin);
            JT<W>::lbu(st, lane) = JT<W>::bound_up(lb);
        }
        if (FXABLE && lane == 0) {
            double q = 0.0;
            for (int w = 0; w < nwarps; w++) q += (double)__uint_as_float((uint32_t)red_u[w]);
            st.fx_rsq = q * (1.0 + (double)(rn + 32) * (1.0 / 8388608.0));   // fp32 sums, rounded up
        }
        if (lane == 0) {
            st.M = m;
            st.g = g;
            st.fx = 0;
            st.size = 0;
            st.cnt = 0;
            st.kth = 0ull;
            st.floor = p.init_thr ? JT<W>::floor_key(p.init_thr[row]) : ((u64)1 << 32);
            st.n_steps = st.n_merges = st.n_rounds = 0;
            st.qcnt = 0;
            st.dq_n = 0;
            st.pred_level = -1;
        }
    }
    if (carry_in) {   // the row's top-k from the earlier S blocks
        for (int q = tid; q < p.k; q += T) topk[q] = __ldcg(p.carry + row * p.k + q);
        __syncthreads();
        if (tid == 0) {
            int n = 0;
            while (n < p.k && topk[n] != 0ull) n++;
            st.size = n;
            st.kth = n == p.k ? topk[p.k - 1] : 0ull;
        }
    }
    if (FXABLE && tid == 0) {
        fx_decide(p, st);
        if (!st.fx) p.fx_flag[row] = 1;   // no usable scale: the fp32 re-join takes the row
    }
    __syncthreads();
    if (FXABLE && !st.fx) return;

    uint32_t n_cand = 0, n_comp = 0, n_push = 0, n_resf = 0;   // this thread's counters
    unsigned long long n_post = 0, n_add = 0;   // postings scanned; shared-memory adds issued
    const int chunks = nb / (T * 4);  // <= 16 by construction (mask has 64 bits)

    // Warp 0 completes and merges the candidates a block deferred (few of them): one lane
    // per candidate, keys inserted into the sorted top-k one at a time.  Runs during the
    // next block's scan, or after the last block.
    auto drain = [&]() {
        const int n = st.dq_n;
        if (n == 0) return;
        const int lvl = st.dq_level;
        const double Mr = st.M;
        const u64 fl = st.floor;
        u64 kth = st.kth;
        int sz = st.size;
        bool merged = false;
        for (int e0 = 0; e0 < n; e0 += 32) {
            const int e = e0 + lane;
            u64 key = 0ull;
            bool ins = false;
            if (e < n) {
                const uint32_t gid = cq_gid[e];
                Acc v = cq_v[e];
                bool ok = true;
                if (lvl > 0) {
                    const double th = JT<W>::score_of_bits((uint32_t)((kth > fl ? kth : fl) >> 32));
                    ok = JT<W>::exact_ok(v, Mr, p.ubound[(int64_t)lvl * p.u_stride + gid], th, st.g);
                    if (ok) {   // Algorithm 4's dot over the unindexed features
                        const int64_t j0 = p.s_indptr[gid];
                        const int m = p.n_unidx[(int64_t)lvl * p.u_stride + gid];
                        Acc res = (Acc)0;
                        for (int q = 0; q < m; q++) {
                            const int32_t d = p.sp_d[j0 + q];
                            const Acc w = (Acc)((const W*)p.sp_w)[j0 + q];
                            res += (rden ? (Acc)rden[d] : lookup_r<W>(rf_d, rf_w, rn, d)) * w;
                        }
                        v += res;
                        n_comp++;
                        n_resf += m;
                    }
                }
                if (ok) {
                    key = make_key(JT<W>::score_bits(v), gid);
                    ins = key >= fl && key > kth;
                }
            }
            for (unsigned bal = __ballot_sync(0xffffffffu, ins); bal; bal &= bal - 1) {
                const u64 kk = __shfl_sync(0xffffffffu, key, __ffs(bal) - 1);
                if (sz == p.k && kk <= kth) continue;
                int c = 0;
                for (int i = lane; i < sz; i += 32) c += topk[i] > kk;
                const int pos = __reduce_add_sync(0xffffffffu, c);
                const int nsz = min(sz + 1, p.k);
                const int i0 = pos + lane, i1 = pos + lane + 32;   // k <= 64
                const u64 t0 = i0 < nsz - 1 ? topk[i0] : 0ull, t1 = i1 < nsz - 1 ? topk[i1] : 0ull;
                __syncwarp();
                if (i0 < nsz - 1) topk[i0 + 1] = t0;
                if (i1 < nsz - 1) topk[i1 + 1] = t1;
                if (lane == 0) topk[pos] = kk;
                __syncwarp();
                sz = nsz;
                kth = sz == p.k ? topk[p.k - 1] : 0ull;
                if (lane == 0) n_push++;
                merged = true;
            }
        }
        if (lane == 0) {
            st.size = sz;
            st.kth = kth;
            st.dq_n = 0;
            if (merged) st.n_merges++;
        }
        __syncwarp();
    };

    for (int b = (rn > 0 ? b0 : b1); b < b1; b++) {
        // ---- 1. level (warp 0: lane l tests level l) ----
        // The list ranges and work items of this block were prepared by warp 0 during the
        // previous block's scan, for the level the threshold then allowed; they are
        // prepared here, by the whole CTA, only for a launch's first block.
        constexpr int V = JT<W>::PER_VEC;   // postings per 16-byte chunk
        constexpr int G = 16, U = 4, CH = G * U;
        uint32_t* lbeg = lbeg_buf + (b & 1) * p.max_r_nnz;
        uint32_t* lend = lend_buf + (b & 1) * p.max_r_nnz;
        uint32_t* ipre = ipre_buf + (b & 1) * (p.max_r_nnz + 1);
        if (warp == 0) {
            u64 fl = st.floor;
            if (p.floor_keys) {
                u64 shared = *(volatile u64*)(p.floor_keys + row);
                if (shared > fl) fl = shared;
            }
            // the highest level l with M * L_l < theta and M * L_l <= margin * theta,
            // compared in the score's own type against thresholds set up per row
            const auto theta = JT<W>::entry_th(st.kth, fl);
            bool ok = false;
            if (p.iiib && lane >= 1 && lane < p.n_levels) ok = theta >= JT<W>::need(st, lane);
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            const int allowed = m ? 31 - __clz(m) : 0;
            // theta never falls within a row, so the level warp 0 prepared this block for
            // (allowed for an earlier theta) is still exact: a block whose allowed level
            // rose keeps it, and the next block is prepared for the new level, instead of
            // the whole CTA preparing this block again
            const int level = (!BF && st.pred_level >= 0 && st.pred_level < allowed) ? st.pred_level : allowed;
            if (lane == 0) {
                st.floor = fl;
                JT<W>::theta(st) = theta;
                st.level = level;
                st.allowed = allowed;
                st.need_prepare = !BF && st.pred_level != level;
                st.pending[b & 1] = 0;
                st.n_steps++;
                st.lb = st.lbnd[level];
                JT<W>::set_cmin(st, JT<W>::cheap_min_th(theta, JT<W>::lbu(st, level)));
            }
        }
        __syncthreads();
        const int level = st.level;
        if (st.need_prepare) {
            const size_t bbase = (size_t)b * (size_t)p.dim;
            for (int i = tid; i < rn; i += T) {
                const size_t base = (bbase + (size_t)rf_d[i]) * (size_t)p.n_levels;
                const uint32_t a = __ldg(p.binoff + base), e = __ldg(p.binoff + base + (p.n_levels - level));
                lbeg[i] = a;
                lend[i] = e;
                ipre[i] = ((e - a + V - 1) / V + CH - 1) / CH;
            }
            __syncthreads();
            cta_exclusive_scan(ipre, rn, (uint32_t*)red_u);
        }
        // ---- 2. scan: acc[lid] += r[d] * w over the indexed prefixes ----
        // Each 16-lane sub-warp takes an equal contiguous range of work items, so every
        // sub-warp runs the same number of iterations; per item each lane loads U chunks
        // (two 128-byte lines per sub-warp per load) before adding; one add instruction
        // covers slot j of 16 consecutive chunks, which the index build placed in distinct
        // banks where it could.  Only the last chunk of a prefix can be partial (lists
        // start on chunk boundaries).
        // With 4 or more warps, warp 0 instead prepares the next block (for the level
        // the current threshold allows) while the others scan, so that work leaves the
        // critical path.
        const bool producer = nwarps >= 4;
        if (producer && warp == 0) {
            drain();   // the previous block's deferred candidates
            if (b + 1 < b1 && !BF)
                prepare_block_warp<V, CH>(p, rf_d, rn, b + 1, st.allowed, lbeg_buf + ((b + 1) & 1) * p.max_r_nnz,
                                          lend_buf + ((b + 1) & 1) * p.max_r_nnz,
                                          ipre_buf + ((b + 1) & 1) * (p.max_r_nnz + 1), lane);
            if (lane == 0) st.pred_level = b + 1 < b1 ? st.allowed : -1;
        } else if (BF) {
            // Algorithm 2 on the GPU (a baseline): every s of the block is scored in full
            // against r, whose weights are read from the dense copy in shared memory (or by
            // binary search in r's sorted features); each entry is written once.
            const int t0 = producer ? 32 : 0;
            const int64_t s0 = (int64_t)b << p.block_shift;
            const int ns = (int)min((int64_t)nb, p.n_s - s0);
            for (int lid = tid - t0; lid < ns; lid += T - t0) {
                const int64_t a = p.s_indptr[s0 + lid], e = p.s_indptr[s0 + lid + 1];
                Acc sum = (Acc)0;
                for (int64_t j = a; j < e; j++) {
                    const int32_t d = p.sp_d[j];
                    const Acc w = (Acc)((const W*)p.sp_w)[j];
                    sum += (rden ? (Acc)rden[d] : lookup_r<W>(rf_d, rf_w, rn, d)) * w;
                }
                acc[lid] = sum;
                if (COUNT) n_post += (unsigned long long)(e - a);
            }
        } else {
            const Post* post = (const Post*)p.postings;
            const int t0 = producer ? 32 : 0;
            const int nsub = (T - t0) / G, sub = (tid - t0) / G, sl = tid % G;
            const uint32_t total = ipre[rn];
            const uint32_t per = (total + nsub - 1) / nsub;
            const uint32_t I0 = min(total, (uint32_t)sub * per), I1 = min(total, I0 + per);
            int li = 0;
            {   // largest li with ipre[li] <= I0
                int lo = 0, hi = rn;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (ipre[mid] <= I0) lo = mid;
                    else hi = mid - 1;
                }
                li = lo;
            }
            using Mul = typename JT<W>::Mul;
            // INT: the row accumulates rounded, scaled products in integers (fx_decide)
            auto scan_items = [&](auto fx_tag, const float fxs) {
                constexpr bool INT = decltype(fx_tag)::value;
                for (uint32_t I = I0; I < I1; I++) {
                    while (ipre[li + 1] <= I) li++;
                    const uint32_t en = lend[li];
                    const Mul m = JT<W>::scan_mul(INT ? rf_w[li] * fxs : rf_w[li]);
                    const uint32_t p0 = lbeg[li] + (I - ipre[li]) * (CH * V) + (uint32_t)sl * V;   // this lane's first posting
                    const uint4* src = (const uint4*)(post + p0);
                    uint4 v[U];
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (p0 + (uint32_t)(G * u * V) < en) v[u] = src[G * u];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const uint32_t q = p0 + (uint32_t)(G * u * V);
                        if (q < en) {
                            // postings of the chunk past the prefix end (level > 0) belong to the
                            // same list: they are added with weight 0 rather than branched around
                            const Post* e = (const Post*)&v[u];
                            const uint32_t nv = en - q;
#pragma unroll
                            for (int j = 0; j < V; j++) {
                                const bool in = j == 0 || (uint32_t)j < nv;
                                const uint32_t addr = acc_s + 4u * (uint32_t)JT<W>::post_lid(e[j]);
                                if constexpr (INT)
                                    red_add_shared(addr, (int32_t)__float2int_rn(JT<W>::post_val(e[j], in ? m : (Mul)0)));
                                else
                                    red_add_shared(addr, JT<W>::post_val(e[j], in ? m : (Mul)0));
                                if (COUNT) n_post += in && JT<W>::post_w(e[j]) != 0;   // padding has weight 0
                            }
                            if (COUNT) n_add += V;
                        }
                    }
                }
            };
            if constexpr (FXABLE) scan_items(std::true_type{}, st.fx_scale);
            else scan_items(std::false_type{}, 1.0f);
        }
        __syncthreads();
        // ---- 3. select ----
        const double M = st.M;
        const double lb = st.lb;
        const Acc cmin = JT<W>::get_cmin(st);   // > 0
        constexpr bool fxrow = FXABLE;   // every row of the fixed-point launch
        const float fxinv = st.fx_inv;
        const int64_t gbase = (int64_t)b << p.block_shift;
        unsigned long long mask = 0ull;
        int mycount = 0;
#pragma unroll 8
        for (int c = 0; c < chunks; c++) {
            int lid0 = c * T * 4 + tid * 4;
            int4 raw = ld_shared_v4(acc_s + 4u * lid0);
            if (FXABLE && fxrow) {   // fixed-point partials back to floats (0 stays 0)
                raw = make_int4(__float_as_int(__int2float_rn(raw.x) * fxinv), __float_as_int(__int2float_rn(raw.y) * fxinv),
                                __float_as_int(__int2float_rn(raw.z) * fxinv), __float_as_int(__int2float_rn(raw.w) * fxinv));
            }
            Acc* v = (Acc*)&raw;
            if (v[0] < cmin && v[1] < cmin && v[2] < cmin && v[3] < cmin) {
                st_shared_v4(acc_s + 4u * lid0, make_int4(0, 0, 0, 0));
                continue;
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (v[e] >= cmin) {
                    mask |= 1ull << (c * 4 + e);
                    mycount++;
                } else {
                    v[e] = (Acc)0;
                }
            }
            st_shared_v4(acc_s + 4u * lid0, raw);
        }
        n_cand += mycount;
        // total candidates of the block
        int wsum = mycount;
        for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
        int& pending = st.pending[b & 1];
        if (lane == 0 && wsum) atomicAdd(&pending, wsum);
        __syncthreads();
        const int pend = pending;   // most blocks, once the threshold has settled, have none
        if (pend > 0 && producer && pend <= CQ_CAP) {
            // Few candidates: queue them for warp 0, which completes and merges them during
            // the next block's scan.  That block's threshold is then one block stale, which
            // only loosens its pruning.
            for (; mask; mask &= mask - 1) {
                const int bit = __ffsll(mask) - 1;
                const int lid = (bit >> 2) * T * 4 + tid * 4 + (bit & 3);
                const int slot = atomicAdd(&st.dq_n, 1);
                cq_gid[slot] = (uint32_t)(gbase + lid);
                cq_v[slot] = acc[lid];
                acc[lid] = (Acc)0;
            }
            if (tid == 0) st.dq_level = level;
        } else if (pend > 0) {
        if (pending > PUSH_CAP) {
            // Too many candidates for one merge (typically the first block, where the
            // threshold is still 0).  Radix-select, on the candidates' partial scores,
            // a value t with at least k candidates >= t and at most PUSH_CAP of them;
            // then a candidate whose full score is below t (partial < t - lb) cannot
            // reach the row's top-k: k entries of this block already beat it.
            unsigned kmax_l = 0;
            for (unsigned long long mm = mask; mm; mm &= mm - 1) {
                int bit = __ffsll(mm) - 1;
                int lid = (bit >> 2) * T * 4 + tid * 4 + (bit & 3);
                kmax_l = max(kmax_l, JT<W>::score_bits(acc[lid]));
            }
            for (int o = 16; o > 0; o >>= 1) kmax_l = max(kmax_l, __shfl_xor_sync(0xffffffffu, kmax_l, o));
            if (lane == 0) red_u[warp] = kmax_l;
            __syncthreads();
            if (tid == 0) {
                unsigned km = 0;
                for (int w = 0; w < nwarps; w++) km = max(km, (unsigned)red_u[w]);
                const unsigned kmin = JT<W>::score_bits(cmin);
                const unsigned diff = km ^ kmin;
                const int hb = diff ? 31 - __clz(diff) : 0;
                st.rs_shift = hb + 1;     // lowest bit already fixed in the prefix
                st.rs_prefix = hb >= 31 ? 0u : (km & ~((2u << hb) - 1u));
                st.rs_need = p.k;
                st.rs_above = 0;
                st.rs_done = diff == 0;   // all candidates equal: nothing to split
                st.rs_key = kmin;
            }
            __syncthreads();
            while (!st.rs_done) {
                const int lo = st.rs_shift;                 // bits >= lo are fixed
                const int shift = lo > 8 ? lo - 8 : 0;      // this pass: bits [shift, lo)
                const unsigned dmask = (1u << (lo - shift)) - 1u;
                const unsigned prefix = st.rs_prefix;
                const unsigned hi_mask = lo >= 32 ? 0u : ~((1u << lo) - 1u);
                for (int i = tid; i < 256; i += T) st.hist[i] = 0;
                __syncthreads();
                for (unsigned long long mm = mask; mm; mm &= mm - 1) {
                    int bit = __ffsll(mm) - 1;
                    int lid = (bit >> 2) * T * 4 + tid * 4 + (bit & 3);
                    unsigned key = JT<W>::score_bits(acc[lid]);
                    if ((key & hi_mask) == (prefix & hi_mask)) atomicAdd(&st.hist[(key >> shift) & dmask], 1u);
                }
                __syncthreads();
                if (tid == 0) {
                    unsigned above = 0;
                    int t = (int)dmask;
                    for (; t > 0; t--) {
                        if (above + st.hist[t] >= (unsigned)st.rs_need) break;
                        above += st.hist[t];
                    }
                    const unsigned newprefix = (prefix & hi_mask) | ((unsigned)t << shift);
                    const unsigned total = st.rs_above + above + st.hist[t];
                    if (total <= (unsigned)PUSH_CAP || shift == 0) {
                        st.rs_key = newprefix;
                        st.rs_done = 1;
                    } else {
                        st.rs_prefix = newprefix;
                        st.rs_need -= (int)above;
                        st.rs_above += above;
                        st.rs_shift = shift;
                    }
                }
                __syncthreads();
            }
            // drop candidates below the selected value
            const double tv = (double)JT<W>::value_of_bits(st.rs_key);
            const Acc c2 = JT<W>::cheap_min(tv, lb);
            int kept = 0;
            for (unsigned long long mm = mask; mm; mm &= mm - 1) {
                int bit = __ffsll(mm) - 1;
                int lid = (bit >> 2) * T * 4 + tid * 4 + (bit & 3);
                if (acc[lid] < c2) {
                    acc[lid] = (Acc)0;
                    mask &= ~(1ull << bit);
                } else {
                    kept++;
                }
            }
            for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
            __syncthreads();
            if (lane == 0) red_u[warp] = (unsigned long long)kept;
            __syncthreads();
            if (tid == 0) {
                unsigned long long t = 0;
                for (int w = 0; w < nwarps; w++) t += red_u[w];
                pending = (int)t;
            }
            __syncthreads();
        }
        const bool one_round = pending <= PUSH_CAP;
        const int per_round = one_round ? 64 : max(1, PUSH_CAP / T);
        while (true) {
            const u64 kth = st.kth;
            const u64 fl = st.floor;
            const double th0 = JT<W>::th_value(JT<W>::theta(st));
            const double th = one_round ? th0 : fmax(th0, JT<W>::score_of_bits((uint32_t)((kth > fl ? kth : fl) >> 32)));
            const Acc cm = one_round ? cmin : JT<W>::cheap_min(th, lb);
            // (a) each thread takes its marked entries: level 0 pushes directly; above
            //     level 0, entries within the per-vector bound go to the completion queue
            int budget = per_round;
            while (mask && budget > 0) {
                const int bit = __ffsll(mask) - 1;
                const int lid = (bit >> 2) * T * 4 + tid * 4 + (bit & 3);
                const Acc v = acc[lid];
                const int64_t gid = gbase + lid;
                if (v >= cm) {
                    if (level == 0) {
                        u64 key = make_key(JT<W>::score_bits(v), (uint32_t)gid);
                        if (key >= fl && key > kth) {
                            sortbuf[atomicAdd(&st.cnt, 1)] = key;
                            n_push++;
                        }
                    } else if (JT<W>::exact_ok(v, M, p.ubound[(int64_t)level * p.u_stride + gid], th, st.g)) {
                        const int slot = atomicAdd(&st.qcnt, 1);
                        if (slot >= CQ_CAP) break;   // queue full: keep this entry for the next pass
                        cq_gid[slot] = (uint32_t)gid;
                        cq_v[slot] = v;
                    }
                }
                acc[lid] = (Acc)0;
                mask &= mask - 1;
                budget--;
            }
            __syncthreads();
            // (b) completion of the queued entries (Algorithm 4's dot over the unindexed
            //     features), one warp per entry, lanes over the features
            const int nq = min(st.qcnt, CQ_CAP);
            for (int e = warp; e < nq; e += nwarps) {
                const int64_t gid = cq_gid[e];
                const int64_t j0 = p.s_indptr[gid];
                const int m = p.n_unidx[(int64_t)level * p.u_stride + gid];
                Acc res = (Acc)0;
                for (int q = lane; q < m; q += 32) {
                    const int32_t d = p.sp_d[j0 + q];
                    const Acc w = (Acc)((const W*)p.sp_w)[j0 + q];
                    const Acc rv = rden ? (Acc)rden[d] : lookup_r<W>(rf_d, rf_w, rn, d);
                    res += rv * w;
                }
                for (int o = 16; o > 0; o >>= 1) res += __shfl_xor_sync(0xffffffffu, res, o);
                if (lane == 0) {
                    n_comp++;
                    n_resf += m;
                    const Acc full = cq_v[e] + res;
                    u64 key = make_key(JT<W>::score_bits(full), (uint32_t)gid);
                    if (key >= fl && key > kth) {
                        sortbuf[atomicAdd(&st.cnt, 1)] = key;
                        n_push++;
                    }
                }
            }
            __syncthreads();
            if (tid == 0) st.qcnt = 0;
            const bool more = __syncthreads_or(mask != 0ull);
            if (one_round && more) continue;   // only the completion queue filled up
            if (tid == 0 && st.cnt > 0) st.n_merges++;
            merge_topk(topk, sortbuf, st, p.k);
            if (!more) break;
            if (tid == 0) st.n_rounds++;
        }
        }   // pend > 0
        // publish this group's k-th key as a floor for the other groups of the row
        if (tid == 0 && p.floor_keys && st.size == p.k) atomicMax(p.floor_keys + row, st.kth);
        // No barrier here: the next block's step 1 (warp 0) writes only state no other warp
        // reads after this block's select barrier (the candidate count is double-buffered),
        // and its barrier orders this block's deferred pushes before warp 0 drains them.
    }
    __syncthreads();
    if (nwarps >= 4) {   // the last block's deferred candidates
        if (warp == 0) drain();
        __syncthreads();
    }

    // ---- output ----
    if (out_mode == OUT_CARRY) {
        for (int q = tid; q < p.k; q += T) p.carry[row * p.k + q] = q < st.size ? topk[q] : 0ull;
    } else if (out_mode == OUT_FINAL) {
        for (int q = tid; q < p.k; q += T) {
            u64 key = q < st.size ? topk[q] : 0ull;
            int64_t o = row * p.k + q;
            p.out_ids[o] = key ? (int32_t)key_gid(key) : -1;
            ((uint32_t*)p.out_scores)[o] = key ? (uint32_t)(key >> 32) : 0u;
        }
        if (tid == 0 && p.n_found) p.n_found[row] = st.size;
        if (FXABLE && tid == 0 && st.size > 0) {   // one fixed-point unit against the smallest score returned
            const double th = (double)__uint_as_float((uint32_t)(topk[st.size - 1] >> 32));
            if ((double)st.fx_scale * th < 8388608.0) p.fx_flag[row] = 1;
        }
    } else {
        for (int q = tid; q < p.k; q += T)
            p.part_keys[((int64_t)row * p.groups + g) * p.k + q] = q < st.size ? topk[q] : 0ull;
    }
    // counters
    if (p.touched || p.stats) {
        const bool t0 = tid == 0;
        unsigned long long c[KNN_STATS_LEN] = {t0 ? st.n_steps : 0ull, n_cand, n_comp, n_push,
                                               t0 ? st.n_merges : 0ull, t0 ? st.n_rounds : 0ull, n_resf, n_post,
                                               n_add, (t0 && FXABLE) ? 1ull : 0ull};
#pragma unroll
        for (int j = 0; j < KNN_STATS_LEN; j++)
            for (int o = 16; o > 0; o >>= 1) c[j] += __shfl_xor_sync(0xffffffffu, c[j], o);
        if (lane == 0) {
            if (p.touched && c[7]) atomicAdd(p.touched, c[7]);
            if (p.stats)
                for (int j = 0; j < KNN_STATS_LEN; j++)
                    if (c[j]) atomicAdd(p.stats + j, c[j]);
        }
    }
}

template <class W, bool COUNT, bool BF, bool FX>
__global__ void __launch_bounds__(1024) k_join(JoinParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int row = p.row_list ? p.row_list[blockIdx.x] : (int)(blockIdx.x / p.groups);   // rows < 2^31
    const int g = p.row_list ? 0 : (int)(blockIdx.x - (unsigned)row * p.groups);
    if (p.groups == 1)
        join_row<W, COUNT, BF, FX>(p, row, 0, p.block_begin, p.block_end, p.carry_in != 0,
                                   p.carry_out ? OUT_CARRY : OUT_FINAL, smem);
    else
        join_row<W, COUNT, BF, FX>(p, row, g, g * p.blocks_per_group,
                                   min(p.n_blocks, (g + 1) * p.blocks_per_group), false, OUT_GROUP, smem);
}

// The posting count (stats, eq. 4 checks) costs a compare per posting, so it is
// compiled into a separate instance that runs only when a counter is requested; the
// fixed-point launch of float joins (fx) is an instance of its own as well.
using JoinKernel = void (*)(JoinParams);
static JoinKernel join_kernel(knn_dtype dt, bool count, bool bf, bool fx = false) {
    if (bf) {
        if (dt == KNN_U8) return count ? k_join<uint8_t, true, true, false> : k_join<uint8_t, false, true, false>;
        return count ? k_join<float, true, true, false> : k_join<float, false, true, false>;
    }
    if (dt == KNN_U8) return count ? k_join<uint8_t, true, false, false> : k_join<uint8_t, false, false, false>;
    if (fx) return count ? k_join<float, true, false, true> : k_join<float, false, false, true>;
    return count ? k_join<float, true, false, false> : k_join<float, false, false, false>;
}


// ---------------------------------------------------------------------------------
// batched form: many joins in one persistent launch
// ---------------------------------------------------------------------------------
constexpr int BATCH_MAX_JOBS = 64;   // jobs per launch (their parameters are kernel parameters)

// Work items (job, S-block group g, row) in rounds: round g holds group g of every job
// that has more than g groups, job by job, row by row.  Jobs are sorted by their group
// count (descending), so the jobs of a round are a prefix of the list, and the rounds
// fall into phases of equal prefix: phase h covers rounds [round[h], round[h+1]) with
// jobs [0, jobs[h]), rows_before[jobs[h]] items per round.
struct BatchParams {
    JoinParams p[BATCH_MAX_JOBS];                // each job's join (groups >= 1), groups descending
    long long rows_before[BATCH_MAX_JOBS + 1];   // rows of the jobs before this one
    long long phase_item[BATCH_MAX_JOBS + 1];    // first item of each phase; [n_phases] = all items
    int phase_round[BATCH_MAX_JOBS + 1];         // first round of each phase
    int phase_jobs[BATCH_MAX_JOBS];              // jobs in each phase's rounds
    int n_jobs, n_phases;
};
static_assert(sizeof(BatchParams) < 32000, "batch parameters must fit the kernel parameter space");

// Persistent CTAs take work items from one counter until it runs out.  A round's items
// of one job run side by side, so that group's postings stay in L2 while its rows read
// them (for all jobs of the round, when they share an index); each row's top-k is
// carried from group to group, and a row's next group comes a whole round of rows later.
// The job, S-block group and row of work item `it` (below the item count) of the round
// layout: its phase, its round within the phase, its job within the round.
__device__ __forceinline__ void decode_item(const BatchParams& bp, long long it, int& job, int& g, int64_t& row) {
    int h = 0, hi = bp.n_phases - 1;
    while (h < hi) {
        const int mid = (h + hi + 1) >> 1;
        if (bp.phase_item[mid] <= it) h = mid;
        else hi = mid - 1;
    }
    const long long per_round = bp.rows_before[bp.phase_jobs[h]];
    const long long off = it - bp.phase_item[h];
    const long long rr = off / per_round;
    g = bp.phase_round[h] + (int)rr;
    const long long q = off - rr * per_round;   // the item's place in its round
    int lo = 0;
    hi = bp.phase_jobs[h] - 1;
    while (lo < hi) {   // its job: the last one whose rows start at or before q
        const int mid = (lo + hi + 1) >> 1;
        if (bp.rows_before[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    job = lo;
    const int64_t li = q - bp.rows_before[lo];
    row = bp.p[lo].row_list ? (int64_t)bp.p[lo].row_list[li] : li;
}

constexpr long long BATCH_WAIT_SPINS = 1LL << 24;   // default bound: x ~128 ns sleeps, a few seconds
template <class W, bool COUNT, bool FX>
__global__ void __launch_bounds__(1024) k_join_batched(const __grid_constant__ BatchParams bp,
                                                       unsigned long long* __restrict__ head,
                                                       unsigned* __restrict__ err, long long wait_spins,
                                                       int no_publish, int flagged_only) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the item's job (-1: no items left), S-block group and row, decoded by thread 0
    __shared__ int s_job, s_g, s_row, s_ok;
    // flagged_only (the fp32 pass of a float batch, where few rows are flagged): warp 0
    // claims 32 items at a time and keeps those of flagged rows, taken in order
    __shared__ long long s_base;
    __shared__ unsigned s_mask;
    // otherwise each CTA claims one item ahead (s_next, -1: none yet), so that the claim's
    // round trip overlaps the loads that start the current item
    __shared__ long long s_next;
    // a finished group to announce (s_pub_job >= 0): its row's done counter becomes
    // s_pub_g + 1 once the next item's first barrier has ordered the CTA's writes of the
    // carried keys before it
    __shared__ int s_pub_job, s_pub_g, s_pub_row;
    const long long total = bp.phase_item[bp.n_phases];
    if (threadIdx.x == 0) {
        s_mask = 0u;
        s_next = -1;
        s_pub_job = -1;
    }
    for (;;) {
        __syncthreads();   // the previous item is finished with shared memory and its outputs
        if (threadIdx.x == 0 && s_pub_job >= 0) {   // announce it before anything that can wait
            __threadfence();
            asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(bp.p[s_pub_job].done + s_pub_row),
                         "r"(s_pub_g + 1)
                         : "memory");
            s_pub_job = -1;
        }
        long long it = total;   // thread 0: the item to run
        unsigned long long ahead = 0;
        if (flagged_only) {
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                for (;;) {
                    const unsigned mask = s_mask;
                    if (mask) {
                        if (lane == 0) {
                            it = s_base + (__ffs(mask) - 1);
                            s_mask = mask & (mask - 1);
                        }
                        break;
                    }
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(head, 32ull);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if ((long long)base >= total) break;
                    const long long my = (long long)base + lane;
                    bool fl = false;
                    if (my < total) {
                        int mj, mg;
                        int64_t mr;
                        decode_item(bp, my, mj, mg, mr);
                        fl = bp.p[mj].fx_flag[mr] != 0;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, fl);
                    if (lane == 0) {
                        s_base = (long long)base;
                        s_mask = m;
                    }
                    __syncwarp();
                }
            }
        } else if (threadIdx.x == 0) {
            it = s_next >= 0 ? s_next : (long long)atomicAdd(head, 1ull);
            // claims stay in order, and a CTA holds at most one item it has not started, larger
            // than the one it runs: the smallest unfinished item is always running
            if (it < total) ahead = atomicAdd(head, 1ull);
        }
        if (threadIdx.x == 0) {
            int lo = -1, g = 0, ok = 0;
            int64_t row = 0;
            if (it < total) {
                decode_item(bp, it, lo, g, row);
                const JoinParams& J = bp.p[lo];
                ok = 1;
                // the fp32 pass after a fixed-point one joins only the rows that pass
                // flagged: the other rows' items are skipped before any wait (none of them
                // publishes, and none of them waits)
                if (!FX && J.fx_flag && !J.fx_flag[row]) ok = 0;
                // group g continues from group g-1's top-k of this row: that item was taken
                // earlier (items are handed out in order -- singly, or in runs of 32 that the
                // claiming CTA takes in order), so it is running or done; wait for it with a
                // bounded spin, and give up with an error flag rather than hang
                if (ok && g > 0) {
                    int* dp = J.done + row;
                    long long spins = 0;
                    int v = 0;
                    for (;;) {
                        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(dp) : "memory");
                        if (v >= g || v < 0) break;   // ready, or an earlier group of this row failed
                        if (++spins > wait_spins) break;
                        __nanosleep(128);
                    }
                    ok = v >= g;
                    if (!ok) {
                        if (v >= 0) atomicOr(err, 1u);   // (v < 0: an earlier group's failure, flagged there)
                        atomicExch(dp, -1);              // later groups of this row give up at once
                    }
                }
                // the shared-memory layout holds rows of up to max_r_nnz features, fixed when
                // the batch was made: a row that has grown since is not joined (error flag 2)
                if (ok && J.r_indptr[row + 1] - J.r_indptr[row] > J.max_r_nnz) {
                    ok = 0;
                    atomicOr(err, 2u);
                    if (J.done) atomicExch(J.done + row, -1);
                }
            }
            s_job = lo;
            s_g = g;
            s_row = (int)row;
            s_ok = ok;
            if (!flagged_only) s_next = it < total ? (long long)ahead : total;
        }
        __syncthreads();
        const int job = s_job;
        if (job < 0) break;
        if (!s_ok) continue;
        const JoinParams& J = bp.p[job];
        const int g = s_g;
        const int64_t row = s_row;
        const bool last = g == J.groups - 1;
        // a row the fixed-point pass flagged early (no usable scale) only passes its groups on
        const bool skip = FX && g > 0 && *(volatile uint8_t*)(J.fx_flag + row);
        if (!skip)
            join_row<W, COUNT, false, FX>(J, row, g, g * J.blocks_per_group,
                                          min(J.n_blocks, (g + 1) * J.blocks_per_group), g > 0,
                                          last ? OUT_FINAL : OUT_CARRY, smem);
        if (!last && !no_publish && threadIdx.x == 0) {   // announced after the next barrier
            // the item, re-read: nothing of it needs to stay in registers across the join
            s_pub_job = *(volatile int*)&s_job;
            s_pub_g = *(volatile int*)&s_g;
            s_pub_row = *(volatile int*)&s_row;
        }
    }
}

using BatchKernel = void (*)(const BatchParams, unsigned long long*, unsigned*, long long, int, int);
static BatchKernel batch_kernel(knn_dtype dt, bool count, bool fx = false) {
    if (dt == KNN_U8) return count ? k_join_batched<uint8_t, true, false> : k_join_batched<uint8_t, false, false>;
    if (fx) return count ? k_join_batched<float, true, true> : k_join_batched<float, false, true>;
    return count ? k_join_batched<float, true, false> : k_join_batched<float, false, false>;
}

// A layout within this leaves room for two CTAs of 512 threads per SM.
constexpr size_t TWO_CTA_SMEM = 110 * 1024;

// Bytes of the dense copy of r's weights (uint8, dimension up to 32768) that a CTA keeps
// for completions when, with rows of up to max_r features, the layout still leaves room
// for two CTAs per SM; else 0 (completions then search r's sorted features).
static int rden_fitting(const knn_index* ix, int nb, int max_r) {
    if (ix->dtype != KNN_U8 || ix->dim > 32768) return 0;
    const int rd = (int)((ix->dim + 15) & ~15);
    return smem_layout(nb, max_r, rd).total <= TWO_CTA_SMEM ? rd : 0;
}

// The longest row length q < max_r whose layout fits TWO_CTA_SMEM (0 if none from 32 up),
// with its dense-copy size in *rden.
static int short_row_limit(const knn_index* ix, int nb, int max_r, int* rden) {
    for (int q = max_r - 1; q >= 32; q--) {
        const int rd = rden_fitting(ix, nb, q);
        if (smem_layout(nb, q, rd).total <= TWO_CTA_SMEM) {
            *rden = rd;
            return q;
        }
    }
    *rden = 0;
    return 0;
}

// Rows with at most r_short features to the front of `lists`, the others to the back
// (each part in no particular order); counts[0] / counts[1] count them.
__global__ void k_split_rows(const int64_t* __restrict__ indptr, int64_t n, int32_t r_short,
                             int32_t* __restrict__ lists, int32_t* __restrict__ counts) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (indptr[i + 1] - indptr[i] <= r_short) lists[atomicAdd(&counts[0], 1)] = (int32_t)i;
    else lists[n - 1 - atomicAdd(&counts[1], 1)] = (int32_t)i;
}

// one CTA per row: top-k of the groups' lists
__global__ void k_merge_groups(const u64* __restrict__ part, int64_t n_rows, int groups, int k, int P,
                               int32_t* out_ids, uint32_t* out_scores, int32_t* n_found) {
    extern __shared__ u64 buf[];
    int64_t row = blockIdx.x;
    int n = groups * k;
    for (int i = threadIdx.x; i < P; i += blockDim.x) buf[i] = i < n ? part[row * n + i] : 0ull;
    __syncthreads();
    cta_bitonic_desc(buf, P);
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
        u64 key = buf[q];
        out_ids[row * k + q] = key ? (int32_t)key_gid(key) : -1;
        out_scores[row * k + q] = key ? (uint32_t)(key >> 32) : 0u;
    }
    if (n_found && threadIdx.x == 0) {
        int c = 0;
        for (int q = 0; q < k; q++) c += buf[q] != 0ull;
        n_found[row] = c;
    }
}

// Top-k of the union of several S shards' lists for the same queries: keys (score,
// global id) from every part, a CTA bitonic sort per row, the first k kept.
struct MergeParts {
    const int32_t* ids[KNN_MAX_PARTS];
    const uint32_t* scores[KNN_MAX_PARTS];   // int32 or float bits (both order like the scores)
    int64_t offset[KNN_MAX_PARTS];           // the shard's first S id
    int32_t n_parts;
};
static_assert(sizeof(MergeParts) < 4000, "merge parameters must fit the kernel parameter space");

__global__ void k_merge_parts(const __grid_constant__ MergeParts mp, int k, int P, int32_t* __restrict__ out_ids,
                              uint32_t* __restrict__ out_scores) {
    extern __shared__ u64 buf[];
    const int64_t row = blockIdx.x;
    const int n = mp.n_parts * k;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        u64 key = 0ull;
        if (i < n) {
            const int part = i / k, q = i - part * k;
            const int32_t id = mp.ids[part][row * k + q];
            if (id >= 0) key = make_key(mp.scores[part][row * k + q], (uint32_t)(id + mp.offset[part]));
        }
        buf[i] = key;
    }
    __syncthreads();
    cta_bitonic_desc(buf, P);
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
        const u64 key = buf[q];
        out_ids[row * k + q] = key ? (int32_t)key_gid(key) : -1;
        out_scores[row * k + q] = key ? (uint32_t)(key >> 32) : 0u;
    }
}

// ---------------------------------------------------------------------------------
// Out-of-core joins.  An index moved to host memory (knn_index_to_host) is streamed
// launch by launch: each S-block-synchronous launch's slice of the index -- its bins,
// postings and the per-vector arrays of its S range -- is copied into one of two device
// staging sets on a copy stream while the previous launch runs, so the kernels read it
// from device memory and L2 as usual (Algorithm 1's block nested loop with the S blocks
// fetched from the host).
// ---------------------------------------------------------------------------------
struct StagedIndex {
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    uint32_t* binoff[2] = {nullptr, nullptr};
    uint8_t* post[2] = {nullptr, nullptr};
    int64_t* sind[2] = {nullptr, nullptr};
    int32_t* spd[2] = {nullptr, nullptr};
    uint8_t* spw[2] = {nullptr, nullptr};
    uint16_t* nun[2] = {nullptr, nullptr};
    uint32_t* ub[2] = {nullptr, nullptr};
    int64_t rows_cap = 0;   // S vectors per launch: the staged arrays' level stride
    ~StagedIndex() {
        for (int i = 0; i < 2; i++) {
            if (copied[i]) cudaEventDestroy(copied[i]);
            if (used[i]) cudaEventDestroy(used[i]);
        }
        if (copy) cudaStreamDestroy(copy);
    }
};

struct SliceRange {
    int64_t b0, b1, g0, g1, p0, p1, f0, f1;   // blocks, S vectors, postings, features
};

// S blocks per launch (or per batched work item) when the caller gives none: as many as
// keep one launch's postings within ~48 MB, so that they stay in the 129 MB L2 while
// every row of the launch reads them; at most 16.  (Spectrum-shaped uint8 S: 2.6 MB of
// postings per block -> 16; the float workload at |S| = 10M: 7.9 MB per block -> 6.)
static int default_blocks_per_launch(const knn_index* ix) {
    const double post_bytes = ix->dtype == KNN_U8 ? 4.0 : 8.0;
    const double per_block = (double)ix->n_postings * post_bytes / (double)std::max(1, ix->n_blocks);
    const int b = per_block > 0.0 ? (int)std::min(16.0, 48.0e6 / per_block) : 16;
    return std::max(1, b);
}

// Level margin when the caller gives none (section 4.2's trade of postings scanned against
// completions): 0.3 for uint8 scores; 0.2 for float scores, whose completions look r's
// weights up by binary search (measured best on the float workload at |S| = 10M).
static float default_margin(knn_dtype dt) { return dt == KNN_F32 ? 0.2f : 0.3f; }

// the largest L2 norm of an S vector as a float not below it (0 when unknown or not finite)
static float maxnorm_up(const knn_index* ix) {
    const double v = ix->max_row_norm;
    if (!(v > 0.0) || v > 1e37) return 0.0f;
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, 3.4e38f);
    return f;
}

static SliceRange slice_of(const knn_index* ix, int li, int per_launch) {
    SliceRange r;
    r.b0 = (int64_t)li * per_launch;
    r.b1 = std::min<int64_t>(ix->n_blocks, r.b0 + per_launch);
    r.g0 = r.b0 << ix->block_shift;
    r.g1 = std::min<int64_t>(ix->n_rows, r.b1 << ix->block_shift);
    const uint32_t* bo = (const uint32_t*)ix->host_arrays[0];
    const int64_t* si = (const int64_t*)ix->host_arrays[2];
    const int64_t lists = (int64_t)ix->dim * ix->n_levels;
    r.p0 = bo[r.b0 * lists];
    r.p1 = bo[r.b1 * lists];
    r.f0 = si[r.g0];
    r.f1 = si[r.g1];
    return r;
}

static knn_status stage_setup(const knn_index* ix, int per_launch, int n_launch, Buffers& tmp, StagedIndex& st) {
    const size_t psz = ix->dtype == KNN_U8 ? 4 : 8, wsz = ix->dtype == KNN_U8 ? 1 : 4;
    int64_t post_cap = 1, feat_cap = 1;
    for (int li = 0; li < n_launch; li++) {
        const SliceRange r = slice_of(ix, li, per_launch);
        post_cap = std::max(post_cap, r.p1 - r.p0);
        feat_cap = std::max(feat_cap, r.f1 - r.f0);
    }
    st.rows_cap = (int64_t)per_launch << ix->block_shift;
    const size_t bins = (size_t)per_launch * ix->dim * ix->n_levels + 1;
    for (int i = 0; i < 2; i++) {
        KNN_TRY(tmp.get(&st.binoff[i], bins));
        KNN_TRY(tmp.get(&st.post[i], (size_t)post_cap * psz));
        KNN_TRY(tmp.get(&st.sind[i], (size_t)st.rows_cap + 1));
        KNN_TRY(tmp.get(&st.spd[i], (size_t)feat_cap));
        KNN_TRY(tmp.get(&st.spw[i], (size_t)feat_cap * wsz));
        KNN_TRY(tmp.get(&st.nun[i], (size_t)st.rows_cap * ix->n_levels));
        KNN_TRY(tmp.get(&st.ub[i], (size_t)st.rows_cap * ix->n_levels));
        KNN_CUDA_TRY(cudaEventCreateWithFlags(&st.copied[i], cudaEventDisableTiming));
        KNN_CUDA_TRY(cudaEventCreateWithFlags(&st.used[i], cudaEventDisableTiming));
    }
    KNN_CUDA_TRY(cudaStreamCreateWithFlags(&st.copy, cudaStreamNonBlocking));
    return KNN_OK;
}

// copies launch li's slice into set li & 1 (after the launch that last used that set)
static knn_status stage_copy(const knn_index* ix, int li, int per_launch, bool wait_used, StagedIndex& st) {
    const int set = li & 1;
    const size_t psz = ix->dtype == KNN_U8 ? 4 : 8, wsz = ix->dtype == KNN_U8 ? 1 : 4;
    const SliceRange r = slice_of(ix, li, per_launch);
    const int64_t lists = (int64_t)ix->dim * ix->n_levels;
    const int64_t rows = r.g1 - r.g0;
    if (wait_used) KNN_CUDA_TRY(cudaStreamWaitEvent(st.copy, st.used[set], 0));
    const uint8_t* const* h = (const uint8_t* const*)ix->host_arrays.data();
    KNN_CUDA_TRY(cudaMemcpyAsync(st.binoff[set], h[0] + 4 * r.b0 * lists, 4 * ((r.b1 - r.b0) * lists + 1),
                                 cudaMemcpyHostToDevice, st.copy));
    KNN_CUDA_TRY(cudaMemcpyAsync(st.post[set], h[1] + psz * r.p0, psz * (r.p1 - r.p0), cudaMemcpyHostToDevice,
                                 st.copy));
    KNN_CUDA_TRY(cudaMemcpyAsync(st.sind[set], h[2] + 8 * r.g0, 8 * (rows + 1), cudaMemcpyHostToDevice, st.copy));
    KNN_CUDA_TRY(cudaMemcpyAsync(st.spd[set], h[3] + 4 * r.f0, 4 * (r.f1 - r.f0), cudaMemcpyHostToDevice, st.copy));
    KNN_CUDA_TRY(cudaMemcpyAsync(st.spw[set], h[4] + wsz * r.f0, wsz * (r.f1 - r.f0), cudaMemcpyHostToDevice,
                                 st.copy));
    // per level: the S range's entries, packed at a stride of rows_cap
    KNN_CUDA_TRY(cudaMemcpy2DAsync(st.nun[set], 2 * st.rows_cap, h[5] + 2 * r.g0, 2 * ix->n_rows, 2 * rows,
                                   ix->n_levels, cudaMemcpyHostToDevice, st.copy));
    KNN_CUDA_TRY(cudaMemcpy2DAsync(st.ub[set], 4 * st.rows_cap, h[6] + 4 * r.g0, 4 * ix->n_rows, 4 * rows,
                                   ix->n_levels, cudaMemcpyHostToDevice, st.copy));
    KNN_CUDA_TRY(cudaEventRecord(st.copied[set], st.copy));
    return KNN_OK;
}

// points the join's index arrays at launch li's staged slice (absolute indices still
// work: every pointer is shifted back by the slice's first index)
static void stage_params(const knn_index* ix, int li, int per_launch, const StagedIndex& st, JoinParams& p) {
    const int set = li & 1;
    const size_t psz = ix->dtype == KNN_U8 ? 4 : 8, wsz = ix->dtype == KNN_U8 ? 1 : 4;
    const SliceRange r = slice_of(ix, li, per_launch);
    const int64_t lists = (int64_t)ix->dim * ix->n_levels;
    p.binoff = st.binoff[set] - r.b0 * lists;
    p.postings = st.post[set] - psz * r.p0;
    p.s_indptr = st.sind[set] - r.g0;
    p.sp_d = st.spd[set] - r.f0;
    p.sp_w = st.spw[set] - wsz * r.f0;
    p.n_unidx = st.nun[set] - r.g0;
    p.ubound = st.ub[set] - r.g0;
    p.u_stride = st.rows_cap;
}

}  // namespace knn

using namespace knn;

extern "C" knn_status knn_join(const knn_index* ix, const knn_csr* R, int32_t k, const knn_join_opts* opts,
                               int32_t* out_ids, void* out_scores, void* stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!ix) return fail(KNN_EINVAL, "index is NULL");
    if (!R) return fail(KNN_EINVAL, "R is NULL");
    if (k < 1) return fail(KNN_EINVAL, "k must be >= 1");
    if (k > KNN_MAX_K) return fail(KNN_EUNSUPPORTED, "k > %d", KNN_MAX_K);
    if (R->dim != ix->dim) return fail(KNN_EINVAL, "R has dim %d, the index %d", R->dim, ix->dim);
    if (R->dtype != ix->dtype) return fail(KNN_EINVAL, "R and the index have different dtypes");
    knn_join_opts o = {};
    if (opts) o = *opts;
    if (o.mode != KNN_MODE_IIIB && o.mode != KNN_MODE_IIB && o.mode != KNN_MODE_BF)
        return fail(KNN_EINVAL, "unknown mode");
    if (R->n_rows > 0 && (!out_ids || !out_scores)) return fail(KNN_EINVAL, "outputs are NULL");

    Buffers tmp(stream);
    DevCSR r;
    KNN_TRY(prepare_csr(R, stream, tmp, !o.skip_validation, true, &r));
    if (r.n_rows == 0) return KNN_OK;
    if (ix->dtype == KNN_U8) {
        double bound = std::min(r.max_row_sum * ix->max_w, ix->max_row_sum * r.max_w);
        if (bound >= 2147483647.0) return fail(KNN_EUNSUPPORTED, "uint8 scores could overflow int32");
    }
    const int nb = ix->block_size;
    int T = o.threads ? o.threads : 512;
    if (T < 128 || T > 1024 || (T & 31)) return fail(KNN_EINVAL, "threads must be a multiple of 32 in [128, 1024]");
    // each thread owns 4 accumulator entries per chunk and a 64-bit candidate mask:
    // T * 4 <= nb and nb / (T * 4) <= 16 (nb and T are powers of two times 32)
    while (nb / (T * 4) > 16) T *= 2;
    while (T > 32 && nb < T * 4) T /= 2;
    if (nb % (T * 4) || nb / (T * 4) > 16 || T > 1024)
        return fail(KNN_EUNSUPPORTED, "block size %d does not fit %d threads", nb, T);
    const int max_r = std::max(1, r.max_row_nnz);
    // r's weights kept densely for completions (uint8, dimension up to 32768) when it
    // still leaves room for two CTAs per SM
    const int rden_dim = rden_fitting(ix, nb, max_r);
    SmemLayout L = smem_layout(nb, max_r, rden_dim);
    int dev = 0;
    KNN_CUDA_TRY(cudaGetDevice(&dev));
    int smem_optin = 0, n_sm = 0;
    KNN_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    KNN_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const size_t static_smem = sizeof(CtaState) + 32 * 8 * 2 + 64;
    if (L.total + static_smem > (size_t)smem_optin)
        return fail(KNN_EUNSUPPORTED, "a row with %d features and S blocks of %d need %zu bytes of shared memory (> %d)",
                    max_r, nb, L.total, smem_optin);

    // groups of S blocks per row
    int per_sm = std::max(1, std::min((int)(228 * 1024 / (L.total + static_smem + 1024)), 2048 / T));
    int groups = o.s_groups;
    if (groups <= 0) {
        int64_t target = (int64_t)n_sm * per_sm * 4;
        groups = (int)std::min<int64_t>(ix->n_blocks, std::max<int64_t>(1, ceil_div(target, r.n_rows)));
    }
    groups = std::max(1, std::min(groups, ix->n_blocks));
    groups = std::min(groups, std::max(1, 4096 / k));
    if (ix->host_bytes) groups = 1;   // a host-resident index is streamed launch by launch
    int bpg = (int)ceil_div(ix->n_blocks, groups);
    groups = (int)ceil_div(ix->n_blocks, bpg);
    if ((int64_t)r.n_rows * groups > (int64_t)INT32_MAX) return fail(KNN_EUNSUPPORTED, "too many rows");

    int32_t* d_ids = out_ids;
    uint32_t* d_sc = (uint32_t*)out_scores;
    if (o.outputs_on_host) {
        KNN_TRY(tmp.get(&d_ids, (size_t)r.n_rows * k));
        KNN_TRY(tmp.get(&d_sc, (size_t)r.n_rows * k));
    }
    JoinParams p;
    memset(&p, 0, sizeof(p));
    p.n_rows = r.n_rows;
    p.r_indptr = r.indptr;
    p.r_idx = r.indices;
    p.r_val = r.values;
    p.n_s = ix->n_rows;
    p.dim = ix->dim;
    p.n_blocks = ix->n_blocks;
    p.n_levels = ix->n_levels;
    p.block_shift = ix->block_shift;
    p.binoff = ix->binoff;
    p.postings = ix->postings;
    p.s_indptr = ix->s_indptr;
    p.sp_d = ix->sp_d;
    p.sp_w = ix->sp_w;
    p.n_unidx = ix->n_unidx;
    p.ubound = ix->ubound;
    p.u_stride = ix->n_rows;
    p.s_maxnorm = maxnorm_up(ix);
    memcpy(p.levels, ix->levels, sizeof(p.levels));
    p.k = k;
    p.groups = groups;
    p.blocks_per_group = bpg;
    p.iiib = o.mode == KNN_MODE_IIIB && ix->n_levels > 1;
    p.bf = o.mode == KNN_MODE_BF;
    p.max_r_nnz = max_r;
    p.rden_dim = rden_dim;
    p.init_thr = o.init_threshold;
    p.out_ids = d_ids;
    p.out_scores = d_sc;
    p.n_found = o.n_found;
    p.touched = (unsigned long long*)o.postings_scanned;
    p.stats = (unsigned long long*)o.stats;
    p.level_margin = o.level_margin > 0.0f ? o.level_margin : default_margin(ix->dtype);
    if (!(p.level_margin <= 1.0f)) return fail(KNN_EINVAL, "level_margin must be in (0, 1]");
    if (groups > 1) {
        KNN_TRY(tmp.get(&p.part_keys, (size_t)r.n_rows * groups * k));
        KNN_TRY(tmp.get(&p.floor_keys, (size_t)r.n_rows));
        KNN_CUDA_TRY(cudaMemsetAsync(p.floor_keys, 0, sizeof(u64) * r.n_rows, stream));
    }
    int64_t grid = r.n_rows * groups;
    const JoinKernel kern = join_kernel(ix->dtype, p.touched || p.stats, p.bf != 0);
    KNN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    // One group per row: S-block-synchronous launches.  Every launch walks all rows over
    // the same few S blocks, so their postings stay in L2 while all rows read them.
    int per_launch = groups == 1 ? (o.blocks_per_launch > 0 ? o.blocks_per_launch : default_blocks_per_launch(ix))
                                 : ix->n_blocks;
    per_launch = std::min(per_launch, ix->n_blocks);
    const int n_launch = groups == 1 ? (int)ceil_div(ix->n_blocks, per_launch) : 1;
    if (n_launch > 1) KNN_TRY(tmp.get(&p.carry, (size_t)r.n_rows * k));
    StagedIndex staged;
    const bool streamed = ix->host_bytes != 0;
    if (streamed) {
        KNN_TRY(stage_setup(ix, per_launch, n_launch, tmp, staged));
        KNN_TRY(stage_copy(ix, 0, per_launch, false, staged));
    }
    // Float joins with one group per row sum their scans in fixed point (fx_decide): every
    // S-block launch runs the fixed-point instance, and one fp32 launch over all S blocks
    // then joins again the rows it flagged (no usable scale, or a result whose fixed-point
    // error is not small enough against its scores); the other rows exit at once.
    const bool use_fx = ix->dtype == KNN_F32 && !p.bf && groups == 1 && !streamed && p.s_maxnorm > 0.0f &&
                        !o.no_fixed_point;
    JoinKernel kern_run = kern;
    if (use_fx) {
        kern_run = join_kernel(ix->dtype, p.touched || p.stats, false, true);
        KNN_CUDA_TRY(cudaFuncSetAttribute(kern_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
        KNN_TRY(tmp.get(&p.fx_flag, (size_t)r.n_rows));
        KNN_CUDA_TRY(cudaMemsetAsync(p.fx_flag, 0, (size_t)r.n_rows, stream));
    }
    // With one group per row, when the longest rows need a shared-memory layout that
    // leaves room for one CTA per SM only, every launch runs in two parts: the rows with at
    // most r_short features (the most a layout within 110 KB -- two CTAs per SM -- holds)
    // with that layout, then the longer rows with the full one.  Rows are independent, so
    // splitting them changes nothing but occupancy.
    int r_short = 0, rden_short = 0, n_short = 0;
    int32_t* row_lists = nullptr;
    size_t smem_short = 0;
    if (groups == 1 && r.n_rows > 1 && L.total > TWO_CTA_SMEM) {
        r_short = short_row_limit(ix, nb, max_r, &rden_short);
        if (r_short > 0) {
            smem_short = smem_layout(nb, r_short, rden_short).total;
            int32_t* counts = nullptr;
            KNN_TRY(tmp.get(&row_lists, (size_t)r.n_rows));
            KNN_TRY(tmp.get(&counts, 2));
            KNN_CUDA_TRY(cudaMemsetAsync(counts, 0, 2 * sizeof(int32_t), stream));
            k_split_rows<<<launch_blocks(r.n_rows, 256), 256, 0, stream>>>(r.indptr, r.n_rows, r_short, row_lists,
                                                                          counts);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
            int32_t hc[2] = {0, 0};
            KNN_CUDA_TRY(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, stream));
            KNN_CUDA_TRY(cudaStreamSynchronize(stream));
            n_short = hc[0];
        }
    }
    auto launch_rows = [&](JoinKernel kf, const JoinParams& q) -> knn_status {
        if (!r_short) {
            kf<<<(unsigned)grid, T, L.total, stream>>>(q);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
            return KNN_OK;
        }
        if (n_short > 0) {
            JoinParams qs = q;
            qs.row_list = row_lists;
            qs.max_r_nnz = r_short;
            qs.rden_dim = rden_short;
            kf<<<(unsigned)n_short, T, smem_short, stream>>>(qs);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
        }
        if (n_short < r.n_rows) {
            JoinParams ql = q;
            ql.row_list = row_lists + n_short;
            kf<<<(unsigned)(r.n_rows - n_short), T, L.total, stream>>>(ql);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
        }
        return KNN_OK;
    };
    for (int li = 0; li < n_launch; li++) {
        p.block_begin = li * per_launch;
        p.block_end = std::min(ix->n_blocks, (li + 1) * per_launch);
        p.carry_in = li > 0;
        p.carry_out = li + 1 < n_launch;
        if (streamed) {
            // the next slice goes into the other set once the launch before this one is done
            if (li + 1 < n_launch) KNN_TRY(stage_copy(ix, li + 1, per_launch, li >= 1, staged));
            KNN_CUDA_TRY(cudaStreamWaitEvent(stream, staged.copied[li & 1], 0));
            stage_params(ix, li, per_launch, staged, p);
        }
        KNN_TRY(launch_rows(kern_run, p));
        if (streamed) KNN_CUDA_TRY(cudaEventRecord(staged.used[li & 1], stream));
    }
    if (use_fx) {   // the fp32 re-join of the flagged rows, over all S blocks in one launch
        p.block_begin = 0;
        p.block_end = ix->n_blocks;
        p.carry_in = 0;
        p.carry_out = 0;
        KNN_TRY(launch_rows(kern, p));
    }
    if (groups > 1) {
        int P = 2;
        while (P < groups * k) P <<= 1;
        KNN_CUDA_TRY(cudaFuncSetAttribute(k_merge_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, P * 8));
        k_merge_groups<<<(unsigned)r.n_rows, 256, P * 8, stream>>>(p.part_keys, r.n_rows, groups, k, P, d_ids, d_sc,
                                                                    o.n_found);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    if (o.outputs_on_host) {
        KNN_CUDA_TRY(cudaMemcpyAsync(out_ids, d_ids, sizeof(int32_t) * r.n_rows * k, cudaMemcpyDeviceToHost, stream));
        KNN_CUDA_TRY(cudaMemcpyAsync(out_scores, d_sc, sizeof(uint32_t) * r.n_rows * k, cudaMemcpyDeviceToHost, stream));
        KNN_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return KNN_OK;
}

extern "C" knn_status knn_merge_topk(int32_t n_parts, const int32_t* const* part_ids, const void* const* part_scores,
                                     const int64_t* id_offset, int64_t n_rows, int32_t k, knn_dtype dtype,
                                     int32_t* out_ids, void* out_scores, void* stream_) {
    if (n_parts < 1 || n_parts > KNN_MAX_PARTS) return fail(KNN_EINVAL, "n_parts must be in [1, %d]", KNN_MAX_PARTS);
    if (k < 1 || k > KNN_MAX_K) return fail(KNN_EINVAL, "k must be in [1, %d]", KNN_MAX_K);
    if (dtype != KNN_U8 && dtype != KNN_F32) return fail(KNN_EINVAL, "unknown dtype");
    if (n_rows < 0) return fail(KNN_EINVAL, "n_rows < 0");
    if (n_rows == 0) return KNN_OK;
    if (!part_ids || !part_scores || !id_offset || !out_ids || !out_scores) return fail(KNN_EINVAL, "NULL argument");
    MergeParts mp;
    memset(&mp, 0, sizeof(mp));
    mp.n_parts = n_parts;
    for (int i = 0; i < n_parts; i++) {
        if (!part_ids[i] || !part_scores[i]) return fail(KNN_EINVAL, "part %d is NULL", i);
        if (id_offset[i] < 0 || id_offset[i] > 0x7FFFFFFF) return fail(KNN_EINVAL, "id offset of part %d", i);
        mp.ids[i] = part_ids[i];
        mp.scores[i] = (const uint32_t*)part_scores[i];
        mp.offset[i] = id_offset[i];
    }
    if (n_rows > (int64_t)INT32_MAX) return fail(KNN_EUNSUPPORTED, "too many rows");
    int P = 2;
    while (P < n_parts * k) P <<= 1;
    cudaStream_t stream = (cudaStream_t)stream_;
    KNN_CUDA_TRY(cudaFuncSetAttribute(k_merge_parts, cudaFuncAttributeMaxDynamicSharedMemorySize, P * 8));
    k_merge_parts<<<(unsigned)n_rows, 256, (size_t)P * 8, stream>>>(mp, k, P, out_ids, (uint32_t*)out_scores);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    return KNN_OK;
}

// ---------------------------------------------------------------------------------
// knn_join_noalloc: the join for callers that must not allocate device memory
//
// Some callers cannot have a library allocate device memory while they run: a server
// that has split the whole GPU between its own fixed pools and would see a foreign
// allocation fail or fragment them, or a latency-critical loop where an allocation (or
// the device-wide synchronisation that freeing memory can cause) is not acceptable.
// This entry point runs the same k_join kernel as knn_join, but its scratch -- the
// per-row check record and the top-k keys each row carries from one S-block launch to
// the next -- lives in one file-scope __device__ array of KNN_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads this library holds that array until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the array's
// device address with cudaGetSymbolAddress and caches it.  Every call also synchronises
// its stream (it reads R's size back and, when validating, R's check record).  All calls
// share the one array and it keeps
// the contents of the last call, so two calls whose work overlaps on the GPU (other
// streams, other host threads) race on it; the check record is cleared on each call,
// and every carried key is written before it is read.
// ---------------------------------------------------------------------------------
namespace knn {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KNN_NOALLOC_SCRATCH_BYTES];

constexpr size_t NOALLOC_HEADER = 256;   // check record of R
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// device address of the scratch array on the current device (looked up once per device)
static knn_status noalloc_scratch(void** out) {
    int dev = 0;
    KNN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(KNN_EUNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(KNN_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return KNN_OK;
}

}  // namespace knn

extern "C" knn_status knn_join_noalloc(const knn_index* ix, const knn_csr* R, int32_t k, const knn_join_opts* opts,
                                       int32_t* out_ids, void* out_scores, void* stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!ix) return fail(KNN_EINVAL, "index is NULL");
    if (!R) return fail(KNN_EINVAL, "R is NULL");
    if (k < 1) return fail(KNN_EINVAL, "k must be >= 1");
    if (k > KNN_MAX_K) return fail(KNN_EUNSUPPORTED, "k > %d", KNN_MAX_K);
    if (R->dim != ix->dim) return fail(KNN_EINVAL, "R has dim %d, the index %d", R->dim, ix->dim);
    if (R->dtype != ix->dtype) return fail(KNN_EINVAL, "R and the index have different dtypes");
    if (!R->on_device) return fail(KNN_EINVAL, "knn_join_noalloc needs R in device memory (on_device = 1)");
    knn_join_opts o = {};
    if (opts) o = *opts;
    if (o.mode != KNN_MODE_IIIB && o.mode != KNN_MODE_IIB && o.mode != KNN_MODE_BF)
        return fail(KNN_EINVAL, "unknown mode");
    if (o.outputs_on_host) return fail(KNN_EINVAL, "knn_join_noalloc writes device outputs only");
    if (R->n_rows < 0) return fail(KNN_EINVAL, "n_rows < 0");
    if (R->n_rows > 0 && (!out_ids || !out_scores)) return fail(KNN_EINVAL, "outputs are NULL");
    const size_t carry_cap = (KNN_NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER) / sizeof(u64);
    if ((uint64_t)R->n_rows * (uint64_t)k > carry_cap)
        return fail(KNN_EUNSUPPORTED,
                    "knn_join_noalloc: n_rows * k = %lld exceeds the %zu top-k keys its %d-byte scratch holds",
                    (long long)R->n_rows * k, carry_cap, (int)KNN_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    KNN_TRY(noalloc_scratch(&scratch));

    DevCSR r;
    KNN_TRY(check_device_csr_into(R, scratch, !o.skip_validation, stream, &r));
    if (r.n_rows == 0) return KNN_OK;
    if (ix->dtype == KNN_U8) {
        double bound = std::min(r.max_row_sum * ix->max_w, ix->max_row_sum * r.max_w);
        if (bound >= 2147483647.0) return fail(KNN_EUNSUPPORTED, "uint8 scores could overflow int32");
    }
    const int nb = ix->block_size;
    int T = o.threads ? o.threads : 512;
    if (T < 128 || T > 1024 || (T & 31)) return fail(KNN_EINVAL, "threads must be a multiple of 32 in [128, 1024]");
    while (nb / (T * 4) > 16) T *= 2;
    while (T > 32 && nb < T * 4) T /= 2;
    if (nb % (T * 4) || nb / (T * 4) > 16 || T > 1024)
        return fail(KNN_EUNSUPPORTED, "block size %d does not fit %d threads", nb, T);
    const int max_r = std::max(1, r.max_row_nnz);
    // r's weights kept densely for completions (uint8, dimension up to 32768) when it
    // still leaves room for two CTAs per SM
    const int rden_dim = rden_fitting(ix, nb, max_r);
    SmemLayout L = smem_layout(nb, max_r, rden_dim);
    int dev = 0, smem_optin = 0;
    KNN_CUDA_TRY(cudaGetDevice(&dev));
    KNN_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (L.total + sizeof(CtaState) + 32 * 8 * 2 + 64 > (size_t)smem_optin)
        return fail(KNN_EUNSUPPORTED, "a row with %d features and S blocks of %d need %zu bytes of shared memory (> %d)",
                    max_r, nb, L.total, smem_optin);
    if (r.n_rows > (int64_t)INT32_MAX) return fail(KNN_EUNSUPPORTED, "too many rows");

    JoinParams p;
    memset(&p, 0, sizeof(p));
    p.n_rows = r.n_rows;
    p.r_indptr = r.indptr;
    p.r_idx = r.indices;
    p.r_val = r.values;
    p.n_s = ix->n_rows;
    p.dim = ix->dim;
    p.n_blocks = ix->n_blocks;
    p.n_levels = ix->n_levels;
    p.block_shift = ix->block_shift;
    p.binoff = ix->binoff;
    p.postings = ix->postings;
    p.s_indptr = ix->s_indptr;
    p.sp_d = ix->sp_d;
    p.sp_w = ix->sp_w;
    p.n_unidx = ix->n_unidx;
    p.ubound = ix->ubound;
    p.u_stride = ix->n_rows;
    p.s_maxnorm = maxnorm_up(ix);
    memcpy(p.levels, ix->levels, sizeof(p.levels));
    p.k = k;
    p.groups = 1;   // one group per row: the only schedule whose scratch is the carry buffer
    p.blocks_per_group = ix->n_blocks;
    p.iiib = o.mode == KNN_MODE_IIIB && ix->n_levels > 1;
    p.bf = o.mode == KNN_MODE_BF;
    p.max_r_nnz = max_r;
    p.rden_dim = rden_dim;
    p.init_thr = o.init_threshold;
    p.out_ids = out_ids;
    p.out_scores = out_scores;
    p.n_found = o.n_found;
    p.touched = (unsigned long long*)o.postings_scanned;
    p.stats = (unsigned long long*)o.stats;
    p.level_margin = o.level_margin > 0.0f ? o.level_margin : default_margin(ix->dtype);
    if (!(p.level_margin <= 1.0f)) return fail(KNN_EINVAL, "level_margin must be in (0, 1]");
    p.carry = (u64*)((unsigned char*)scratch + NOALLOC_HEADER);

    const JoinKernel kern = join_kernel(ix->dtype, p.touched || p.stats, p.bf != 0);
    KNN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    const int per_launch =
        std::min(ix->n_blocks, o.blocks_per_launch > 0 ? o.blocks_per_launch : default_blocks_per_launch(ix));
    const int n_launch = (int)ceil_div(ix->n_blocks, per_launch);
    for (int li = 0; li < n_launch; li++) {
        p.block_begin = li * per_launch;
        p.block_end = std::min(ix->n_blocks, (li + 1) * per_launch);
        p.carry_in = li > 0;
        p.carry_out = li + 1 < n_launch;
        kern<<<(unsigned)r.n_rows, T, L.total, stream>>>(p);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    return KNN_OK;
}

// ---------------------------------------------------------------------------------
// batched joins: a prepared plan (validated jobs, work items, scratch) whose launch
// sequence -- reset the item counter, one persistent k_join_batched, one group merge
// per job with several groups -- is captured once into a CUDA graph and replayed.
// ---------------------------------------------------------------------------------
struct knn_batch {
    cudaStream_t cap_stream = nullptr;
    knn::Buffers* bufs = nullptr;
    knn_dtype dtype = KNN_U8;
    int n_jobs = 0, T = 512, grid = 0;
    size_t smem = 0;
    int64_t total = 0;
    std::vector<knn::BatchParams> chunks;   // up to BATCH_MAX_JOBS (sub-)jobs per launch
    std::vector<size_t> chunk_smem;         // each chunk's layout (its largest)
    std::vector<int> chunk_grid;            // each chunk's persistent grid
    unsigned long long* d_head = nullptr;   // one work counter per chunk
    unsigned* d_err = nullptr;     // set when a bounded wait gave up
    int32_t* done = nullptr;       // per row of every multi-group job: groups finished
    size_t done_n = 0;
    long long wait_spins = 0;
    int no_publish = 0;
    bool count = false;            // stats requested: the posting-counting kernel instance
    bool fx = false;               // float: a fixed-point pass, then an fp32 pass of the flagged rows
    uint8_t* fx_flag = nullptr;    // per row of every job: flagged by the fixed-point pass
    size_t fx_n = 0;
    int64_t n_items_all = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches_per_run = 0;
};

namespace knn {

static knn_status batch_enqueue(const knn_batch* b, cudaStream_t s) {
    KNN_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), s));
    if (b->fx) KNN_CUDA_TRY(cudaMemsetAsync(b->fx_flag, 0, b->fx_n, s));
    // float batches: the fixed-point pass over every item, then the fp32 pass that joins
    // the rows it flagged; otherwise the one pass
    for (int pass = b->fx ? 0 : 1; pass < 2; pass++) {
        KNN_CUDA_TRY(cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long) * b->chunks.size(), s));
        if (b->done_n) KNN_CUDA_TRY(cudaMemsetAsync(b->done, 0, sizeof(int32_t) * b->done_n, s));
        const BatchKernel kern = batch_kernel(b->dtype, b->count, pass == 0);
        for (size_t c = 0; c < b->chunks.size(); c++) {
            const BatchParams& bp = b->chunks[c];
            if (bp.phase_item[bp.n_phases] == 0) continue;
            kern<<<b->chunk_grid[c], b->T, b->chunk_smem[c], s>>>(bp, b->d_head + c, b->d_err, b->wait_spins,
                                                                 b->no_publish, b->fx && pass == 1);
            KNN_CUDA_TRY(cudaGetLastError());
        }
    }
    return KNN_OK;
}

}  // namespace knn

extern "C" void knn_batch_destroy(knn_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->bufs) {
        b->bufs->release();
        delete b->bufs;
    }
    delete b;
}

extern "C" knn_status knn_batch_create(int32_t n_jobs, const knn_job* jobs, const knn_batch_opts* opts, void* stream_,
                                       knn_batch** out) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!out) return fail(KNN_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_jobs < 1 || !jobs) return fail(KNN_EINVAL, "no jobs");
    knn_batch_opts o = {};
    if (opts) o = *opts;
    if (o.mode != KNN_MODE_IIIB && o.mode != KNN_MODE_IIB) return fail(KNN_EINVAL, "unknown mode");
    const float margin = o.level_margin > 0.0f
                             ? o.level_margin
                             : default_margin(jobs[0].index ? jobs[0].index->dtype : KNN_U8);
    if (!(margin <= 1.0f)) return fail(KNN_EINVAL, "level_margin must be in (0, 1]");
    int dev = 0, smem_optin = 0, n_sm = 0;
    KNN_CUDA_TRY(cudaGetDevice(&dev));
    KNN_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    KNN_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));

    knn_batch* b = new knn_batch();
    b->bufs = new Buffers(stream);
    auto bail = [&](knn_status st) {
        knn_batch_destroy(b);
        return st;
    };
    b->n_jobs = n_jobs;
    b->dtype = jobs[0].index ? jobs[0].index->dtype : KNN_U8;
    b->wait_spins = o.wait_spins > 0 ? o.wait_spins : BATCH_WAIT_SPINS;
    b->no_publish = o.test_never_publish ? 1 : 0;
    int T = o.threads ? o.threads : 512;
    if (T < 64 || T > 1024 || (T & 31) || (T & (T - 1)))
        return bail(fail(KNN_EINVAL, "threads must be a power of two in [64, 1024]"));
    b->T = T;

    Buffers tmp(stream);
    struct JobPlan {
        JoinParams p;
        size_t smem;         // shared-memory layout for its longest row
        int r_short = 0;     // > 0: rows up to this length run as a sub-job with a layout within 110 KB
        int rden_short = 0;
        int32_t* lists = nullptr;   // its rows, short ones first
    };
    std::vector<JobPlan> hj(n_jobs);
    std::vector<double> cost(n_jobs);
    for (int j = 0; j < n_jobs; j++) {
        const knn_job& jb = jobs[j];
        const knn_index* ix = jb.index;
        if (!ix) return bail(fail(KNN_EINVAL, "job %d: index is NULL", j));
        if (ix->dtype != b->dtype) return bail(fail(KNN_EINVAL, "job %d: all jobs must have the same dtype", j));
        if (jb.k < 1) return bail(fail(KNN_EINVAL, "job %d: k must be >= 1", j));
        if (jb.k > KNN_MAX_K) return bail(fail(KNN_EUNSUPPORTED, "job %d: k > %d", j, KNN_MAX_K));
        if (jb.R.dim != ix->dim || jb.R.dtype != ix->dtype)
            return bail(fail(KNN_EINVAL, "job %d: R does not match its index", j));
        if (!jb.R.on_device) return bail(fail(KNN_EINVAL, "job %d: R must be in device memory", j));
        DevCSR r;
        knn_status st = prepare_csr(&jb.R, stream, tmp, !o.skip_validation, true, &r);
        if (st != KNN_OK) return bail(fail(st, "job %d: %s", j, knn_last_error()));
        if (r.n_rows > 0 && (!jb.out_ids || !jb.out_scores)) return bail(fail(KNN_EINVAL, "job %d: outputs are NULL", j));
        if (ix->dtype == KNN_U8 && std::min(r.max_row_sum * ix->max_w, ix->max_row_sum * r.max_w) >= 2147483647.0)
            return bail(fail(KNN_EUNSUPPORTED, "job %d: uint8 scores could overflow int32", j));
        const int nb = ix->block_size;
        if (T * 4 > nb || nb / (T * 4) > 16)
            return bail(fail(KNN_EUNSUPPORTED, "job %d: S blocks of %d do not fit %d threads (need 4*T <= block <= 64*T)",
                             j, nb, T));
        const int max_r = std::max(1, r.max_row_nnz);
        const int rden_dim = rden_fitting(ix, nb, max_r);
        const size_t sm = smem_layout(nb, max_r, rden_dim).total;
        if (sm + sizeof(CtaState) + 32 * 8 * 2 + 128 > (size_t)smem_optin)
            return bail(fail(KNN_EUNSUPPORTED, "job %d: needs %zu bytes of shared memory", j, sm));
        hj[j].smem = sm;
        if (sm > TWO_CTA_SMEM && r.n_rows > 1) hj[j].r_short = short_row_limit(ix, nb, max_r, &hj[j].rden_short);
        int bpg = std::min(o.blocks_per_group > 0 ? o.blocks_per_group : default_blocks_per_launch(ix), ix->n_blocks);
        int groups = (int)ceil_div(ix->n_blocks, bpg);

        JoinParams& p = hj[j].p;
        memset(&p, 0, sizeof(p));
        p.n_rows = r.n_rows;
        p.r_indptr = r.indptr;
        p.r_idx = r.indices;
        p.r_val = r.values;
        p.n_s = ix->n_rows;
        p.dim = ix->dim;
        p.n_blocks = ix->n_blocks;
        p.n_levels = ix->n_levels;
        p.block_shift = ix->block_shift;
        p.binoff = ix->binoff;
        p.postings = ix->postings;
        p.s_indptr = ix->s_indptr;
        p.sp_d = ix->sp_d;
        p.sp_w = ix->sp_w;
        p.n_unidx = ix->n_unidx;
        p.ubound = ix->ubound;
        p.u_stride = ix->n_rows;
        p.s_maxnorm = maxnorm_up(ix);
        memcpy(p.levels, ix->levels, sizeof(p.levels));
        p.k = jb.k;
        p.groups = groups;
        p.blocks_per_group = bpg;
        p.block_begin = 0;
        p.block_end = ix->n_blocks;
        p.iiib = o.mode == KNN_MODE_IIIB && ix->n_levels > 1;
        p.max_r_nnz = max_r;
        p.rden_dim = rden_dim;
        p.level_margin = margin;
        p.out_ids = jb.out_ids;
        p.out_scores = jb.out_scores;
        p.stats = (unsigned long long*)o.stats;
        // larger items first: a row's postings in one group grow with |S| / groups and nnz(r)
        cost[j] = (double)ix->nnz / std::max(1, groups) * (double)(r.nnz + 1) / (double)std::max<int64_t>(1, r.n_rows);
    }
    // scratch of jobs with several groups: each row's carried keys and finished groups
    for (int j = 0; j < n_jobs; j++) {
        JoinParams& p = hj[j].p;
        if (p.groups > 1 && p.n_rows > 0) {
            knn_status st = b->bufs->get(&p.carry, (size_t)p.n_rows * p.k);
            if (st != KNN_OK) return bail(st);
            b->done_n += (size_t)p.n_rows;
        }
    }
    // float batches: per row of every job, the fixed-point pass's flag (join again in fp32)
    b->fx = b->dtype == KNN_F32;
    if (b->fx) {
        for (int j = 0; j < n_jobs; j++) b->fx_n += (size_t)std::max<int64_t>(0, hj[j].p.n_rows);
        knn_status st = b->bufs->get(&b->fx_flag, std::max<size_t>(1, b->fx_n));
        if (st != KNN_OK) return bail(st);
        size_t off = 0;
        for (int j = 0; j < n_jobs; j++) {
            hj[j].p.fx_flag = b->fx_flag + off;
            off += (size_t)std::max<int64_t>(0, hj[j].p.n_rows);
        }
    }
    if (b->done_n) {
        knn_status st = b->bufs->get(&b->done, b->done_n);
        if (st != KNN_OK) return bail(st);
        size_t off = 0;
        for (int j = 0; j < n_jobs; j++)
            if (hj[j].p.groups > 1 && hj[j].p.n_rows > 0) {
                hj[j].p.done = b->done + off;
                off += (size_t)hj[j].p.n_rows;
            }
    }
    // A job whose longest rows need a layout above TWO_CTA_SMEM (one CTA per SM) is split
    // in two sub-jobs: its rows of at most r_short features, with the largest layout
    // within TWO_CTA_SMEM, and the rest with the full one.  Each sub-job lists its rows
    // (k_split_rows, once here); both share the job's outputs, carried keys, done counters
    // and flags, which are indexed by the row.
    int n_split = 0;
    for (int j = 0; j < n_jobs; j++) n_split += hj[j].r_short > 0;
    std::vector<int32_t> split_n(2 * (size_t)n_split, 0);
    if (n_split) {
        int32_t* counts = nullptr;
        knn_status st = tmp.get(&counts, 2 * (size_t)n_split);
        if (st != KNN_OK) return bail(st);
        if (cudaMemsetAsync(counts, 0, 2 * sizeof(int32_t) * n_split, stream) != cudaSuccess)
            return bail(fail(KNN_ECUDA, "memset of the row-split counts failed"));
        for (int j = 0, q = 0; j < n_jobs; j++) {
            if (!hj[j].r_short) continue;
            const JoinParams& p = hj[j].p;
            if ((st = b->bufs->get(&hj[j].lists, (size_t)p.n_rows)) != KNN_OK) return bail(st);
            k_split_rows<<<launch_blocks(p.n_rows, 256), 256, 0, stream>>>(p.r_indptr, p.n_rows, hj[j].r_short,
                                                                          hj[j].lists, counts + 2 * q++);
            if (cudaGetLastError() != cudaSuccess) return bail(fail(KNN_ECUDA, "k_split_rows launch failed"));
            count_launch();
        }
        if (cudaMemcpyAsync(split_n.data(), counts, 2 * sizeof(int32_t) * n_split, cudaMemcpyDeviceToHost, stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return bail(fail(KNN_ECUDA, "reading the row-split counts failed"));
    }
    struct SubJob {
        JoinParams p;
        int64_t rows;   // rows its items cover (each in all of its groups)
        size_t smem;
        double cost;
    };
    std::vector<SubJob> subs;   // jobs without rows have no items and are left out
    for (int j = 0, q = 0; j < n_jobs; j++) {
        const JobPlan& h = hj[j];
        if (!h.r_short) {
            if (h.p.n_rows > 0) subs.push_back({h.p, h.p.n_rows, h.smem, cost[j]});
            continue;
        }
        const int64_t n_short = split_n[2 * q++];
        if (n_short > 0) {
            SubJob sj{h.p, n_short, smem_layout(1 << h.p.block_shift, h.r_short, h.rden_short).total, cost[j]};
            sj.p.row_list = h.lists;
            sj.p.max_r_nnz = h.r_short;
            sj.p.rden_dim = h.rden_short;
            subs.push_back(sj);
        }
        if (n_short < h.p.n_rows) {
            SubJob sj{h.p, h.p.n_rows - n_short, h.smem, cost[j]};
            sj.p.row_list = h.lists + n_short;
            subs.push_back(sj);
        }
    }
    // Chunks: the sub-jobs within TWO_CTA_SMEM, then the others, each class in persistent
    // launches of up to BATCH_MAX_JOBS sub-jobs, sorted by group count (descending: the
    // round layout of BatchParams), larger items first among equal counts.
    for (int cls = 0; cls < 2; cls++) {
        std::vector<int> order;
        for (int i = 0; i < (int)subs.size(); i++)
            if ((subs[i].smem > TWO_CTA_SMEM) == (cls == 1)) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            if (subs[a].p.groups != subs[c].p.groups) return subs[a].p.groups > subs[c].p.groups;
            return subs[a].cost > subs[c].cost;
        });
        for (size_t i = 0; i < order.size(); i += BATCH_MAX_JOBS) {
            BatchParams bp;
            memset(&bp, 0, sizeof(bp));
            size_t sm = 0;
            for (size_t q = i; q < std::min(order.size(), i + BATCH_MAX_JOBS); q++) {
                const SubJob& sj = subs[order[q]];
                bp.p[bp.n_jobs] = sj.p;
                bp.rows_before[bp.n_jobs + 1] = bp.rows_before[bp.n_jobs] + sj.rows;
                sm = std::max(sm, sj.smem);
                bp.n_jobs++;
            }
            // phases: while every job has groups left, all of them; then, as the jobs with
            // the fewest groups run out, shorter prefixes
            long long item = 0;
            int round = 0;
            for (int a = bp.n_jobs; a >= 1; a--) {
                const int end_round = bp.p[a - 1].groups;
                if (end_round <= round) continue;
                bp.phase_item[bp.n_phases] = item;
                bp.phase_round[bp.n_phases] = round;
                bp.phase_jobs[bp.n_phases] = a;
                bp.n_phases++;
                item += (long long)(end_round - round) * bp.rows_before[a];
                round = end_round;
            }
            bp.phase_item[bp.n_phases] = item;
            bp.phase_round[bp.n_phases] = round;
            b->chunks.push_back(bp);
            b->chunk_smem.push_back(sm);
            b->n_items_all += item;
            b->smem = std::max(b->smem, sm);
        }
    }
    b->total = b->n_items_all;
    knn_status st;
    if ((st = b->bufs->get(&b->d_head, std::max<size_t>(1, b->chunks.size()))) != KNN_OK) return bail(st);
    if ((st = b->bufs->get(&b->d_err, 1)) != KNN_OK) return bail(st);
#define BATCH_CUDA(expr)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) return bail(fail(KNN_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_))); \
    } while (0)
    b->count = o.stats != nullptr;
    for (int pass = b->fx ? 0 : 1; pass < 2; pass++)
        BATCH_CUDA(cudaFuncSetAttribute(batch_kernel(b->dtype, b->count, pass == 0),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    int active = 0;
    for (size_t c = 0; c < b->chunks.size(); c++) {
        // CTAs per SM that both kernel instances reach with this chunk's layout
        int per_sm = 0;
        for (int pass = b->fx ? 0 : 1; pass < 2; pass++) {
            int ps = 0;
            BATCH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, batch_kernel(b->dtype, b->count, pass == 0), T,
                                                                     b->chunk_smem[c]));
            per_sm = per_sm ? std::min(per_sm, ps) : ps;
        }
        if (per_sm < 1) return bail(fail(KNN_EUNSUPPORTED, "the batched kernel does not fit an SM"));
        const long long items = b->chunks[c].phase_item[b->chunks[c].n_phases];
        b->chunk_grid.push_back((int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * n_sm, items)));
        b->grid = std::max(b->grid, b->chunk_grid.back());
        active += items > 0;
    }
    b->launches_per_run = active * (b->fx ? 2 : 1);
    BATCH_CUDA(cudaStreamSynchronize(stream));
    tmp.release();
    if (o.use_graph) {
        BATCH_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        BATCH_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        st = batch_enqueue(b, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != KNN_OK) {
            if (g) cudaGraphDestroy(g);
            return bail(st);
        }
        if (e != cudaSuccess) return bail(fail(KNN_ECUDA, "graph capture: %s", cudaGetErrorString(e)));
        b->graph = g;
        BATCH_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
#undef BATCH_CUDA
    *out = b;
    return KNN_OK;
}

extern "C" knn_status knn_batch_launch(knn_batch* b, void* stream_) {
    if (!b) return fail(KNN_EINVAL, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream_;
    if (b->total == 0) return KNN_OK;
    if (b->exec) {
        KNN_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    } else {
        KNN_TRY(batch_enqueue(b, s));
    }
    count_launch(b->launches_per_run);
    return KNN_OK;
}

extern "C" knn_status knn_batch_check(const knn_batch* b, void* stream_) {
    if (!b) return fail(KNN_EINVAL, "batch is NULL");
    unsigned e = 0;
    KNN_CUDA_TRY(cudaMemcpyAsync(&e, b->d_err, sizeof(e), cudaMemcpyDeviceToHost, (cudaStream_t)stream_));
    KNN_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream_));
    if (e & 2u) return fail(KNN_EINVAL, "a row of a batched job has more features than when the batch was made");
    if (e) return fail(KNN_ETIMEOUT, "a batched work item waited too long for its row's previous group");
    return KNN_OK;
}

extern "C" knn_status knn_batch_get_info(const knn_batch* b, knn_batch_info* info) {
    if (!b || !info) return fail(KNN_EINVAL, "NULL argument");
    info->work_items = b->total;
    info->ctas = b->grid;
    info->threads = b->T;
    info->shared_bytes = (int64_t)b->smem;
    info->graph = b->exec != nullptr;
    info->kernels_per_launch = b->launches_per_run;
    return KNN_OK;
}

extern "C" knn_status knn_join_batched(int32_t n_jobs, const knn_job* jobs, const knn_batch_opts* opts, void* stream) {
    knn_batch_opts o = {};
    if (opts) o = *opts;
    o.use_graph = 0;
    knn_batch* b = nullptr;
    KNN_TRY(knn_batch_create(n_jobs, jobs, &o, stream, &b));
    knn_status st = knn_batch_launch(b, stream);
    if (st == KNN_OK) st = knn_batch_check(b, stream);
    knn_batch_destroy(b);
    return st;
}

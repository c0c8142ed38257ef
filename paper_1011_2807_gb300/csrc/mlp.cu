// Learned start threshold for the join (not in the paper; it generalises Section 4.4's
// MinPruneScore, "a threshold derived from previous computation", to a threshold
// predicted for each query before any S block is scanned).
//
// A query r is summarised by a sketch x(r) of SKETCH_IN = 516 values:
//   x[0..511]  signed feature hashing: each feature (d, w) adds sign(d) * w / ||r||_2 to
//              bucket(d), both drawn from one 32-bit integer hash of d;
//   x[512..515] log1p of (nnz, sum of weights, ||r||_2, largest weight).
// An MLP 516 -> 256 -> 256 -> 1 (ReLU) with BF16 weights and FP32 accumulation predicts
// y = log(k-th best score of r).  It is trained with the pinball (quantile) loss at a
// low quantile q, so that exp(y) tends to sit below the true k-th score; the join then
// keeps every s with score >= exp(y) and verifies that k were found (knn_join_learned).
//
// Kernels: k_sketch, k_gemm_bf16 (tcgen05 tensor cores, TMEM accumulator), bias/ReLU,
// the output layer, the loss gradient, the backward reductions and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "common.cuh"

namespace knn {

constexpr int SKETCH_BUCKETS = 512;
constexpr int SKETCH_IN = SKETCH_BUCKETS + 4;   // 516
constexpr int IN_PAD = 528;                     // input width padded to a multiple of 16
constexpr int HID = 256;

// ---------------------------------------------------------------------------------
// sketch
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // integer finaliser (xor-shift / multiply rounds of the MurmurHash3 family)
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// one warp per row; writes bf16 x[row][0..IN_PAD) (zeros past SKETCH_IN)
template <class W>
__global__ void k_sketch(const int64_t* __restrict__ indptr, const int32_t* __restrict__ idx,
                         const W* __restrict__ val, int64_t n, uint32_t seed, __nv_bfloat16* __restrict__ X) {
    __shared__ float buf[8][SKETCH_BUCKETS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    float* b = buf[wib];
    for (int i = lane; i < SKETCH_BUCKETS; i += 32) b[i] = 0.0f;
    __syncwarp();
    if (row < n) {
        const int64_t a = indptr[row], e = indptr[row + 1];
        float sum = 0.0f, sq = 0.0f, mx = 0.0f;
        for (int64_t j = a + lane; j < e; j += 32) {
            float w = (float)val[j];
            sum += w;
            sq += w * w;
            mx = fmaxf(mx, w);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        const float norm = sqrtf(sq);
        const float inv = norm > 0.0f ? 1.0f / norm : 0.0f;
        for (int64_t j = a + lane; j < e; j += 32) {
            uint32_t h = mix32((uint32_t)idx[j] * 0x9E3779B1u + seed);
            float w = (float)val[j] * inv;
            atomicAdd(&b[h & (SKETCH_BUCKETS - 1)], (h >> 31) ? -w : w);
        }
        __syncwarp();
        __nv_bfloat16* xr = X + row * IN_PAD;
        for (int i = lane; i < IN_PAD; i += 32) {
            float v = 0.0f;
            if (i < SKETCH_BUCKETS) v = b[i];
            else if (i == SKETCH_BUCKETS) v = log1pf((float)(e - a));
            else if (i == SKETCH_BUCKETS + 1) v = log1pf(sum);
            else if (i == SKETCH_BUCKETS + 2) v = log1pf(norm);
            else if (i == SKETCH_BUCKETS + 3) v = log1pf(mx);
            xr[i] = __float2bfloat16(v);
        }
    }
}

// ---------------------------------------------------------------------------------
// BF16 GEMM on the 5th-generation tensor cores: C[m][n] (+)= sum_k A(m,k) * B(k,n) with
// FP32 accumulation in tensor memory.  A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk +
// n*sbn] (bf16, any strides), so one kernel serves X W^T, dH W and dH^T X.
// CTA tile 128 x 64, K step 32.  The operands are staged in shared memory in the
// canonical K-major layout without swizzle (8 x 8 core matrices of 16-byte rows, the
// next core matrix along K 128 bytes on, the next 8-row group 512 bytes on); one thread
// issues tcgen05.mma (kind::f16, M = 128, N = 64, K = 16 each) and commits to an
// mbarrier, which every thread waits on (bounded) before the tiles are overwritten; at
// the end each warp reads its 32 accumulator rows (TMEM lanes) with tcgen05.ld.
// ---------------------------------------------------------------------------------
constexpr int TM = 128, TN = 64, TK = 32;
constexpr long long GEMM_WAIT_SPINS = 1LL << 22;   // try_wait polls before giving up
__device__ unsigned g_gemm_err;                     // set when a bounded wait gave up

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// element (r, k) of a [rows][TK] tile in the canonical K-major layout without swizzle
__device__ __forceinline__ int canon(int r, int k) {
    return ((r >> 3) * (TK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: start address, leading byte offset (next core matrix
// along K), stride byte offset (next 8-row group), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t GEMM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                   int64_t sam, int64_t sak, const __nv_bfloat16* __restrict__ B,
                                                   int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t scm,
                                                   int64_t scn, int accumulate) {
    __shared__ __align__(128) __nv_bfloat16 As[TM * TK];
    __shared__ __align__(128) __nv_bfloat16 Bs[TN * TK];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const uint32_t mbar_a = smem_u32(&mbar);
    if (warp == 0) {   // TN fp32 columns of tensor memory for the 128 x TN accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "n"(TN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    uint32_t phase = 0;
    bool issued = false;
    // With K contiguous (stride 1) and 16-byte aligned rows, 8 consecutive k of a row are
    // one 16-byte row of a core matrix: staged with one 128-bit load and store.
    const bool a_vec = sak == 1 && (sam & 7) == 0 && (((uintptr_t)A) & 15) == 0;
    const bool b_vec = sbk == 1 && (sbn & 7) == 0 && (((uintptr_t)B) & 15) == 0;
    for (int k0 = 0; k0 < K; k0 += TK) {
        if (a_vec) {
            for (int i = tid; i < TM * (TK / 8); i += 128) {
                const int r = i / (TK / 8), c = (i % (TK / 8)) * 8;
                const int m = m0 + r, k = k0 + c;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (m < M && k + 8 <= K) {
                    v = *(const uint4*)(A + (int64_t)m * sam + k);
                } else if (m < M) {
                    __nv_bfloat16* e = (__nv_bfloat16*)&v;
                    for (int q = 0; q < 8 && k + q < K; q++) e[q] = A[(int64_t)m * sam + k + q];
                }
                *(uint4*)(As + canon(r, c)) = v;
            }
        } else {
            for (int i = tid; i < TM * TK; i += 128) {
                const int r = i / TK, c = i % TK;
                const int m = m0 + r, k = k0 + c;
                As[canon(r, c)] = (m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : zero;
            }
        }
        if (b_vec) {
            for (int i = tid; i < TN * (TK / 8); i += 128) {
                const int r = i / (TK / 8), c = (i % (TK / 8)) * 8;   // r: n, c: k
                const int n = n0 + r, k = k0 + c;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (n < N && k + 8 <= K) {
                    v = *(const uint4*)(B + k + (int64_t)n * sbn);
                } else if (n < N) {
                    __nv_bfloat16* e = (__nv_bfloat16*)&v;
                    for (int q = 0; q < 8 && k + q < K; q++) e[q] = B[k + q + (int64_t)n * sbn];
                }
                *(uint4*)(Bs + canon(r, c)) = v;
            }
        } else {
            for (int i = tid; i < TN * TK; i += 128) {
                const int r = i / TK, c = i % TK;   // r: n, c: k
                const int n = n0 + r, k = k0 + c;
                Bs[canon(r, c)] = (n < N && k < K) ? B[(int64_t)k * sbk + (int64_t)n * sbn] : zero;
            }
        }
        // the tiles were written through the generic proxy; the tensor core reads them
        // through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TK; kk += 16) {
                const uint64_t ad = smem_desc(smem_u32(As) + (kk / 8) * 128, 128, (TK / 8) * 128);
                const uint64_t bd = smem_desc(smem_u32(Bs) + (kk / 8) * 128, 128, (TK / 8) * 128);
                const uint32_t acc_in = (k0 > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(GEMM_IDESC), "r"(acc_in) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(mbar_a) : "memory");
        }
        issued = true;
        // every thread waits until the MMAs have consumed the tiles (bounded)
        uint32_t done = 0;
        for (long long spins = 0; spins < GEMM_WAIT_SPINS; spins++) {
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done) : "r"(mbar_a), "r"(phase) : "memory");
            if (done) break;
        }
        if (!done) s_fail = 1;
        __syncthreads();
        if (s_fail) break;   // `phase` still names the step whose MMAs may be in flight
        phase ^= 1u;
    }
    if (s_fail) {
        // The MMAs of the step whose wait gave up may still be running, and the
        // accumulator's tensor memory must not be released under them: wait for their
        // commit once more, with the same bound.  If that wait gives up too, the
        // columns stay allocated (the kernel returns without tcgen05.dealloc) and the
        // error flag says so.
        if (tid == 0) {
            uint32_t done = 0;
            for (long long spins = 0; spins < GEMM_WAIT_SPINS && !done; spins++)
                asm volatile(
                    "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                    "selp.u32 %0, 1, 0, p;\n\t}"
                    : "=r"(done) : "r"(mbar_a), "r"(phase) : "memory");
            s_fail = done ? 1 : 2;
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            if (issued) {
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int q = 0; q < 16; q++) r[q] = 0u;
            }
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int n = n0 + c0 + q;
                    if (n < N) {
                        float* c = C + (int64_t)row * scm + (int64_t)n * scn;
                        *c = accumulate ? *c + __uint_as_float(r[q]) : __uint_as_float(r[q]);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicMax(&g_gemm_err, (unsigned)s_fail);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && s_fail != 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TN) : "memory");
}

static knn_status gemm(int M, int N, int K, const __nv_bfloat16* A, int64_t sam, int64_t sak, const __nv_bfloat16* B,
                       int64_t sbk, int64_t sbn, float* C, int64_t scm, int64_t scn, bool accumulate,
                       cudaStream_t stream) {
    if (M <= 0 || N <= 0) return KNN_OK;
    dim3 grid((unsigned)ceil_div(N, TN), (unsigned)ceil_div(M, TM));
    k_gemm_bf16<<<grid, 128, 0, stream>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, scm, scn, accumulate ? 1 : 0);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    return KNN_OK;
}

// Reports (and clears) a GEMM that gave up its bounded wait since the last check; the
// caller has synchronised the stream.
static knn_status gemm_check() {
    unsigned e = 0;
    KNN_CUDA_TRY(cudaMemcpyFromSymbol(&e, g_gemm_err, sizeof(e)));
    if (e) {
        const unsigned z = 0;
        KNN_CUDA_TRY(cudaMemcpyToSymbol(g_gemm_err, &z, sizeof(z)));
        if (e >= 2)
            return fail(KNN_ETIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs twice and left its "
                                      "tensor memory allocated; treat this GPU context as unusable");
        return fail(KNN_ETIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs");
    }
    return KNN_OK;
}

// ---------------------------------------------------------------------------------
// elementwise pieces
// ---------------------------------------------------------------------------------
// H[b][j] = relu(P[b][j] + bias[j]) as bf16 (P is the fp32 pre-activation)
__global__ void k_bias_relu(const float* __restrict__ P, const float* __restrict__ bias, int64_t B, int H,
                            __nv_bfloat16* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * H) return;
    float v = P[i] + bias[i % H];
    out[i] = __float2bfloat16(v > 0.0f ? v : 0.0f);
}

// y[b] = h2[b] . w3 + b3 (one warp per row)
__global__ void k_out_layer(const __nv_bfloat16* __restrict__ H2, const __nv_bfloat16* __restrict__ w3, const float* b3,
                            int64_t B, float* __restrict__ y) {
    int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= B) return;
    float s = 0.0f;
    for (int j = lane; j < HID; j += 32) s += __bfloat162float(H2[row * HID + j]) * __bfloat162float(w3[j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + b3[0];
}

// pinball loss at quantile q on (pred, target); g = dL/dpred / B; loss summed into *loss
__global__ void k_pinball(const float* __restrict__ pred, const float* __restrict__ target, int64_t B, float q,
                          float* __restrict__ g, float* __restrict__ loss) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < B) {
        float e = target[i] - pred[i];
        l = e > 0.0f ? q * e : (q - 1.0f) * e;
        g[i] = (e > 0.0f ? -q : (1.0f - q)) / (float)B;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// output layer backward: dH2[b][j] = g[b] * w3[j] * (h2 > 0) (bf16), dw3[j] = sum_b g[b] h2[b][j], db3 = sum g
__global__ void k_back_out(const float* __restrict__ g, const __nv_bfloat16* __restrict__ H2,
                           const __nv_bfloat16* __restrict__ w3, int64_t B, __nv_bfloat16* __restrict__ dH2,
                           float* __restrict__ dw3, float* __restrict__ db3) {
    // one thread per hidden unit j, looping over the batch (B is a mini-batch)
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < HID) {
        float s = 0.0f;
        const float wj = __bfloat162float(w3[j]);
        for (int64_t b = 0; b < B; b++) {
            float h = __bfloat162float(H2[b * HID + j]);
            s += g[b] * h;
            dH2[b * HID + j] = __float2bfloat16(h > 0.0f ? g[b] * wj : 0.0f);
        }
        dw3[j] = s;
    }
    if (j == 0) {
        float s = 0.0f;
        for (int64_t b = 0; b < B; b++) s += g[b];
        db3[0] = s;
    }
}

// D[b][j] *= (H[b][j] > 0) and store as bf16; column sums into dbias
__global__ void k_relu_back(const float* __restrict__ D, const __nv_bfloat16* __restrict__ H, int64_t B, int Hn,
                            __nv_bfloat16* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * Hn) return;
    out[i] = __float2bfloat16(__bfloat162float(H[i]) > 0.0f ? D[i] : 0.0f);
}

__global__ void k_colsum(const __nv_bfloat16* __restrict__ D, int64_t B, int Hn, float* __restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Hn) return;
    float s = 0.0f;
    for (int64_t b = 0; b < B; b++) s += __bfloat162float(D[b * Hn + j]);
    out[j] = s;
}

// Adam on fp32 master weights; refreshes the bf16 copy
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, int64_t n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = grad[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(in[i]);
}

// gather rows of X (bf16, IN_PAD wide) and targets for a mini-batch
__global__ void k_gather_batch(const __nv_bfloat16* __restrict__ X, const float* __restrict__ y,
                               const int32_t* __restrict__ idx, int64_t B, __nv_bfloat16* __restrict__ Xb,
                               float* __restrict__ yb) {
    int64_t b = blockIdx.x;
    if (b >= B) return;
    int64_t r = idx[b];
    for (int i = threadIdx.x; i < IN_PAD; i += blockDim.x) Xb[b * IN_PAD + i] = X[r * IN_PAD + i];
    if (threadIdx.x == 0) yb[b] = y[r];
}

// log of the k-th scores (float or int32 bits), rows with no k-th score marked invalid (NaN)
__global__ void k_log_labels(const float* __restrict__ kth, int64_t n, float* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = kth[i];
    y[i] = v > 0.0f ? logf(v) : __int_as_float(0x7fc00000);
}

// tau = exp(y) (the predicted k-th score), optional scale
// kth / tau per row (+inf where the row has no k-th score: it falls back whatever tau is)
__global__ void k_kth_ratio(const float* __restrict__ kth, const float* __restrict__ tau, int64_t n,
                            float* __restrict__ ratio) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) ratio[i] = kth[i] > 0.0f && tau[i] > 0.0f ? kth[i] / tau[i] : __int_as_float(0x7f800000);
}

__global__ void k_exp_tau(const float* __restrict__ y, int64_t n, float scale, float* __restrict__ tau) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) tau[i] = expf(y[i]) * scale;
}

}  // namespace knn

// =================================================================================
// the model object
// =================================================================================
struct knn_model {
    uint32_t hash_seed = 0;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    knn::Buffers* bufs = nullptr;
    // fp32 master parameters, bf16 copies, Adam moments; one flat array each:
    //   W1 [HID][IN_PAD] | b1 [HID] | W2 [HID][HID] | b2 [HID] | w3 [HID] | b3 [1]
    float* w = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    __nv_bfloat16* wb = nullptr;
    int64_t n_params = 0;
    float tau_scale = 1.0f;   // calibrated multiplier of the predictions (1 until calibrated)
};

namespace knn {

constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + (int64_t)HID * IN_PAD;
constexpr int64_t OFF_W2 = OFF_B1 + HID;
constexpr int64_t OFF_B2 = OFF_W2 + (int64_t)HID * HID;
constexpr int64_t OFF_W3 = OFF_B2 + HID;
constexpr int64_t OFF_B3 = OFF_W3 + HID;
constexpr int64_t N_PARAMS = OFF_B3 + 1;

// activations and gradients for a batch of up to `cap` rows
struct MlpWork {
    int64_t cap = 0;
    __nv_bfloat16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *D1 = nullptr, *D2 = nullptr;
    float *P = nullptr, *y = nullptr, *g = nullptr, *t = nullptr, *loss = nullptr;
    knn_status alloc(Buffers& b, int64_t n) {
        cap = n;
        KNN_TRY(b.get(&X, (size_t)n * IN_PAD));
        KNN_TRY(b.get(&H1, (size_t)n * HID));
        KNN_TRY(b.get(&H2, (size_t)n * HID));
        KNN_TRY(b.get(&D1, (size_t)n * HID));
        KNN_TRY(b.get(&D2, (size_t)n * HID));
        KNN_TRY(b.get(&P, (size_t)n * HID));
        KNN_TRY(b.get(&y, (size_t)n));
        KNN_TRY(b.get(&g, (size_t)n));
        KNN_TRY(b.get(&t, (size_t)n));
        KNN_TRY(b.get(&loss, 1));
        return KNN_OK;
    }
};

static knn_status mlp_forward(const knn_model* md, MlpWork& w, int64_t B, const __nv_bfloat16* X,
                              cudaStream_t s) {
    const __nv_bfloat16* W1 = md->wb + OFF_W1;
    const __nv_bfloat16* W2 = md->wb + OFF_W2;
    // H1 = relu(X W1^T + b1)
    KNN_TRY(gemm((int)B, HID, IN_PAD, X, IN_PAD, 1, W1, 1, IN_PAD, w.P, HID, 1, false, s));
    k_bias_relu<<<launch_blocks(B * HID, 256), 256, 0, s>>>(w.P, md->w + OFF_B1, B, HID, w.H1);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    // H2 = relu(H1 W2^T + b2)
    KNN_TRY(gemm((int)B, HID, HID, w.H1, HID, 1, W2, 1, HID, w.P, HID, 1, false, s));
    k_bias_relu<<<launch_blocks(B * HID, 256), 256, 0, s>>>(w.P, md->w + OFF_B2, B, HID, w.H2);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    k_out_layer<<<launch_blocks(B * 32, 256), 256, 0, s>>>(w.H2, md->wb + OFF_W3, md->w + OFF_B3, B, w.y);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    return KNN_OK;
}

// gradients of the mean pinball loss into md->grad (overwritten)
static knn_status mlp_backward(knn_model* md, MlpWork& w, int64_t B, const __nv_bfloat16* X, cudaStream_t s) {
    float* G = md->grad;
    k_back_out<<<1, HID, 0, s>>>(w.g, w.H2, md->wb + OFF_W3, B, w.D2, G + OFF_W3, G + OFF_B3);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    k_colsum<<<1, HID, 0, s>>>(w.D2, B, HID, G + OFF_B2);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    // dW2 = dH2^T H1  [HID x HID]
    KNN_TRY(gemm(HID, HID, (int)B, w.D2, 1, HID, w.H1, HID, 1, G + OFF_W2, HID, 1, false, s));
    // dH1 = (dH2 W2) * relu'(H1)
    KNN_TRY(gemm((int)B, HID, HID, w.D2, HID, 1, md->wb + OFF_W2, HID, 1, w.P, HID, 1, false, s));
    k_relu_back<<<launch_blocks(B * HID, 256), 256, 0, s>>>(w.P, w.H1, B, HID, w.D1);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    k_colsum<<<1, HID, 0, s>>>(w.D1, B, HID, G + OFF_B1);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    // dW1 = dH1^T X  [HID x IN_PAD]
    KNN_TRY(gemm(HID, IN_PAD, (int)B, w.D1, 1, HID, X, IN_PAD, 1, G + OFF_W1, IN_PAD, 1, false, s));
    return KNN_OK;
}

static knn_status sketch(const DevCSR& r, uint32_t seed, __nv_bfloat16* X, cudaStream_t s) {
    if (r.n_rows == 0) return KNN_OK;
    unsigned grid = (unsigned)ceil_div(r.n_rows, 8);
    if (r.dtype == KNN_U8)
        k_sketch<uint8_t><<<grid, 256, 0, s>>>(r.indptr, r.indices, (const uint8_t*)r.values, r.n_rows, seed, X);
    else
        k_sketch<float><<<grid, 256, 0, s>>>(r.indptr, r.indices, (const float*)r.values, r.n_rows, seed, X);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    return KNN_OK;
}

float model_tau_scale(const knn_model* md) { return md->tau_scale; }

knn_status model_check() { return gemm_check(); }

// predicted k-th scores for every row of r (device float[n_rows]) in chunks
knn_status model_predict_tau(const knn_model* md, const DevCSR& r, float tau_scale, float* tau, cudaStream_t s,
                             Buffers& tmp) {
    const int64_t CH = 65536;
    MlpWork w;
    KNN_TRY(w.alloc(tmp, std::min<int64_t>(CH, std::max<int64_t>(1, r.n_rows))));
    __nv_bfloat16* X = nullptr;
    KNN_TRY(tmp.get(&X, (size_t)std::max<int64_t>(1, r.n_rows) * IN_PAD));
    KNN_TRY(sketch(r, md->hash_seed, X, s));
    for (int64_t a = 0; a < r.n_rows; a += CH) {
        int64_t B = std::min(CH, r.n_rows - a);
        KNN_TRY(mlp_forward(md, w, B, X + a * IN_PAD, s));
        k_exp_tau<<<launch_blocks(B, 256), 256, 0, s>>>(w.y, B, tau_scale, tau + a);
        KNN_CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    return KNN_OK;
}

}  // namespace knn

using namespace knn;

extern "C" knn_status knn_threshold_model_create(const knn_model_opts* opts, void* stream_, knn_model** out) {
    if (!out) return fail(KNN_EINVAL, "out is NULL");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream_;
    knn_model_opts o = {};
    if (opts) o = *opts;
    knn_model* md = new knn_model();
    md->bufs = new Buffers(s);
    md->stream = s;
    md->hash_seed = (uint32_t)(o.seed ^ 0x5bd1e995u);
    md->n_params = N_PARAMS;
    auto bail = [&](knn_status st) {
        md->bufs->release();
        delete md->bufs;
        delete md;
        return st;
    };
    knn_status st;
    if ((st = md->bufs->get(&md->w, N_PARAMS)) != KNN_OK) return bail(st);
    if ((st = md->bufs->get(&md->m, N_PARAMS)) != KNN_OK) return bail(st);
    if ((st = md->bufs->get(&md->v, N_PARAMS)) != KNN_OK) return bail(st);
    if ((st = md->bufs->get(&md->grad, N_PARAMS)) != KNN_OK) return bail(st);
    if ((st = md->bufs->get(&md->wb, N_PARAMS)) != KNN_OK) return bail(st);
    // He-uniform initial weights from a seeded generator; zero biases
    std::vector<float> h(N_PARAMS, 0.0f);
    std::mt19937_64 rng(o.seed);
    auto fill = [&](int64_t off, int64_t n, int fan_in, int valid_cols, int row_len) {
        float lim = std::sqrt(6.0f / (float)fan_in);
        std::uniform_real_distribution<float> U(-lim, lim);
        for (int64_t i = 0; i < n; i++) {
            int col = row_len ? (int)(i % row_len) : 0;
            h[off + i] = (row_len && col >= valid_cols) ? 0.0f : U(rng);
        }
    };
    fill(OFF_W1, (int64_t)HID * IN_PAD, SKETCH_IN, SKETCH_IN, IN_PAD);
    fill(OFF_W2, (int64_t)HID * HID, HID, 0, 0);
    fill(OFF_W3, HID, HID, 0, 0);
    cudaError_t e = cudaMemcpyAsync(md->w, h.data(), sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(md->m, 0, sizeof(float) * N_PARAMS, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(md->v, 0, sizeof(float) * N_PARAMS, s);
    if (e != cudaSuccess) return bail(fail(KNN_ECUDA, "model init: %s", cudaGetErrorString(e)));
    k_to_bf16<<<launch_blocks(N_PARAMS, 256), 256, 0, s>>>(md->w, md->wb, N_PARAMS);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(fail(KNN_ECUDA, "model init: %s", cudaGetErrorString(e)));
    count_launch();
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(fail(KNN_ECUDA, "model init: %s", cudaGetErrorString(e)));
    *out = md;
    return KNN_OK;
}

extern "C" void knn_threshold_model_destroy(knn_model* md) {
    if (!md) return;
    if (md->bufs) {
        md->bufs->release();
        delete md->bufs;
    }
    delete md;
}

extern "C" knn_status knn_threshold_model_train(knn_model* md, const knn_csr* Q, const float* kth_scores,
                                               const knn_train_opts* topts, float* final_loss, void* stream_) {
    if (!md) return fail(KNN_EINVAL, "model is NULL");
    if (!kth_scores) return fail(KNN_EINVAL, "kth_scores is NULL");
    cudaStream_t s = (cudaStream_t)stream_;
    knn_train_opts o = {};
    if (topts) o = *topts;
    const int epochs = o.epochs > 0 ? o.epochs : 20;
    const int batch = o.batch > 0 ? o.batch : 512;
    const float lr = o.lr > 0.0f ? o.lr : 1e-3f;
    const float q = o.quantile > 0.0f ? o.quantile : 0.1f;
    if (!(q > 0.0f && q < 1.0f)) return fail(KNN_EINVAL, "quantile must be in (0, 1)");
    Buffers tmp(s);
    DevCSR r;
    KNN_TRY(prepare_csr(Q, s, tmp, true, false, &r));
    if (r.n_rows == 0) return fail(KNN_EINVAL, "no training queries");
    __nv_bfloat16* X = nullptr;
    float* y = nullptr;
    KNN_TRY(tmp.get(&X, (size_t)r.n_rows * IN_PAD));
    KNN_TRY(tmp.get(&y, (size_t)r.n_rows));
    KNN_TRY(sketch(r, md->hash_seed, X, s));
    k_log_labels<<<launch_blocks(r.n_rows, 256), 256, 0, s>>>(kth_scores, r.n_rows, y);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    // valid rows (a k-th score exists) and the mean target (initial output bias)
    std::vector<float> hy(r.n_rows);
    KNN_CUDA_TRY(cudaMemcpyAsync(hy.data(), y, sizeof(float) * r.n_rows, cudaMemcpyDeviceToHost, s));
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int32_t> valid;
    double mean = 0.0;
    for (int64_t i = 0; i < r.n_rows; i++)
        if (hy[i] == hy[i]) {
            valid.push_back((int32_t)i);
            mean += hy[i];
        }
    if (valid.empty()) return fail(KNN_EINVAL, "no training query has a k-th score");
    mean /= (double)valid.size();
    if (md->step == 0) {
        float b3 = (float)mean;
        KNN_CUDA_TRY(cudaMemcpyAsync(md->w + OFF_B3, &b3, sizeof(float), cudaMemcpyHostToDevice, s));
        KNN_CUDA_TRY(cudaStreamSynchronize(s));
    }
    MlpWork w;
    KNN_TRY(w.alloc(tmp, batch));
    int32_t* d_idx = nullptr;
    KNN_TRY(tmp.get(&d_idx, valid.size()));
    std::mt19937_64 rng(o.seed ^ 0x9e3779b97f4a7c15ull);
    const int64_t nb = (int64_t)valid.size() / batch;   // full batches only
    if (nb == 0) return fail(KNN_EINVAL, "fewer valid training queries (%zu) than one batch (%d)", valid.size(), batch);
    double last_loss = 0.0;
    for (int ep = 0; ep < epochs; ep++) {
        std::shuffle(valid.begin(), valid.end(), rng);
        KNN_CUDA_TRY(cudaMemcpyAsync(d_idx, valid.data(), sizeof(int32_t) * valid.size(), cudaMemcpyHostToDevice, s));
        KNN_CUDA_TRY(cudaMemsetAsync(w.loss, 0, sizeof(float), s));
        for (int64_t bi = 0; bi < nb; bi++) {
            k_gather_batch<<<(unsigned)batch, 128, 0, s>>>(X, y, d_idx + bi * batch, batch, w.X, w.t);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
            KNN_TRY(mlp_forward(md, w, batch, w.X, s));
            k_pinball<<<launch_blocks(batch, 256), 256, 0, s>>>(w.y, w.t, batch, q, w.g, w.loss);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
            KNN_TRY(mlp_backward(md, w, batch, w.X, s));
            md->step++;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.0f - std::pow(b1, (float)md->step), c2 = 1.0f - std::pow(b2, (float)md->step);
            k_adam<<<launch_blocks(N_PARAMS, 256), 256, 0, s>>>(md->w, md->grad, md->m, md->v, md->wb, N_PARAMS, lr,
                                                                b1, b2, c1, c2, 1e-8f);
            KNN_CUDA_TRY(cudaGetLastError());
            count_launch();
        }
        float hl = 0.0f;
        KNN_CUDA_TRY(cudaMemcpyAsync(&hl, w.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        KNN_CUDA_TRY(cudaStreamSynchronize(s));
        KNN_TRY(gemm_check());
        last_loss = hl / (double)(nb * batch);
    }
    if (final_loss) *final_loss = (float)last_loss;
    return KNN_OK;
}

extern "C" knn_status knn_threshold_model_predict(const knn_model* md, const knn_csr* R, float* out_tau,
                                                 void* stream_) {
    if (!md) return fail(KNN_EINVAL, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream_;
    Buffers tmp(s);
    DevCSR r;
    KNN_TRY(prepare_csr(R, s, tmp, true, false, &r));
    if (r.n_rows == 0) return KNN_OK;
    if (!out_tau) return fail(KNN_EINVAL, "out_tau is NULL");
    KNN_TRY(model_predict_tau(md, r, 1.0f, out_tau, s, tmp));
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    return gemm_check();
}

extern "C" knn_status knn_threshold_model_calibrate(knn_model* md, const knn_csr* Q, const float* kth_scores,
                                                   float miss_rate, float* out_scale, void* stream_) {
    if (!md || !Q || !kth_scores) return fail(KNN_EINVAL, "NULL argument");
    if (!(miss_rate >= 0.0f && miss_rate < 1.0f)) return fail(KNN_EINVAL, "miss_rate must be in [0, 1)");
    cudaStream_t s = (cudaStream_t)stream_;
    Buffers tmp(s);
    DevCSR q;
    KNN_TRY(prepare_csr(Q, s, tmp, true, false, &q));
    if (q.n_rows == 0) return fail(KNN_EINVAL, "no calibration queries");
    float* tau = nullptr;
    float* ratio = nullptr;
    KNN_TRY(tmp.get(&tau, (size_t)q.n_rows));
    KNN_TRY(tmp.get(&ratio, (size_t)q.n_rows));
    KNN_TRY(model_predict_tau(md, q, 1.0f, tau, s, tmp));
    k_kth_ratio<<<launch_blocks(q.n_rows, 256), 256, 0, s>>>(kth_scores, tau, q.n_rows, ratio);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    std::vector<float> h((size_t)q.n_rows);
    KNN_CUDA_TRY(cudaMemcpyAsync(h.data(), ratio, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, s));
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    KNN_TRY(gemm_check());
    // A row falls back iff scale * tau > kth, i.e. scale > kth / tau.  The value at rank
    // floor(miss_rate * n) leaves at most that many rows of Q below it; it is stepped down
    // by a relative 1e-6 so that the rounding of scale * tau cannot lift the row at that
    // rank (or rows tied with it) above their k-th score.
    const size_t idx = std::min(h.size() - 1, (size_t)std::floor((double)miss_rate * (double)h.size()));
    std::nth_element(h.begin(), h.begin() + (ptrdiff_t)idx, h.end());
    float scale = (float)((double)h[idx] * (1.0 - 1e-6));
    if (!(scale < 3.0e38f)) return fail(KNN_EINVAL, "too few calibration rows with a k-th score");
    if (!(scale > 0.0f)) scale = 1.0e-30f;
    md->tau_scale = scale;
    if (out_scale) *out_scale = scale;
    return KNN_OK;
}

extern "C" knn_status knn_threshold_model_get_params(const knn_model* md, void* host_buf, size_t bytes,
                                                    size_t* needed) {
    if (!md) return fail(KNN_EINVAL, "model is NULL");
    const size_t need = sizeof(uint32_t) * 2 + sizeof(int64_t) + sizeof(float) * (3 * N_PARAMS + 1);
    if (needed) *needed = need;
    if (!host_buf) return KNN_OK;
    if (bytes < need) return fail(KNN_EINVAL, "buffer of %zu bytes, %zu needed", bytes, need);
    unsigned char* p = (unsigned char*)host_buf;
    uint32_t hdr[2] = {0x4b4e4e4du, md->hash_seed};   // "KNNM", hash seed
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    memcpy(p, &md->step, sizeof(int64_t));
    p += sizeof(int64_t);
    KNN_CUDA_TRY(cudaMemcpyAsync(p, md->w, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, md->stream));
    KNN_CUDA_TRY(cudaMemcpyAsync(p + sizeof(float) * N_PARAMS, md->m, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost,
                                 md->stream));
    KNN_CUDA_TRY(cudaMemcpyAsync(p + 2 * sizeof(float) * N_PARAMS, md->v, sizeof(float) * N_PARAMS,
                                 cudaMemcpyDeviceToHost, md->stream));
    memcpy(p + 3 * sizeof(float) * N_PARAMS, &md->tau_scale, sizeof(float));
    KNN_CUDA_TRY(cudaStreamSynchronize(md->stream));
    return KNN_OK;
}

extern "C" knn_status knn_threshold_model_set_params(knn_model* md, const void* host_buf, size_t bytes) {
    if (!md || !host_buf) return fail(KNN_EINVAL, "NULL argument");
    const size_t need = sizeof(uint32_t) * 2 + sizeof(int64_t) + sizeof(float) * (3 * N_PARAMS + 1);
    if (bytes < need) return fail(KNN_EINVAL, "buffer of %zu bytes, %zu needed", bytes, need);
    const unsigned char* p = (const unsigned char*)host_buf;
    uint32_t hdr[2];
    memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != 0x4b4e4e4du) return fail(KNN_EINVAL, "not a threshold model parameter buffer");
    md->hash_seed = hdr[1];
    p += sizeof(hdr);
    memcpy(&md->step, p, sizeof(int64_t));
    p += sizeof(int64_t);
    KNN_CUDA_TRY(cudaMemcpyAsync(md->w, p, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, md->stream));
    KNN_CUDA_TRY(cudaMemcpyAsync(md->m, p + sizeof(float) * N_PARAMS, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice,
                                 md->stream));
    KNN_CUDA_TRY(cudaMemcpyAsync(md->v, p + 2 * sizeof(float) * N_PARAMS, sizeof(float) * N_PARAMS,
                                 cudaMemcpyHostToDevice, md->stream));
    float scale = 1.0f;
    memcpy(&scale, p + 3 * sizeof(float) * N_PARAMS, sizeof(float));
    if (!(scale > 0.0f) || !(scale < 3.0e38f)) return fail(KNN_EINVAL, "stored tau scale %g is not a positive number", scale);
    md->tau_scale = scale;
    k_to_bf16<<<launch_blocks(N_PARAMS, 256), 256, 0, md->stream>>>(md->w, md->wb, N_PARAMS);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    KNN_CUDA_TRY(cudaStreamSynchronize(md->stream));
    return KNN_OK;
}

// ---------------------------------------------------------------------------------
// test hooks: one forward/backward step on given inputs (sketch bypassed)
// ---------------------------------------------------------------------------------
extern "C" knn_status knn_threshold_model_forward_backward(knn_model* md, const void* x_bf16, const float* target,
                                                          int64_t B, float quantile, float* out_pred,
                                                          float* out_grads, void* stream_) {
    if (!md || !x_bf16 || !target || B < 1) return fail(KNN_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream_;
    Buffers tmp(s);
    MlpWork w;
    KNN_TRY(w.alloc(tmp, B));
    KNN_CUDA_TRY(cudaMemcpyAsync(w.X, x_bf16, sizeof(__nv_bfloat16) * B * IN_PAD, cudaMemcpyDeviceToDevice, s));
    KNN_CUDA_TRY(cudaMemcpyAsync(w.t, target, sizeof(float) * B, cudaMemcpyDeviceToDevice, s));
    KNN_CUDA_TRY(cudaMemsetAsync(w.loss, 0, sizeof(float), s));
    KNN_TRY(mlp_forward(md, w, B, w.X, s));
    k_pinball<<<launch_blocks(B, 256), 256, 0, s>>>(w.y, w.t, B, quantile, w.g, w.loss);
    KNN_CUDA_TRY(cudaGetLastError());
    count_launch();
    KNN_TRY(mlp_backward(md, w, B, w.X, s));
    if (out_pred) KNN_CUDA_TRY(cudaMemcpyAsync(out_pred, w.y, sizeof(float) * B, cudaMemcpyDeviceToDevice, s));
    if (out_grads)
        KNN_CUDA_TRY(cudaMemcpyAsync(out_grads, md->grad, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToDevice, s));
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    return gemm_check();
}

extern "C" knn_status knn_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int64_t sam, int64_t sak,
                                    const void* B, int64_t sbk, int64_t sbn, float* C, int64_t scm, int64_t scn,
                                    int32_t accumulate, void* stream) {
    if (M < 0 || N < 0 || K < 0 || (M && N && (!A || !B || !C))) return fail(KNN_EINVAL, "bad GEMM arguments");
    KNN_TRY(gemm(M, N, K, (const __nv_bfloat16*)A, sam, sak, (const __nv_bfloat16*)B, sbk, sbn, C, scm, scn,
                 accumulate != 0, (cudaStream_t)stream));
    KNN_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return gemm_check();
}

extern "C" knn_status knn_threshold_sketch(const knn_model* md, const knn_csr* R, void* out_x_bf16, void* stream_) {
    if (!md || !out_x_bf16) return fail(KNN_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream_;
    Buffers tmp(s);
    DevCSR r;
    KNN_TRY(prepare_csr(R, s, tmp, true, false, &r));
    KNN_TRY(sketch(r, md->hash_seed, (__nv_bfloat16*)out_x_bf16, s));
    KNN_CUDA_TRY(cudaStreamSynchronize(s));
    return KNN_OK;
}

extern "C" knn_status knn_threshold_model_params(const knn_model* md, const float** w, int64_t* n) {
    if (!md || !w || !n) return fail(KNN_EINVAL, "NULL argument");
    *w = md->w;
    *n = md->n_params;
    return KNN_OK;
}

// mlp.cu -- the learned selectivity estimator beside the exact COUNT.
//
// The paper computes selectivity exactly (§3.1); this module adds a small
// surrogate that answers from predicate features alone and falls back to the
// exact batched count whenever its predicted uncertainty is too high, so the
// exact answer stays one threshold away for every probe.
//
//  * a6 features: per-column empirical CDFs from a SplitMix64 sample of rows
//    (sorted order keys), and for each predicate in OR-of-ANDs form up to six
//    24-float clause slots (column / operator / group one-hots, NOT flag,
//    [F_lo, F_hi] from the CDF, the leaf's log selectivity).
//  * a7 forward: 144 -> 256 -> 256 -> 256 on the tensor cores (gemm.cu, BF16
//    operands, FP32 accumulation in TMEM, bias + ReLU fused), and the 256 -> 2
//    head (mu and log sigma^2 of y = ln(1 + count)) on the CUDA cores.
//  * a8 backward + Adam: Gaussian NLL gradients; the five products of the
//    backward pass also run on the tensor cores (ReLU gradient and bias-grad
//    column sums fused); Adam on FP32 masters writes the BF16 weight copies
//    (and the transposes the backward products read).
//  * a9 gate: sigma = exp(lv / 2) > tau (or a predicate without a feature
//    form) -> exact count from one batched scan; otherwise exp(mu) - 1.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <random>
#include <vector>

#include "gemm.h"
#include "internal.h"

namespace sel {
namespace mlpk {

constexpr int kSlots = 6, kSlot = 24, kFeat = kSlots * kSlot, kHid = 256, kCols = 8;
constexpr float kLvMin = -8.f, kLvMax = 8.f;
// flat parameter layout: W1 b1 W2 b2 W3 b3 W4 b4
constexpr int64_t oW1 = 0, oB1 = oW1 + kHid * kFeat, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid,
                  oW3 = oB2 + kHid, oB3 = oW3 + kHid * kHid, oW4 = oB3 + kHid, oB4 = oW4 + 2 * kHid,
                  kParams = oB4 + 2;

__host__ __device__ inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Order-preserving 64-bit keys: integers by value, binary32 by value (-0 == +0).
__host__ __device__ inline uint64_t key_int(int64_t v) { return static_cast<uint64_t>(v) ^ 0x8000000000000000ull; }
__host__ __device__ inline uint64_t key_f32(float f) {
    if (f == 0.f) f = 0.f;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return static_cast<uint64_t>(u);
}

struct FeatClause {
    int32_t col, opi, neg, group;
    int32_t mode, set_n, present, pad;
    uint64_t ka, kb;
    uint64_t set_off;
};
enum { M_EQ = 0, M_LT = 1, M_LE = 2, M_GT = 3, M_GE = 4, M_BETWEEN = 5, M_SET = 6 };

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------

// One CTA per column: m sampled order keys, bitonic-sorted in shared memory.
__global__ void __launch_bounds__(1024) cdf_kernel(const uint8_t* const* cols, const int32_t* types, int64_t n,
                                                   int32_t m, uint64_t seed, uint64_t* keys) {
    extern __shared__ uint64_t sk[];
    const int c = blockIdx.x;
    const uint8_t* col = cols[c];
    const int ty = types[c];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const uint64_t z = seed + (static_cast<uint64_t>(c + 1) << 40) + static_cast<uint64_t>(i);
        const int64_t idx = static_cast<int64_t>(splitmix64(z) % static_cast<uint64_t>(n));
        uint64_t k;
        if (ty == SEL_I64) k = key_int(reinterpret_cast<const int64_t*>(col)[idx]);
        else if (ty == SEL_F32) k = key_f32(reinterpret_cast<const float*>(col)[idx]);
        else k = key_int(reinterpret_cast<const int32_t*>(col)[idx]);
        sk[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t a = sk[i], b = sk[j];
                    if ((a > b) == up) {
                        sk[i] = b;
                        sk[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) keys[static_cast<size_t>(c) * m + i] = sk[i];
}

__device__ inline int lower_bound_u64(const uint64_t* a, int n, uint64_t k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ inline int upper_bound_u64(const uint64_t* a, int n, uint64_t k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One warp per (predicate, slot): writes the slot's 24 features (bf16).  The
// lanes split a set's values (an IN list, or the codes of a LIKE prefix);
// lane 0 does the other comparisons.
__global__ void featurize_kernel(const FeatClause* cl, const uint64_t* set_keys, const uint64_t* cdf, int32_t m,
                                 int32_t n, __nv_bfloat16* feat) {
    const int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (t >= static_cast<int64_t>(n) * kSlots) return;   // whole warps leave together
    const FeatClause c = cl[t];
    const uint64_t* s = cdf + static_cast<size_t>(c.present ? c.col : 0) * m;
    const float fm = static_cast<float>(m);
    auto frac = [&](int k) { return static_cast<float>(k) / fm; };
    float lo = 0.f, hi = 0.f;
    if (c.present && c.mode == M_SET) {   // sample mass of a set of values
        int cnt = 0;
        for (int j = static_cast<int>(lane); j < c.set_n; j += 32) {
            const uint64_t k = set_keys[c.set_off + j];
            cnt += upper_bound_u64(s, m, k) - lower_bound_u64(s, m, k);
        }
        cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        hi = frac(min(cnt, m));
    }
    if (lane != 0) return;
    float f[kSlot];
#pragma unroll
    for (int i = 0; i < kSlot; ++i) f[i] = 0.f;
    if (c.present) {
        switch (c.mode) {
        case M_EQ: lo = frac(lower_bound_u64(s, m, c.ka)); hi = frac(upper_bound_u64(s, m, c.ka)); break;
        case M_LT: hi = frac(lower_bound_u64(s, m, c.ka)); break;
        case M_LE: hi = frac(upper_bound_u64(s, m, c.ka)); break;
        case M_GT: lo = frac(upper_bound_u64(s, m, c.ka)); hi = 1.f; break;
        case M_GE: lo = frac(lower_bound_u64(s, m, c.ka)); hi = 1.f; break;
        case M_BETWEEN: {
            const int a = lower_bound_u64(s, m, c.ka);
            lo = frac(a);
            hi = frac(max(a, upper_bound_u64(s, m, c.kb)));
            break;
        }
        default: break;   // M_SET: done above
        }
        // log selectivity of the leaf from the sample, in [-1, 0]: ln(max(p, 1/(2m))) / ln(2m),
        // p = hi - lo, complemented for <> and for a negated leaf (evaluated in double)
        double p = fmax((double)hi - (double)lo, 0.0);
        if (c.opi == 1) p = 1.0 - p;
        if (c.neg) p = 1.0 - p;
        const float ls = (float)(log(fmax(p, 0.5 / (double)m)) / log(2.0 * (double)m));
        f[c.col] = 1.f;
        f[8 + c.opi] = 1.f;
        f[17] = c.neg ? 1.f : 0.f;
        f[18] = lo;
        f[19] = hi;
        f[20 + c.group] = 1.f;
        f[23] = ls;
    }
    __nv_bfloat16* dst = feat + t * kSlot;   // slot s of predicate p starts at (p * 6 + s) * 24
#pragma unroll
    for (int i = 0; i < kSlot; ++i) dst[i] = __float2bfloat16_rn(f[i]);
}

// out[i] = (mu, raw log-variance) = a3[i] . W4^T + b4 (one row per thread).
// With y != nullptr also the training head: the loss and dO of each row, then
// (one hidden unit per thread, over the block's rows) dZ3 = (dO W4) * (a3 > 0)
// as bf16 rows and the db3, dW4, db4 and loss sums.
__global__ void __launch_bounds__(128) head_kernel(const __nv_bfloat16* a3, const __nv_bfloat16* w4b,
                                                   const float* b4, int32_t n, float* out, const float* y,
                                                   int32_t bsz, __nv_bfloat16* dz3, float* g_b3, float* g_w4,
                                                   float* g_b4, float* loss_sum) {
    __shared__ float w[2][kHid];
    __shared__ float sd[2][128];   // dO of the block's rows
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        w[0][k] = __bfloat162float(w4b[k]);
        w[1][k] = __bfloat162float(w4b[kHid + k]);
    }
    __syncthreads();
    const int r0 = blockIdx.x * blockDim.x;
    const int i = r0 + threadIdx.x;
    const bool ok = i < n;
    const __nv_bfloat16* row = a3 + static_cast<size_t>(ok ? i : 0) * kHid;
    float o0 = 0.f, o1 = 0.f;
    for (int k = 0; k < kHid; k += 8) {
        const uint4 v = *reinterpret_cast<const uint4*>(row + k);
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float a = __bfloat162float(h[j]);
            o0 = fmaf(a, w[0][k + j], o0);
            o1 = fmaf(a, w[1][k + j], o1);
        }
    }
    o0 += b4[0];
    o1 += b4[1];
    if (ok) {
        out[2 * static_cast<size_t>(i)] = o0;
        out[2 * static_cast<size_t>(i) + 1] = o1;
    }
    if (!y) return;
    float d0 = 0.f, d1 = 0.f, li = 0.f;
    if (ok) {
        const float lv = fminf(fmaxf(o1, kLvMin), kLvMax);
        const float inv = expf(-lv);
        const float r = y[i] - o0;
        li = 0.5f * (lv + r * r * inv);
        d0 = -r * inv / static_cast<float>(bsz);
        d1 = (o1 > kLvMin && o1 < kLvMax) ? 0.5f * (1.f - r * r * inv) / static_cast<float>(bsz) : 0.f;
    }
    sd[0][threadIdx.x] = d0;
    sd[1][threadIdx.x] = d1;
    const uint32_t lane = threadIdx.x & 31u;
    float t0 = d0, t1 = d1, tl = li;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xFFFFFFFFu, t0, o);
        t1 += __shfl_xor_sync(0xFFFFFFFFu, t1, o);
        tl += __shfl_xor_sync(0xFFFFFFFFu, tl, o);
    }
    if (lane == 0) {
        atomicAdd(&g_b4[0], t0);
        atomicAdd(&g_b4[1], t1);
        atomicAdd(loss_sum, tl);
    }
    __syncthreads();
    const int nr = min(static_cast<int>(blockDim.x), n - r0);
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        const float w0 = w[0][k], w1 = w[1][k];
        for (int r = 0; r < nr; ++r) {
            const size_t at = static_cast<size_t>(r0 + r) * kHid + k;
            const float a = __bfloat162float(a3[at]);
            const float e0 = sd[0][r], e1 = sd[1][r];
            const float dz = (a > 0.f) ? e0 * w0 + e1 * w1 : 0.f;
            dz3[at] = __float2bfloat16_rn(dz);
            s0 += dz;
            s1 = fmaf(e0, a, s1);
            s2 = fmaf(e1, a, s2);
        }
        atomicAdd(&g_b3[k], s0);
        atomicAdd(&g_w4[k], s1);
        atomicAdd(&g_w4[kHid + k], s2);
    }
}

// Transpose a bf16 [rows x cols] matrix into [cols x rows].
__global__ void transpose_bf16(const __nv_bfloat16* src, int rows, int cols, __nv_bfloat16* dst) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 32 + threadIdx.y;
    for (int j = 0; j < 32; j += 8)
        if (y + j < rows && x < cols) tile[threadIdx.y + j][threadIdx.x] = src[static_cast<size_t>(y + j) * cols + x];
    __syncthreads();
    const int tx = blockIdx.y * 32 + threadIdx.x, ty = blockIdx.x * 32 + threadIdx.y;
    for (int j = 0; j < 32; j += 8)
        if (ty + j < cols && tx < rows) dst[static_cast<size_t>(ty + j) * rows + tx] = tile[threadIdx.x][threadIdx.y + j];
}

// Rows idx[i] of (feat, y) into the minibatch buffers.
__global__ void gather_kernel(const __nv_bfloat16* feat, const float* y, const int32_t* idx, int32_t b,
                              __nv_bfloat16* xb, float* yb) {
    const int i = blockIdx.x;
    const int src = idx[i];
    for (int k = threadIdx.x; k < kFeat / 8; k += blockDim.x)
        reinterpret_cast<uint4*>(xb + static_cast<size_t>(i) * kFeat)[k] =
            reinterpret_cast<const uint4*>(feat + static_cast<size_t>(src) * kFeat)[k];
    if (threadIdx.x == 0) yb[i] = y[src];
}

// Adam on the FP32 masters (then the gradient is cleared) and the BF16 copies.
__global__ void adam_kernel(float* p, float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16* w1b, __nv_bfloat16* w2b, __nv_bfloat16* w3b,
                            __nv_bfloat16* w4b, __nv_bfloat16* w2t, __nv_bfloat16* w3t, int update) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float w = p[i];
    if (update) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = w;
        g[i] = 0.f;
    }
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    if (i < oB1) {
        w1b[i - oW1] = wb;
    } else if (i >= oW2 && i < oB2) {
        const int64_t j = i - oW2;
        w2b[j] = wb;
        w2t[(j % kHid) * kHid + j / kHid] = wb;
    } else if (i >= oW3 && i < oB3) {
        const int64_t j = i - oW3;
        w3b[j] = wb;
        w3t[(j % kHid) * kHid + j / kHid] = wb;
    } else if (i >= oW4 && i < oB4) {
        w4b[i - oW4] = wb;
    }
}

}  // namespace mlpk
}  // namespace sel

using namespace sel;
using namespace sel::mlpk;

// ----------------------------------------------------------------------------
// model object
// ----------------------------------------------------------------------------

struct sel_mlp {
    int32_t n_cols = 0, m = 0;
    uint64_t seed = 0;
    int64_t step = 0;
    std::vector<int32_t> types;
    // device state
    float *p = nullptr, *g = nullptr, *mm = nullptr, *vv = nullptr;
    __nv_bfloat16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w4b = nullptr, *w2t = nullptr, *w3t = nullptr;
    uint64_t* cdf = nullptr;   // n_cols x m sorted keys
    unsigned int* err = nullptr;
    float* loss = nullptr;
    // activation buffers (grown to the largest batch)
    int cap = 0;
    __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *a1t = nullptr, *a2t = nullptr, *xt = nullptr;
    __nv_bfloat16 *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr, *dz1t = nullptr, *dz2t = nullptr, *dz3t = nullptr;
    float* out = nullptr;
    bool fused = true;   // inference in one kernel (gemm.cu); false: layer by layer as in training
    std::vector<void*> owned;
    // featurize staging: pinned host block -> device block, reused across calls;
    // stage_done marks the end of the last copy out of the host block
    uint8_t* h_stage = nullptr;
    uint8_t* d_stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t stage_done = nullptr;
    // what the device staging block holds: the predicates (by id) whose clause
    // records were uploaded last, their featurizable flags and offsets; a call
    // with the same predicates in the same order reuses it
    std::vector<uint64_t> stage_ids;
    std::vector<uint8_t> stage_ok;
    size_t stage_keys_off = 0, stage_ok_off = 0;
    ~sel_mlp() {
        if (stage_done) cudaEventSynchronize(stage_done);
        if (h_stage) cudaFreeHost(h_stage);
        if (d_stage) cudaFree(d_stage);
        if (stage_done) cudaEventDestroy(stage_done);
        for (void* q : owned) cudaFree(q);
    }
};

namespace {

template <typename T>
sel_status dalloc(sel_mlp* m, T** p, size_t count, const char* what) {
    void* q = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&q), std::max<size_t>(count * sizeof(T), 256));
    if (e != cudaSuccess) {
        set_error("%s: cudaMalloc: %s", what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SEL_ERR_OOM : SEL_ERR_CUDA;
    }
    m->owned.push_back(q);
    *p = static_cast<T*>(q);
    return SEL_OK;
}

#define MLP_TRY(x)                       \
    do {                                 \
        sel_status s__ = (x);            \
        if (s__ != SEL_OK) return s__;   \
    } while (0)

sel_status cuda_ok(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return SEL_OK;
    set_error("%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SEL_ERR_OOM : SEL_ERR_CUDA;
}

sel_status ensure_batch(sel_mlp* m, int n) {
    if (n <= m->cap) return SEL_OK;
    const int cap = (n + 127) / 128 * 128;
    // earlier, smaller buffers stay in `owned` and are freed with the model
    MLP_TRY(dalloc(m, &m->a1, (size_t)cap * kHid, "activations"));
    MLP_TRY(dalloc(m, &m->a2, (size_t)cap * kHid, "activations"));
    MLP_TRY(dalloc(m, &m->a3, (size_t)cap * kHid, "activations"));
    MLP_TRY(dalloc(m, &m->a1t, (size_t)cap * kHid, "activations"));
    MLP_TRY(dalloc(m, &m->a2t, (size_t)cap * kHid, "activations"));
    MLP_TRY(dalloc(m, &m->xt, (size_t)cap * kFeat, "activations"));
    MLP_TRY(dalloc(m, &m->dz1, (size_t)cap * kHid, "gradients"));
    MLP_TRY(dalloc(m, &m->dz2, (size_t)cap * kHid, "gradients"));
    MLP_TRY(dalloc(m, &m->dz3, (size_t)cap * kHid, "gradients"));
    MLP_TRY(dalloc(m, &m->dz1t, (size_t)cap * kHid, "gradients"));
    MLP_TRY(dalloc(m, &m->dz2t, (size_t)cap * kHid, "gradients"));
    MLP_TRY(dalloc(m, &m->dz3t, (size_t)cap * kHid, "gradients"));
    MLP_TRY(dalloc(m, &m->out, (size_t)cap * 2, "outputs"));
    m->cap = cap;
    return SEL_OK;
}

GemmArgs gemm(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb, int M, int N, int K,
              int epi, unsigned int* err) {
    GemmArgs g{};
    g.A = A;
    g.B = B;
    g.lda = lda;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epi;
    g.err = err;
    return g;
}

sel_status run_gemm(const GemmArgs& g, int splits, cudaStream_t st) {
    ++thread_launches();
    return cuda_ok(launch_gemm(g, splits, st), "tensor-core GEMM launch");
}

// a7: activations a1..a3 (and a1t, a2t when training) and out for n rows of features x.
// Inference (the default) runs as one kernel that keeps the activations in
// shared memory and writes only out.
sel_status forward(sel_mlp* m, const __nv_bfloat16* x, int n, bool training, cudaStream_t st) {
    MLP_TRY(ensure_batch(m, n));
    if (!training && m->fused) {
        MlpFwdArgs f{};
        f.x = x;
        f.w[0] = m->w1b;
        f.w[1] = m->w2b;
        f.w[2] = m->w3b;
        f.b[0] = m->p + oB1;
        f.b[1] = m->p + oB2;
        f.b[2] = m->p + oB3;
        f.w4 = m->w4b;
        f.b4 = m->p + oB4;
        f.out = m->out;
        f.n = n;
        f.err = m->err;
        ++thread_launches();
        return cuda_ok(launch_mlp_forward(f, st), "fused estimator forward launch");
    }
    GemmArgs g = gemm(x, kFeat, m->w1b, kFeat, n, kHid, kFeat, EPI_BIAS_RELU, m->err);
    g.bias = m->p + oB1;
    g.out = m->a1;
    g.ldo = kHid;
    if (training) {
        g.outT = m->a1t;
        g.ldoT = n;
    }
    MLP_TRY(run_gemm(g, 1, st));
    g = gemm(m->a1, kHid, m->w2b, kHid, n, kHid, kHid, EPI_BIAS_RELU, m->err);
    g.bias = m->p + oB2;
    g.out = m->a2;
    g.ldo = kHid;
    if (training) {
        g.outT = m->a2t;
        g.ldoT = n;
    }
    MLP_TRY(run_gemm(g, 1, st));
    g = gemm(m->a2, kHid, m->w3b, kHid, n, kHid, kHid, EPI_BIAS_RELU, m->err);
    g.bias = m->p + oB3;
    g.out = m->a3;
    g.ldo = kHid;
    MLP_TRY(run_gemm(g, 1, st));
    if (!training) {
        ++thread_launches();
        head_kernel<<<(n + 127) / 128, 128, 0, st>>>(m->a3, m->w4b, m->p + oB4, n, m->out, nullptr, n, nullptr,
                                                      nullptr, nullptr, nullptr, nullptr);
        MLP_TRY(cuda_ok(cudaGetLastError(), "head launch"));
    }
    return SEL_OK;
}

// a8: loss and gradients (accumulated into m->g) for a minibatch; n % 8 == 0.
sel_status backward(sel_mlp* m, const __nv_bfloat16* x, const float* y, int n, cudaStream_t st) {
    MLP_TRY(forward(m, x, n, true, st));
    dim3 tb(32, 8), tg((kFeat + 31) / 32, (n + 31) / 32);
    ++thread_launches();
    transpose_bf16<<<tg, tb, 0, st>>>(x, n, kFeat, m->xt);
    ++thread_launches();
    head_kernel<<<(n + 127) / 128, 128, 0, st>>>(m->a3, m->w4b, m->p + oB4, n, m->out, y, n, m->dz3, m->g + oB3,
                                                  m->g + oW4, m->g + oB4, m->loss);
    MLP_TRY(cuda_ok(cudaGetLastError(), "head launch"));
    ++thread_launches();
    transpose_bf16<<<dim3((kHid + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, st>>>(m->dz3, n, kHid, m->dz3t);
    const int splits = std::max(1, std::min(32, n / 256));
    // dW3 = dZ3^T A2 ; dA2 = dZ3 W3 -> dZ2 (ReLU gradient), db2
    GemmArgs g = gemm(m->dz3t, n, m->a2t, n, kHid, kHid, n, EPI_F32, m->err);
    g.C = m->g + oW3;
    g.ldc = kHid;
    MLP_TRY(run_gemm(g, splits, st));
    g = gemm(m->dz3, kHid, m->w3t, kHid, n, kHid, kHid, EPI_DRELU, m->err);
    g.mask = m->a2;
    g.ldm = kHid;
    g.out = m->dz2;
    g.ldo = kHid;
    g.outT = m->dz2t;
    g.ldoT = n;
    g.colsum = m->g + oB2;
    MLP_TRY(run_gemm(g, 1, st));
    // dW2 = dZ2^T A1 ; dA1 = dZ2 W2 -> dZ1, db1
    g = gemm(m->dz2t, n, m->a1t, n, kHid, kHid, n, EPI_F32, m->err);
    g.C = m->g + oW2;
    g.ldc = kHid;
    MLP_TRY(run_gemm(g, splits, st));
    g = gemm(m->dz2, kHid, m->w2t, kHid, n, kHid, kHid, EPI_DRELU, m->err);
    g.mask = m->a1;
    g.ldm = kHid;
    g.out = m->dz1;
    g.ldo = kHid;
    g.outT = m->dz1t;
    g.ldoT = n;
    g.colsum = m->g + oB1;
    MLP_TRY(run_gemm(g, 1, st));
    // dW1 = dZ1^T X
    g = gemm(m->dz1t, n, m->xt, n, kHid, kFeat, n, EPI_F32, m->err);
    g.C = m->g + oW1;
    g.ldc = kFeat;
    MLP_TRY(run_gemm(g, splits, st));
    return SEL_OK;
}

sel_status adam(sel_mlp* m, const sel_train_cfg* cfg, bool update, cudaStream_t st) {
    float c1 = 1.f, c2 = 1.f;
    if (update) {
        m->step++;
        c1 = (float)(1.0 / (1.0 - std::pow((double)cfg->beta1, (double)m->step)));
        c2 = (float)(1.0 / (1.0 - std::pow((double)cfg->beta2, (double)m->step)));
    }
    ++thread_launches();
    adam_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, st>>>(
        m->p, m->g, m->mm, m->vv, cfg ? cfg->lr : 0.f, cfg ? cfg->beta1 : 0.f, cfg ? cfg->beta2 : 0.f,
        cfg ? cfg->eps : 1.f, c1, c2, m->w1b, m->w2b, m->w3b, m->w4b, m->w2t, m->w3t, update ? 1 : 0);
    return cuda_ok(cudaGetLastError(), "adam launch");
}

sel_status check_pred_schema(const sel_mlp* m, const sel_pred* p) {
    if (!p) {
        set_error("learned estimator: predicate is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    for (size_t c = 0; c < p->col_types.size() && c < m->types.size(); ++c)
        if (p->col_types[c] != m->types[c]) {
            set_error("learned estimator: predicate compiled for another schema (column %zu)", c);
            return SEL_ERR_TYPE;
        }
    return SEL_OK;
}

// Feature form of one predicate: kSlots clause records (set_off relative to
// the predicate's own key list) or false when the predicate has none.  Depends
// only on the predicate (its dictionary codes and the column types it was
// compiled against), so it is built once and kept with the predicate.
bool pred_features(const sel_pred* p, FeatClause* rec, std::vector<uint64_t>& keys, int32_t& max_col) {
    for (int s = 0; s < kSlots; ++s) rec[s] = FeatClause{};
    keys.clear();
    max_col = -1;
    if (!p->dnf_ok || p->dnf.empty() || p->dnf.size() > 3) return false;
    size_t total = 0;
    for (auto& g : p->dnf) {
        total += g.size();
        for (auto& c : g) {
            if (c.col >= kCols) return false;
            max_col = std::max(max_col, c.col);
        }
    }
    if (total > (size_t)kSlots) return false;
    int s = 0;
    for (size_t gi = 0; gi < p->dnf.size(); ++gi) {
        for (const Clause& c : p->dnf[gi]) {
            FeatClause& f = rec[s++];
            f.present = 1;
            f.col = c.col;
            f.neg = c.nnf_neg;
            f.group = (int32_t)gi;
            const bool isf = p->col_types[c.col] == SEL_F32;
            auto key = [&](int64_t iv, float fv) { return isf ? key_f32(fv) : key_int(iv); };
            if (c.kind == SEL_N_CMP) {
                f.opi = c.op;
                f.mode = (c.op == SEL_EQ || c.op == SEL_NE) ? M_EQ
                         : c.op == SEL_LT                  ? M_LT
                         : c.op == SEL_LE                  ? M_LE
                         : c.op == SEL_GT                  ? M_GT
                                                           : M_GE;
                f.ka = key(c.raw_i0, c.raw_f0);
            } else if (c.kind == SEL_N_BETWEEN) {
                f.opi = 6;
                f.mode = M_BETWEEN;
                f.ka = key(c.raw_i0, c.raw_f0);
                f.kb = key(c.raw_i1, c.raw_f1);
            } else {
                f.opi = c.kind == SEL_N_IN ? 7 : 8;
                f.mode = M_SET;
                std::vector<uint64_t> ks;
                if (c.kind == SEL_N_IN) {
                    if (isf)
                        for (float v : c.fvals) ks.push_back(key_f32(v));
                    else
                        for (int64_t v : c.ivals) ks.push_back(key_int(v));
                } else {
                    for (int32_t code : c.like_codes) ks.push_back(key_int(code));
                }
                std::sort(ks.begin(), ks.end());
                ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
                f.set_off = keys.size();
                f.set_n = (int32_t)ks.size();
                keys.insert(keys.end(), ks.begin(), ks.end());
            }
        }
    }
    return true;
}

// Host side of a6: clause records of n predicates (ok = 0 where a predicate
// has no feature form), from each predicate's cached feature form.
sel_status build_clauses(const sel_mlp* m, const sel_pred* const* preds, int32_t n, std::vector<FeatClause>& cl,
                         std::vector<uint64_t>& set_keys, std::vector<uint8_t>& ok) {
    cl.assign((size_t)n * kSlots, FeatClause{});
    ok.assign((size_t)n, 0);
    set_keys.clear();
    for (int32_t i = 0; i < n; ++i) {
        MLP_TRY(check_pred_schema(m, preds[i]));
        sel_pred* p = const_cast<sel_pred*>(preds[i]);
        std::lock_guard<std::mutex> g(p->mu);
        if (!p->feat_built) {
            p->feat_rec.resize(kSlots * sizeof(FeatClause));
            p->feat_ok = pred_features(p, reinterpret_cast<FeatClause*>(p->feat_rec.data()), p->feat_keys,
                                       p->feat_max_col);
            p->feat_built = true;
        }
        if (!p->feat_ok || p->feat_max_col >= m->n_cols) continue;
        FeatClause* dst = &cl[(size_t)i * kSlots];
        std::memcpy(dst, p->feat_rec.data(), kSlots * sizeof(FeatClause));
        for (int s = 0; s < kSlots; ++s)
            if (dst[s].mode == M_SET) dst[s].set_off += set_keys.size();
        set_keys.insert(set_keys.end(), p->feat_keys.begin(), p->feat_keys.end());
        ok[i] = 1;
    }
    return SEL_OK;
}

struct DeviceVec {
    void* p = nullptr;
    ~DeviceVec() {
        if (p) cudaFree(p);
    }
};

// Makes the staging blocks hold `bytes`; waits for the last copy out of the
// host block, so the caller may overwrite it.
sel_status stage_reserve(sel_mlp* m, size_t bytes) {
    if (!m->stage_done) MLP_TRY(cuda_ok(cudaEventCreateWithFlags(&m->stage_done, cudaEventDisableTiming), "featurize"));
    MLP_TRY(cuda_ok(cudaEventSynchronize(m->stage_done), "featurize"));
    if (bytes <= m->stage_cap) return SEL_OK;
    const size_t cap = std::max<size_t>(bytes, 2 * m->stage_cap);
    if (m->h_stage) cudaFreeHost(m->h_stage);
    if (m->d_stage) cudaFree(m->d_stage);
    m->h_stage = m->d_stage = nullptr;
    m->stage_cap = 0;
    MLP_TRY(cuda_ok(host_alloc(reinterpret_cast<void**>(&m->h_stage), cap), "featurize staging"));
    MLP_TRY(cuda_ok(dev_alloc(reinterpret_cast<void**>(&m->d_stage), cap), "featurize staging"));
    m->stage_cap = cap;
    return SEL_OK;
}

// a6 on n predicates: host clause records -> one pinned copy -> featurize_kernel.
// Asynchronous on st (the staging block is protected by stage_done).
sel_status featurize(sel_mlp* m, cudaStream_t st, const sel_pred* const* preds, int32_t n, __nv_bfloat16* feat,
                     std::vector<uint8_t>* ok_out, uint8_t* dev_ok) {
    // predicates are immutable and their ids unique: the same ids in the same
    // order mean the staged clause records are still the right ones
    std::vector<uint64_t> ids((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        if (!preds[i]) {
            set_error("learned estimator: predicate is NULL");
            return SEL_ERR_INVALID_ARG;
        }
        ids[(size_t)i] = preds[i]->id;
    }
    if (ids != m->stage_ids) {
        m->stage_ids.clear();
        std::vector<FeatClause> cl;
        std::vector<uint64_t> keys;
        std::vector<uint8_t> ok;
        MLP_TRY(build_clauses(m, preds, n, cl, keys, ok));
        const size_t cl_bytes = cl.size() * sizeof(FeatClause);
        const size_t keys_off = (cl_bytes + 15) / 16 * 16;
        const size_t ok_off = keys_off + (keys.size() * 8 + 15) / 16 * 16;
        const size_t total = ok_off + (size_t)n;
        MLP_TRY(stage_reserve(m, total));
        std::memcpy(m->h_stage, cl.data(), cl_bytes);
        if (!keys.empty()) std::memcpy(m->h_stage + keys_off, keys.data(), keys.size() * 8);
        std::memcpy(m->h_stage + ok_off, ok.data(), (size_t)n);
        MLP_TRY(cuda_ok(cudaMemcpyAsync(m->d_stage, m->h_stage, total, cudaMemcpyHostToDevice, st), "featurize"));
        MLP_TRY(cuda_ok(cudaEventRecord(m->stage_done, st), "featurize"));
        m->stage_ids = std::move(ids);
        m->stage_ok = std::move(ok);
        m->stage_keys_off = keys_off;
        m->stage_ok_off = ok_off;
    }
    const size_t keys_off = m->stage_keys_off, ok_off = m->stage_ok_off;
    if (dev_ok)
        MLP_TRY(cuda_ok(cudaMemcpyAsync(dev_ok, m->d_stage + ok_off, (size_t)n, cudaMemcpyDeviceToDevice, st),
                        "featurize"));
    const int64_t threads = (int64_t)n * kSlots * 32;   // one warp per (predicate, slot)
    ++thread_launches();
    featurize_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const FeatClause*>(m->d_stage), reinterpret_cast<const uint64_t*>(m->d_stage + keys_off),
        m->cdf, m->m, n, feat);
    MLP_TRY(cuda_ok(cudaGetLastError(), "featurize launch"));
    if (ok_out) *ok_out = m->stage_ok;
    return SEL_OK;
}

sel_status alloc_model(sel_mlp* m) {
    MLP_TRY(dalloc(m, &m->p, kParams, "parameters"));
    MLP_TRY(dalloc(m, &m->g, kParams, "parameters"));
    MLP_TRY(dalloc(m, &m->mm, kParams, "parameters"));
    MLP_TRY(dalloc(m, &m->vv, kParams, "parameters"));
    MLP_TRY(dalloc(m, &m->w1b, (size_t)kHid * kFeat, "weights"));
    MLP_TRY(dalloc(m, &m->w2b, (size_t)kHid * kHid, "weights"));
    MLP_TRY(dalloc(m, &m->w3b, (size_t)kHid * kHid, "weights"));
    MLP_TRY(dalloc(m, &m->w4b, (size_t)2 * kHid, "weights"));
    MLP_TRY(dalloc(m, &m->w2t, (size_t)kHid * kHid, "weights"));
    MLP_TRY(dalloc(m, &m->w3t, (size_t)kHid * kHid, "weights"));
    MLP_TRY(dalloc(m, &m->cdf, (size_t)m->n_cols * m->m, "cdf"));
    MLP_TRY(dalloc(m, &m->err, 4, "flags"));
    MLP_TRY(dalloc(m, &m->loss, 4, "flags"));
    return SEL_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------

extern "C" sel_status sel_mlp_create(sel_ctx* ctx, const sel_table* table, int32_t sample_rows, uint64_t seed,
                                     sel_mlp** out) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !table || !out || table->n_cols <= 0 || !table->cols || table->n_rows <= 0 || sample_rows < 2 ||
        sample_rows > 8192 || (sample_rows & (sample_rows - 1))) {
        set_error("sel_mlp_create: bad arguments (sample_rows: a power of two in [2, 8192]; a non-empty table)");
        return SEL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::unique_ptr<sel_mlp> m(new sel_mlp());
    cudaStream_t st = ctx_stream(ctx);
    m->n_cols = std::min<int32_t>(table->n_cols, kCols);
    m->m = sample_rows;
    m->seed = seed;
    for (int32_t c = 0; c < table->n_cols; ++c) {
        const sel_column& col = table->cols[c];
        if (col.type < SEL_I32 || col.type > SEL_DICT || !col.data) {
            set_error("sel_mlp_create: column %d has no data or an unknown type", c);
            return SEL_ERR_INVALID_ARG;
        }
        m->types.push_back(col.type);
    }
    MLP_TRY(alloc_model(m.get()));
    // He-uniform initial weights from SplitMix64, zero biases
    std::vector<float> p((size_t)kParams, 0.f);
    auto fill = [&](int64_t off, int rows, int cols) {
        const double bound = std::sqrt(6.0 / cols);
        for (int64_t i = 0; i < (int64_t)rows * cols; ++i) {
            const double u = (double)(splitmix64(seed ^ splitmix64((uint64_t)(off + i))) >> 11) * (1.0 / 9007199254740992.0);
            p[(size_t)(off + i)] = (float)((2.0 * u - 1.0) * bound);
        }
    };
    fill(oW1, kHid, kFeat);
    fill(oW2, kHid, kHid);
    fill(oW3, kHid, kHid);
    fill(oW4, 2, kHid);
    MLP_TRY(cuda_ok(cudaMemcpyAsync(m->p, p.data(), kParams * 4, cudaMemcpyHostToDevice, st), "sel_mlp_create"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->g, 0, kParams * 4, st), "sel_mlp_create"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->mm, 0, kParams * 4, st), "sel_mlp_create"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->vv, 0, kParams * 4, st), "sel_mlp_create"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->err, 0, 4, st), "sel_mlp_create"));
    MLP_TRY(adam(m.get(), nullptr, false, st));
    // CDF samples of columns 0 .. n_cols-1
    std::vector<const uint8_t*> ptrs;
    for (int32_t c = 0; c < m->n_cols; ++c) ptrs.push_back(static_cast<const uint8_t*>(table->cols[c].data));
    DeviceVec dptr, dty;
    MLP_TRY(cuda_ok(dev_alloc(&dptr.p, ptrs.size() * 8), "sel_mlp_create"));
    MLP_TRY(cuda_ok(dev_alloc(&dty.p, ptrs.size() * 4), "sel_mlp_create"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(dptr.p, ptrs.data(), ptrs.size() * 8, cudaMemcpyHostToDevice, st), "sel_mlp_create"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(dty.p, m->types.data(), ptrs.size() * 4, cudaMemcpyHostToDevice, st),
                    "sel_mlp_create"));
    const size_t smem = (size_t)sample_rows * 8;
    MLP_TRY(cuda_ok(cudaFuncSetAttribute(cdf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "sel_mlp_create"));
    ++thread_launches();
    cdf_kernel<<<m->n_cols, 1024, smem, st>>>(static_cast<const uint8_t* const*>(dptr.p),
                                             static_cast<const int32_t*>(dty.p), table->n_rows, sample_rows, seed,
                                             m->cdf);
    MLP_TRY(cuda_ok(cudaGetLastError(), "cdf launch"));
    MLP_TRY(cuda_ok(cudaStreamSynchronize(st), "sel_mlp_create"));
    *out = m.release();
    return SEL_OK;
}

extern "C" void sel_mlp_free(sel_mlp* m) { delete m; }

extern "C" sel_status sel_mlp_featurize(sel_ctx* ctx, sel_mlp* m, const sel_pred* const* preds, int32_t n,
                                        void* dev_features, uint8_t* dev_ok) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !m || !preds || n <= 0 || !dev_features) {
        set_error("sel_mlp_featurize: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    return featurize(m, ctx_stream(ctx), preds, n, static_cast<__nv_bfloat16*>(dev_features), nullptr, dev_ok);
}

extern "C" sel_status sel_mlp_forward(sel_ctx* ctx, sel_mlp* m, const void* dev_features, int32_t n, float* dev_out) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !m || !dev_features || n <= 0 || !dev_out || reinterpret_cast<uintptr_t>(dev_features) % 16) {
        set_error("sel_mlp_forward: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx_stream(ctx);
    MLP_TRY(forward(m, static_cast<const __nv_bfloat16*>(dev_features), n, false, st));
    return cuda_ok(cudaMemcpyAsync(dev_out, m->out, (size_t)n * 8, cudaMemcpyDeviceToDevice, st), "sel_mlp_forward");
}

extern "C" sel_status sel_debug_mlp_fused(sel_mlp* m, int32_t on) {
    if (!m || (on != 0 && on != 1)) {
        set_error("sel_debug_mlp_fused: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    m->fused = on == 1;
    return SEL_OK;
}

static sel_status check_cfg(const sel_train_cfg* cfg) {
    if (!cfg || !(cfg->lr >= 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
        !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f)) {
        set_error("learned estimator: bad training configuration");
        return SEL_ERR_INVALID_ARG;
    }
    return SEL_OK;
}

extern "C" sel_status sel_mlp_train_step(sel_ctx* ctx, sel_mlp* m, const void* dev_features, const float* dev_y,
                                         int32_t n, const sel_train_cfg* cfg, float* loss_out) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !m || !dev_features || !dev_y || n <= 0 || n % 8 || reinterpret_cast<uintptr_t>(dev_features) % 16) {
        set_error("sel_mlp_train_step: bad arguments (batch rows a positive multiple of 8)");
        return SEL_ERR_INVALID_ARG;
    }
    MLP_TRY(check_cfg(cfg));
    cudaStream_t st = ctx_stream(ctx);
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->loss, 0, 4, st), "sel_mlp_train_step"));
    MLP_TRY(backward(m, static_cast<const __nv_bfloat16*>(dev_features), dev_y, n, st));
    if (cfg->apply_update) MLP_TRY(adam(m, cfg, true, st));
    float l = 0.f;
    unsigned int err = 0;
    MLP_TRY(cuda_ok(cudaMemcpyAsync(&l, m->loss, 4, cudaMemcpyDeviceToHost, st), "sel_mlp_train_step"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(&err, m->err, 4, cudaMemcpyDeviceToHost, st), "sel_mlp_train_step"));
    MLP_TRY(cuda_ok(cudaStreamSynchronize(st), "sel_mlp_train_step"));
    if (err) {
        set_error("sel_mlp_train_step: a bounded tensor-core wait gave up");
        return SEL_ERR_TIMEOUT;
    }
    if (loss_out) *loss_out = l / (float)n;
    return SEL_OK;
}

extern "C" sel_status sel_mlp_train(sel_ctx* ctx, sel_mlp* m, const sel_pred* const* preds,
                                    const uint64_t* exact_counts, int64_t n, const sel_train_cfg* cfg,
                                    float* final_loss) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !m || !preds || !exact_counts || n <= 0 || n > (1ll << 30)) {
        set_error("sel_mlp_train: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    MLP_TRY(check_cfg(cfg));
    if (cfg->batch <= 0 || cfg->batch % 8 || cfg->epochs <= 0) {
        set_error("sel_mlp_train: batch must be a positive multiple of 8 and epochs positive");
        return SEL_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx_stream(ctx);
    DeviceVec feat, y, idx, xb, yb;
    MLP_TRY(cuda_ok(dev_alloc(&feat.p, (size_t)n * kFeat * 2), "sel_mlp_train"));
    std::vector<uint8_t> ok_all;
    ok_all.reserve((size_t)n);
    for (int64_t b0 = 0; b0 < n; b0 += 65536) {
        const int32_t nb = (int32_t)std::min<int64_t>(65536, n - b0);
        std::vector<uint8_t> ok;
        MLP_TRY(featurize(m, st, preds + b0, nb, static_cast<__nv_bfloat16*>(feat.p) + (size_t)b0 * kFeat, &ok, nullptr));
        ok_all.insert(ok_all.end(), ok.begin(), ok.end());
    }
    std::vector<int32_t> usable;
    std::vector<float> yh((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        yh[(size_t)i] = (float)std::log1p((double)exact_counts[i]);
        if (ok_all[(size_t)i]) usable.push_back((int32_t)i);
    }
    if ((int64_t)usable.size() < cfg->batch) {
        set_error("sel_mlp_train: %zu featurizable predicates, fewer than one batch", usable.size());
        return SEL_ERR_INVALID_ARG;
    }
    MLP_TRY(cuda_ok(dev_alloc(&y.p, (size_t)n * 4), "sel_mlp_train"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(y.p, yh.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st), "sel_mlp_train"));
    MLP_TRY(cuda_ok(dev_alloc(&idx.p, usable.size() * 4), "sel_mlp_train"));
    MLP_TRY(cuda_ok(dev_alloc(&xb.p, (size_t)cfg->batch * kFeat * 2), "sel_mlp_train"));
    MLP_TRY(cuda_ok(dev_alloc(&yb.p, (size_t)cfg->batch * 4), "sel_mlp_train"));
    if (m->step == 0) {
        // start the head at the targets' mean and log-variance (an untrained model)
        double s1 = 0.0, s2 = 0.0;
        for (int32_t i : usable) {
            s1 += yh[(size_t)i];
            s2 += (double)yh[(size_t)i] * yh[(size_t)i];
        }
        const double mean = s1 / (double)usable.size();
        const double var = std::max(s2 / (double)usable.size() - mean * mean, 1e-4);
        const float b4[2] = {(float)mean, (float)std::log(var)};
        MLP_TRY(cuda_ok(cudaMemcpyAsync(m->p + oB4, b4, 8, cudaMemcpyHostToDevice, st), "sel_mlp_train"));
        MLP_TRY(cuda_ok(cudaStreamSynchronize(st), "sel_mlp_train"));
    }
    std::mt19937_64 rng(cfg->seed);
    const int64_t steps = (int64_t)usable.size() / cfg->batch;
    double last = 0.0;
    for (int e = 0; e < cfg->epochs; ++e) {
        std::shuffle(usable.begin(), usable.end(), rng);
        MLP_TRY(cuda_ok(cudaMemcpyAsync(idx.p, usable.data(), usable.size() * 4, cudaMemcpyHostToDevice, st),
                        "sel_mlp_train"));
        double sum = 0.0;
        for (int64_t s = 0; s < steps; ++s) {
            ++thread_launches();
            gather_kernel<<<cfg->batch, 32, 0, st>>>(static_cast<const __nv_bfloat16*>(feat.p),
                                                    static_cast<const float*>(y.p),
                                                    static_cast<const int32_t*>(idx.p) + s * cfg->batch, cfg->batch,
                                                    static_cast<__nv_bfloat16*>(xb.p), static_cast<float*>(yb.p));
            MLP_TRY(cuda_ok(cudaGetLastError(), "gather launch"));
            float l = 0.f;
            sel_train_cfg c = *cfg;
            c.apply_update = 1;
            MLP_TRY(sel_mlp_train_step(ctx, m, xb.p, static_cast<const float*>(yb.p), cfg->batch, &c, &l));
            sum += l;
        }
        last = sum / (double)steps;
        MLP_TRY(cuda_ok(cudaStreamSynchronize(st), "sel_mlp_train"));   // idx is rewritten next epoch
    }
    if (final_loss) *final_loss = (float)last;
    return SEL_OK;
}

extern "C" sel_status sel_mlp_estimate(sel_ctx* ctx, sel_mlp* m, const sel_pred* const* preds,
                                       const sel_table* table, int32_t n, float tau, double* est, float* sigma,
                                       uint8_t* used_exact) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !m || !preds || !table || n <= 0 || !est) {
        set_error("sel_mlp_estimate: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx_stream(ctx);
    DeviceVec feat;
    MLP_TRY(cuda_ok(dev_alloc(&feat.p, (size_t)n * kFeat * 2), "sel_mlp_estimate"));
    std::vector<uint8_t> ok;
    MLP_TRY(featurize(m, st, preds, n, static_cast<__nv_bfloat16*>(feat.p), &ok, nullptr));
    MLP_TRY(forward(m, static_cast<const __nv_bfloat16*>(feat.p), n, false, st));
    std::vector<float> out((size_t)n * 2);
    MLP_TRY(cuda_ok(cudaMemcpyAsync(out.data(), m->out, (size_t)n * 8, cudaMemcpyDeviceToHost, st), "sel_mlp_estimate"));
    MLP_TRY(cuda_ok(cudaStreamSynchronize(st), "sel_mlp_estimate"));
    std::vector<const sel_pred*> exact_preds;
    std::vector<const sel_table*> exact_tabs;
    std::vector<int32_t> exact_idx;
    for (int32_t i = 0; i < n; ++i) {
        const float lv = std::min(std::max(out[2 * (size_t)i + 1], kLvMin), kLvMax);
        const float sg = std::exp(0.5f * lv);
        if (sigma) sigma[i] = ok[(size_t)i] ? sg : INFINITY;
        const bool ex = !ok[(size_t)i] || !(sg <= tau);
        if (used_exact) used_exact[i] = ex ? 1 : 0;
        if (ex) {
            exact_preds.push_back(preds[i]);
            exact_tabs.push_back(table);
            exact_idx.push_back(i);
        } else {
            est[i] = std::max(0.0, std::expm1((double)out[2 * (size_t)i]));
        }
    }
    if (!exact_preds.empty()) {
        // the exact fallback: batched scans over the uncertain probes
        std::vector<uint64_t> counts(exact_preds.size());
        for (size_t b0 = 0; b0 < exact_preds.size(); b0 += 2048) {
            const int32_t nb = (int32_t)std::min<size_t>(2048, exact_preds.size() - b0);
            sel_batch_plan* plan = nullptr;
            MLP_TRY(sel_batch_plan_create(ctx, exact_preds.data() + b0, exact_tabs.data() + b0, nb, 0, &plan));
            sel_status s = sel_batch_plan_run(plan, nullptr, counts.data() + b0);
            sel_batch_plan_free(plan);
            if (s != SEL_OK) return s;
        }
        for (size_t j = 0; j < exact_idx.size(); ++j) est[exact_idx[j]] = (double)counts[j];
    }
    return SEL_OK;
}

// a9 calibration: the largest tau among the held-out sigmas whose accepted
// estimates (sigma <= tau) keep the `quantile` percentile of the q-error at or
// below max_q.  The accepted set grows in sigma order; a Fenwick tree over the
// q-error ranks gives the two order statistics of each percentile in O(log n).
extern "C" sel_status sel_mlp_choose_tau(const float* sigma, const double* est, const uint64_t* exact, int64_t n,
                                         double max_q, double quantile, float* tau_out, double* answered_out) {
    if (!sigma || !est || !exact || n < 0 || !tau_out || !(quantile >= 0.0 && quantile <= 100.0)) {
        set_error("sel_mlp_choose_tau: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    std::vector<double> q((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double e = std::max(est[i], 1.0), t = std::max((double)exact[i], 1.0);
        q[(size_t)i] = std::max(e / t, t / e);
    }
    std::vector<int64_t> by_q((size_t)n), by_sigma;
    for (int64_t i = 0; i < n; ++i) by_q[(size_t)i] = i;
    std::sort(by_q.begin(), by_q.end(), [&](int64_t a, int64_t b) { return q[(size_t)a] < q[(size_t)b]; });
    std::vector<int64_t> rank((size_t)n);
    for (int64_t r = 0; r < n; ++r) rank[(size_t)by_q[(size_t)r]] = r;
    for (int64_t i = 0; i < n; ++i)
        if (std::isfinite(sigma[i])) by_sigma.push_back(i);
    std::sort(by_sigma.begin(), by_sigma.end(), [&](int64_t a, int64_t b) { return sigma[a] < sigma[b]; });
    std::vector<int64_t> fen((size_t)n + 1, 0);
    auto add = [&](int64_t r) {
        for (int64_t x = r + 1; x <= n; x += x & -x) ++fen[(size_t)x];
    };
    int64_t top = 1;
    while (top * 2 <= n) top *= 2;
    auto kth = [&](int64_t k) {   // the k-th smallest inserted q-error (0-based)
        int64_t pos = 0;
        for (int64_t step = top; step > 0; step >>= 1)
            if (pos + step <= n && fen[(size_t)(pos + step)] <= k) {
                pos += step;
                k -= fen[(size_t)pos];
            }
        return q[(size_t)by_q[(size_t)pos]];
    };
    float best = 0.f;
    int64_t best_cnt = 0, cnt = 0;
    for (size_t j = 0; j < by_sigma.size();) {
        const float t = sigma[by_sigma[j]];
        for (; j < by_sigma.size() && sigma[by_sigma[j]] == t; ++j, ++cnt) add(rank[(size_t)by_sigma[j]]);
        const double h = (double)(cnt - 1) * (quantile / 100.0);
        const int64_t lo = (int64_t)std::floor(h);
        const double a = kth(lo);
        const double p = lo + 1 >= cnt ? kth(cnt - 1) : a + (h - (double)lo) * (kth(lo + 1) - a);
        if (p <= max_q) {
            best = t;
            best_cnt = cnt;
        }
    }
    *tau_out = best;
    if (answered_out) *answered_out = n > 0 ? (double)best_cnt / (double)n : 0.0;
    return SEL_OK;
}

extern "C" int64_t sel_mlp_param_count(void) { return kParams; }

extern "C" sel_status sel_mlp_get_params(const sel_mlp* m, float* host, int64_t n_floats) {
    if (!m || !host || n_floats != kParams) {
        set_error("sel_mlp_get_params: need %lld floats", (long long)kParams);
        return SEL_ERR_INVALID_ARG;
    }
    return cuda_ok(cudaMemcpy(host, m->p, kParams * 4, cudaMemcpyDeviceToHost), "sel_mlp_get_params");
}

extern "C" sel_status sel_mlp_get_grads(const sel_mlp* m, float* host, int64_t n_floats) {
    if (!m || !host || n_floats != kParams) {
        set_error("sel_mlp_get_grads: need %lld floats", (long long)kParams);
        return SEL_ERR_INVALID_ARG;
    }
    return cuda_ok(cudaMemcpy(host, m->g, kParams * 4, cudaMemcpyDeviceToHost), "sel_mlp_get_grads");
}

extern "C" sel_status sel_mlp_set_params(sel_ctx* ctx, sel_mlp* m, const float* host, int64_t n_floats) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !m || !host || n_floats != kParams) {
        set_error("sel_mlp_set_params: need %lld floats", (long long)kParams);
        return SEL_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx_stream(ctx);
    MLP_TRY(cuda_ok(cudaMemcpyAsync(m->p, host, kParams * 4, cudaMemcpyHostToDevice, st), "sel_mlp_set_params"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->g, 0, kParams * 4, st), "sel_mlp_set_params"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->mm, 0, kParams * 4, st), "sel_mlp_set_params"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->vv, 0, kParams * 4, st), "sel_mlp_set_params"));
    m->step = 0;
    MLP_TRY(adam(m, nullptr, false, st));
    return cuda_ok(cudaStreamSynchronize(st), "sel_mlp_set_params");
}

static const char kMagic[8] = {'S', 'E', 'L', 'M', 'L', 'P', '1', 0};

extern "C" sel_status sel_mlp_save(const sel_mlp* m, const char* path) {
    if (!m || !path) {
        set_error("sel_mlp_save: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    std::vector<float> p((size_t)kParams), mm((size_t)kParams), vv((size_t)kParams);
    std::vector<uint64_t> cdf((size_t)m->n_cols * m->m);
    MLP_TRY(cuda_ok(cudaMemcpy(p.data(), m->p, kParams * 4, cudaMemcpyDeviceToHost), "sel_mlp_save"));
    MLP_TRY(cuda_ok(cudaMemcpy(mm.data(), m->mm, kParams * 4, cudaMemcpyDeviceToHost), "sel_mlp_save"));
    MLP_TRY(cuda_ok(cudaMemcpy(vv.data(), m->vv, kParams * 4, cudaMemcpyDeviceToHost), "sel_mlp_save"));
    MLP_TRY(cuda_ok(cudaMemcpy(cdf.data(), m->cdf, cdf.size() * 8, cudaMemcpyDeviceToHost), "sel_mlp_save"));
    FILE* f = std::fopen(path, "wb");
    if (!f) {
        set_error("sel_mlp_save: cannot open %s", path);
        return SEL_ERR_INVALID_ARG;
    }
    const int64_t hdr[6] = {kParams, m->n_cols, m->m, (int64_t)m->seed, m->step, (int64_t)m->types.size()};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, 8, 6, f) == 6 &&
              std::fwrite(m->types.data(), 4, m->types.size(), f) == m->types.size() &&
              std::fwrite(p.data(), 4, p.size(), f) == p.size() && std::fwrite(mm.data(), 4, mm.size(), f) == mm.size() &&
              std::fwrite(vv.data(), 4, vv.size(), f) == vv.size() &&
              std::fwrite(cdf.data(), 8, cdf.size(), f) == cdf.size();
    ok &= std::fclose(f) == 0;
    if (!ok) {
        set_error("sel_mlp_save: write to %s failed", path);
        return SEL_ERR_INVALID_ARG;
    }
    return SEL_OK;
}

extern "C" sel_status sel_mlp_load(sel_ctx* ctx, const char* path, sel_mlp** out) {
    LaunchTally tally(ctx);   // this call's kernel launches count on ctx
    if (!ctx || !path || !out) {
        set_error("sel_mlp_load: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) {
        set_error("sel_mlp_load: cannot open %s", path);
        return SEL_ERR_INVALID_ARG;
    }
    char magic[8];
    int64_t hdr[6];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 && std::fread(hdr, 8, 6, f) == 6 &&
              hdr[0] == kParams && hdr[1] > 0 && hdr[1] <= kCols && hdr[2] >= 2 && hdr[2] <= 8192 && hdr[5] > 0 &&
              hdr[5] < 1024;
    std::unique_ptr<sel_mlp> m(new sel_mlp());
    std::vector<float> p, mm, vv;
    std::vector<uint64_t> cdf;
    if (ok) {
        m->n_cols = (int32_t)hdr[1];
        m->m = (int32_t)hdr[2];
        m->seed = (uint64_t)hdr[3];
        m->step = hdr[4];
        m->types.resize((size_t)hdr[5]);
        p.resize((size_t)kParams);
        mm.resize((size_t)kParams);
        vv.resize((size_t)kParams);
        cdf.resize((size_t)m->n_cols * m->m);
        ok = std::fread(m->types.data(), 4, m->types.size(), f) == m->types.size() &&
             std::fread(p.data(), 4, p.size(), f) == p.size() && std::fread(mm.data(), 4, mm.size(), f) == mm.size() &&
             std::fread(vv.data(), 4, vv.size(), f) == vv.size() && std::fread(cdf.data(), 8, cdf.size(), f) == cdf.size();
    }
    std::fclose(f);
    if (!ok) {
        set_error("sel_mlp_load: %s is not a saved estimator", path);
        return SEL_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx_stream(ctx);
    MLP_TRY(alloc_model(m.get()));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(m->p, p.data(), kParams * 4, cudaMemcpyHostToDevice, st), "sel_mlp_load"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(m->mm, mm.data(), kParams * 4, cudaMemcpyHostToDevice, st), "sel_mlp_load"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(m->vv, vv.data(), kParams * 4, cudaMemcpyHostToDevice, st), "sel_mlp_load"));
    MLP_TRY(cuda_ok(cudaMemcpyAsync(m->cdf, cdf.data(), cdf.size() * 8, cudaMemcpyHostToDevice, st), "sel_mlp_load"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->g, 0, kParams * 4, st), "sel_mlp_load"));
    MLP_TRY(cuda_ok(cudaMemsetAsync(m->err, 0, 4, st), "sel_mlp_load"));
    MLP_TRY(adam(m.get(), nullptr, false, st));
    MLP_TRY(cuda_ok(cudaStreamSynchronize(st), "sel_mlp_load"));
    *out = m.release();
    return SEL_OK;
}

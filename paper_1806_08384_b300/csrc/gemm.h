// gemm.h -- launch interface of the tcgen05 BF16 GEMM (gemm.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sel {

enum GemmEpilogue : int {
    EPI_F32 = 0,        // C = acc (split-K: C += acc, C zeroed by the caller)
    EPI_BIAS_RELU = 1,  // y = relu(acc + bias[col]) -> out (bf16, M x N) and outT (bf16, N x M)
    EPI_DRELU = 2,      // y = acc where mask[row][col] > 0 else 0 -> out / outT; colsum[col] += sum over rows
};

struct GemmArgs {
    const __nv_bfloat16* A;   // M x K, row stride lda (elements, multiple of 8)
    const __nv_bfloat16* B;   // N x K, row stride ldb
    long long lda, ldb;
    int M, N, K;              // K multiple of 8
    int epi;
    float* C;                 // EPI_F32
    long long ldc;
    const float* bias;        // EPI_BIAS_RELU
    __nv_bfloat16* out;       // optional
    long long ldo;
    __nv_bfloat16* outT;      // optional
    long long ldoT;
    const __nv_bfloat16* mask;  // EPI_DRELU
    long long ldm;
    float* colsum;            // EPI_DRELU, optional
    unsigned int* err;        // set when a bounded wait gave up
};

size_t gemm_smem_bytes();
cudaError_t launch_gemm(const GemmArgs& g, int k_splits, cudaStream_t st);

// The estimator's whole inference pass in one kernel: per 128-row tile,
// h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), h3 = relu(h2 W3^T + b3)
// (BF16 activations, FP32 accumulation in TMEM; the activations never leave
// shared memory) and out = h3 W4^T + b4 on the CUDA cores.
struct MlpFwdArgs {
    const __nv_bfloat16* x;      // n x 144, rows contiguous, 16-byte aligned
    const __nv_bfloat16* w[3];   // W1 256 x 144, W2 and W3 256 x 256 (K contiguous)
    const float* b[3];           // b1, b2, b3: 256 each
    const __nv_bfloat16* w4;     // 2 x 256
    const float* b4;             // 2
    float* out;                  // n x 2: (mu, raw log-variance)
    int n;
    unsigned int* err;           // set when a bounded wait gave up
};
size_t mlp_forward_smem_bytes();
cudaError_t launch_mlp_forward(const MlpFwdArgs& a, cudaStream_t st);

}  // namespace sel

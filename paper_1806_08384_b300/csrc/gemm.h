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

}  // namespace sel

// Tensor-core GEMM C = A . B^T with fused epilogues (internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mls2mc {

enum GemmEpiKind {
    kEpiStoreF32 = 0,      // out_f32 = acc (+ bias[col])
    kEpiBiasGelu = 1,      // pre = acc + bias; act (and act_t, transposed) = bf16(GELU(pre))
    kEpiGeluBackward = 2,  // act (and act_t) = bf16(acc * GELU'(pre_in))
    kEpiExp = 3,           // out_f32 = exp(acc)
};

struct GemmEpi {
    int kind = kEpiStoreF32;
    float* out_f32 = nullptr;
    int ld_out = 0;
    const float* bias = nullptr;
    float* pre = nullptr;           // kEpiBiasGelu output / kEpiGeluBackward reads pre_in with ld_pre
    const float* pre_in = nullptr;
    int ld_pre = 0;
    __nv_bfloat16* act = nullptr;
    int ld_act = 0;
    __nv_bfloat16* act_t = nullptr;
    int ld_act_t = 0;
    int tma_out = 0;                // set by umma_gemm: the FP32 output leaves by TMA stores
    float* ws = nullptr;            // kEpiStoreF32 without bias: workspace for split-K partial tiles
    size_t ws_floats = 0;           //   (splits x M x ld_out floats at most; null: no split)
};

// A: M x K BF16 (row stride lda elements), B: N x K BF16 (row stride ldb); lda, ldb multiples of 8,
// base pointers 16-byte aligned. *err (device int) is set to 1 if a bounded wait timed out.
cudaError_t umma_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const GemmEpi& epi,
                      int* err, cudaStream_t st);

}  // namespace mls2mc

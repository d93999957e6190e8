// Small BF16 tensor-core helpers for the proposal network (mma.sync
// m16n8k16, FP32 accumulation) and the network's fixed shape.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace gk {

// Proposal network: 375 patch features (padded to 384) -> 128 -> 128 -> 4.
constexpr int kIn = 375, kInPad = 384, kH = 128, kOut = 4, kOutPad = 8;
constexpr int kPatch = 5;                 // 5 x 5 x 5 patch (5 x 5 in 2D)

struct MlpWeights {                        // device pointers, bf16 copies used by the GEMMs
    const __nv_bfloat16* W1;               // [kH][kInPad]
    const __nv_bfloat16* W2;               // [kH][kH]
    const __nv_bfloat16* W3;               // [kOutPad][kH] (rows >= kOut are zero)
    const float* b1;                       // [kH]
    const float* b2;                       // [kH]
    const float* b3;                       // [kOutPad]
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragment loads from shared memory, both operands stored with K contiguous:
// A as [m][k] (row stride lda elements), B as [n][k] (row stride ldb).
__device__ __forceinline__ void load_a_frag(uint32_t (&a)[4], const __nv_bfloat16* A, int lda,
                                            int lane)
{
    const int g = lane >> 2, t = lane & 3;
    a[0] = *(const uint32_t*)(A + g * lda + 2 * t);
    a[1] = *(const uint32_t*)(A + (g + 8) * lda + 2 * t);
    a[2] = *(const uint32_t*)(A + g * lda + 2 * t + 8);
    a[3] = *(const uint32_t*)(A + (g + 8) * lda + 2 * t + 8);
}

__device__ __forceinline__ void load_b_frag(uint32_t (&b)[2], const __nv_bfloat16* B, int ldb,
                                            int lane)
{
    const int g = lane >> 2, t = lane & 3;
    b[0] = *(const uint32_t*)(B + g * ldb + 2 * t);
    b[1] = *(const uint32_t*)(B + g * ldb + 2 * t + 8);
}

}  // namespace gk

// The proposal network's fixed shape and the device view of its BF16 weights.
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

}  // namespace gk

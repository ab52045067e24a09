// Device helpers shared by the per-step kernels of the 2D TK-WFP evaluator.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace wfp {

template <typename T>
struct Cplx;
template <>
struct Cplx<double> {
    using type = double2;
};
template <>
struct Cplx<float> {
    using type = float2;
};

// Double-float accumulation (FP32 arithmetic, ~2x24-bit significand): (sh, sl) += (ah + al) * b,
// with the product ah*b made exact by an FMA and the sum by TwoSum.  Explicit round-to-nearest
// intrinsics keep the compiler from contracting the error terms away.
__device__ __forceinline__ void df_acc(float& sh, float& sl, float ah, float al, float b) {
    float p = __fmul_rn(ah, b);
    float e = fmaf(ah, b, -p);
    e = fmaf(al, b, e);
    float s = __fadd_rn(sh, p);
    float bb = __fsub_rn(s, sh);
    float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sl = __fadd_rn(sl, __fadd_rn(t, e));
    sh = s;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
    using type = double2;
};
template <>
struct Vec16<float> {
    using type = float4;
};

}  // namespace wfp

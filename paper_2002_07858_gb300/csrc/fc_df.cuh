// fc_df.cuh -- double-float arithmetic (a value is hi + lo, two binary32
// numbers with |lo| <= ulp(hi)/2) for the binary64-accuracy residual chi2 of
// the mixed path.  GB300 runs binary32 about 60 times faster than binary64,
// and a double-float multiply-add costs about a dozen binary32 operations:
//   - the product of two binary32 numbers is split exactly by one fma
//     (Dekker's TwoProduct with a fused multiply-add);
//   - sums use Knuth's TwoSum (six operations, exact error term);
//   - the lo * lo cross term is dropped (below 2^-48 relative).
// The relative error of a dot product of n terms is about n 2^-47 of the sum
// of the absolute terms, far below what the certified decisions and the
// output tolerances need.  Every function here is a fixed sequence of IEEE
// binary32 operations, so a value is the same bits wherever it is computed.
#pragma once

#include <cuda_runtime.h>

namespace fcdev {

// binary64 -> hi + lo (exact for |x| within the binary32 range up to 2^-48 |x|)
__device__ __forceinline__ float2 df_from(double x) {
    const float h = (float)x;
    const float l = (float)(x - (double)h);
    return make_float2(h, l);
}

__device__ __forceinline__ double df_to(float2 a) { return (double)a.x + (double)a.y; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// renormalise hi + lo (requires |hi| >= |lo| or hi == 0)
__device__ __forceinline__ float2 df_norm(float hi, float lo) {
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

// acc + a * b, a and b double-float
__device__ __forceinline__ float2 df_fma(float2 acc, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float s, err;
    two_sum(acc.x, p, s, err);
    return make_float2(s, __fadd_rn(acc.y, __fadd_rn(err, e)));
}

// a + b, both double-float
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

// a - b for a double-float a and a binary32 b (exact up to the lo rounding)
__device__ __forceinline__ float2 df_sub_f(float2 a, float b) {
    float s, e;
    two_sum(a.x, -b, s, e);
    return df_norm(s, __fadd_rn(e, a.y));
}

}  // namespace fcdev

// Double-float arithmetic on the FP32 pipe (Dekker, Numer. Math. 18, 1971;
// Knuth's two-sum, TAOCP vol. 2): a value is the unevaluated sum hi + lo of two
// floats, about 48 significant bits.  On this GPU an FP64 instruction of a warp
// holds the SM's FP64 pipe for tens of cycles, so the normal-equation kernels
// keep their accurate sums here and use FP64 only for what they store.
// The _rn intrinsics keep the compiler from fusing a product into a following
// sum, which would break the exact error terms.
#pragma once

#include <cuda_runtime.h>

namespace cpdf {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah, al) += (vh + vl)(ph + pl): the leading product exact (two-product by FMA),
// the cross terms in FP32 (relative size 2^-24), lo * lo dropped (2^-48)
__device__ __forceinline__ void fma_acc(float vh, float vl, float ph, float pl, float& ah, float& al) {
    const float m = __fmul_rn(vh, ph);
    float e = __fmaf_rn(vh, ph, -m);
    e = __fmaf_rn(vh, pl, __fmaf_rn(vl, ph, e));
    float s, t;
    two_sum(ah, m, s, t);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(t, e));
}
// (ah, al) += (bh, bl)
__device__ __forceinline__ void add(float& ah, float& al, float bh, float bl) {
    float s, t;
    two_sum(ah, bh, s, t);
    t = __fadd_rn(t, __fadd_rn(al, bl));
    fast_two_sum(s, t, ah, al);
}
// (ah, al) * (bh, bl): exact leading product, cross terms in FP32, renormalised
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
    const float m = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -m);
    e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
    float h, l;
    fast_two_sum(m, e, h, l);
    return make_float2(h, l);
}
// a double as a float pair
__device__ __forceinline__ float2 split(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

}  // namespace cpdf

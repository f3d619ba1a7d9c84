// Double-float arithmetic on the FP32 pipes: a value is an unevaluated sum hi + lo of
// two floats (48 significant bits).  The error-free steps use explicit round-to-nearest
// intrinsics so that the compiler cannot contract them into FMAs, which would break the
// two-sum and two-product identities (Knuth two-sum; Dekker product via FMA).
#pragma once

#include <cuda_runtime.h>

namespace wfq {

// hi = fp32(v), lo = fp32(v - hi)
__device__ __forceinline__ void df_split(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// (sh, sl) += (ah + al) (bh + bl): the exact product ah*bh (its rounding error recovered
// with an FMA) plus the cross terms ah*bl + al*bh, added to the running sum by two-sum.
// The dropped al*bl term and the cross-term roundings are ~2^-48 relative.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &sh, float &sl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);           // exact rounding error of p
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = __fadd_rn(sh, p);
    const float v = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));   // sh + p - s exactly
    sh = s;
    sl += t + e;
}

// The same multiply-add on two independent lanes at once with the packed FP32x2
// instructions (one instruction per pair of FP32 operations: half the issue slots of
// df_mac, the same arithmetic on each lane).
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void df_mac2(float2 ah, float2 al, float2 bh, float2 bl, float2 &sh, float2 &sl) {
    const float2 p = __fmul2_rn(ah, bh);
    float2 e = __ffma2_rn(ah, bh, f2neg(p));          // exact rounding error of p
    e = __ffma2_rn(ah, bl, e);
    e = __ffma2_rn(al, bh, e);
    const float2 s = __fadd2_rn(sh, p);
    const float2 v = __fadd2_rn(s, f2neg(sh));
    const float2 t = __fadd2_rn(__fadd2_rn(sh, f2neg(__fadd2_rn(s, f2neg(v)))), __fadd2_rn(p, f2neg(v)));
    sh = s;
    sl = __fadd2_rn(sl, __fadd2_rn(t, e));
}

// (sh, sl) += (bh, bl)
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl) {
    const float s = __fadd_rn(sh, bh);
    const float v = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(bh, v));
    sh = s;
    sl = sl + bl + t;
}

}  // namespace wfq

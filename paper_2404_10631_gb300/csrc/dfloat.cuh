// Double-float arithmetic on the FP32 pipe, shared by the eigensolver's
// refinement and the covariance reduction: GB300's FP64 pipe runs under two
// multiply-adds per clock per SM, so the FP64-level work of both is done in
// pairs of FP32 numbers.
#pragma once

#include <cuda_runtime.h>

namespace hsc {
namespace {

// ---- double-float arithmetic: a value is an unevaluated sum h + l of two
// FP32 numbers with |l| <= ulp(h)/2 (Dekker 1971; Knuth's TwoSum). The
// intrinsics keep the compiler from contracting or reassociating.
struct dfl {
    float h, l;
};

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly when |a| >= |b| (Dekker's Fast2Sum)
__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    float s, e;
    two_sum(x.h, y.h, s, e);
    e = __fadd_rn(e, __fadd_rn(x.l, y.l));
    return fast_two_sum(s, e);
}

// x * y: the product of the heads split exactly by an FMA (two-product),
// plus the cross terms
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return fast_two_sum(p, e);
}

// x / y by one correction of the FP32 quotient (the long-division step of
// double-length arithmetic): q1 = x/y, q2 = (x - q1 y)/y
__device__ __forceinline__ dfl df_div(dfl x, dfl y)
{
    const float q1 = __fdiv_rn(x.h, y.h);
    const dfl p = df_mul({q1, 0.f}, y);
    const dfl r = df_add(x, {-p.h, -p.l});
    const float q2 = __fdiv_rn(r.h, y.h);
    return fast_two_sum(q1, q2);
}

}  // namespace
}  // namespace hsc

// Double-single arithmetic on the FP32 pipe: a value is the unevaluated sum
// hi + lo of two floats (~46 significant bits).  Building blocks (Dekker 1971;
// Knuth TAOCP vol. 2, 4.2.2): TwoSum, Fast2Sum and the FMA form of the exact
// product, written with round-to-nearest intrinsics so that no operation is
// contracted or fused.  Used by the double-single force mode and the
// double-single potential of the energy diagnostic.
#pragma once

#include "ptx.cuh"

namespace nb {
namespace dsa {

struct ds {
    float h, l;
};

__device__ __forceinline__ ds two_sum(const float a, const float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ ds fast_two_sum(const float a, const float b)  // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ds ds_add(const ds x, const ds y)
{
    const ds s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

__device__ __forceinline__ ds ds_neg(const ds x) { return {-x.h, -x.l}; }

__device__ __forceinline__ ds ds_mul(const ds x, const ds y)
{
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ds ds_mul_f(const ds x, const float f)
{
    const float p = __fmul_rn(x.h, f);
    float e = __fmaf_rn(x.h, f, -p);
    e = __fmaf_rn(x.l, f, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ds ds_rsqrt(const ds r2)
{
    const float y0 = rsqrt_mufu(r2.h);
    const float p = __fmul_rn(y0, y0);
    const ds y0sq = {p, __fmaf_rn(y0, y0, -p)};      // exact
    const ds t = ds_mul(r2, y0sq);                    // 1 - rho
    const ds rho = ds_add({1.0f, 0.0f}, ds_neg(t));  // small: its hi carries the needed bits
    const float c = y0 * (rho.h * fmaf(0.375f, rho.h, 0.5f));
    return fast_two_sum(y0, c);
}

}  // namespace dsa
}  // namespace nb

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

// One pair term of Appendix A in double-single arithmetic, j given by its
// (hi, lo) position and mass a, b = (x, y, z, m) and velocity u, w4 = (vx, vy, vz, .),
// i by xi, vi: dx = x_j - x_i, dv = v_j - v_i, r2 = eps2 + dx.dx, rinv = r2^-1/2
// (ds_rsqrt), then a += m r^-3 dx, k += m r^-3 (dv - 3 (dx.dv) r^-2 dx),
// phi -= m r^-1 into sum[0..2], sum[3..5], sum[6].
__device__ __forceinline__ void ds_pair_term(const float4 a, const float4 b, const float4 u, const float4 w4,
                                             const ds (&xi)[3], const ds (&vi)[3], const ds eps2, ds (&sum)[7])
{
    const ds dx[3] = {ds_add({a.x, b.x}, ds_neg(xi[0])), ds_add({a.y, b.y}, ds_neg(xi[1])),
                      ds_add({a.z, b.z}, ds_neg(xi[2]))};
    const ds dv[3] = {ds_add({u.x, w4.x}, ds_neg(vi[0])), ds_add({u.y, w4.y}, ds_neg(vi[1])),
                      ds_add({u.z, w4.z}, ds_neg(vi[2]))};
    const ds r2 = ds_add(ds_add(ds_add(eps2, ds_mul(dx[0], dx[0])), ds_mul(dx[1], dx[1])), ds_mul(dx[2], dx[2]));
    const ds rinv = ds_rsqrt(r2);
    const ds rinv2 = ds_mul(rinv, rinv);
    const ds mr = ds_mul({a.w, b.w}, rinv);
    const ds mr3 = ds_mul(mr, rinv2);
    const ds xv = ds_add(ds_add(ds_mul(dx[0], dv[0]), ds_mul(dx[1], dv[1])), ds_mul(dx[2], dv[2]));
    const ds w = ds_mul_f(ds_mul(xv, rinv2), 3.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        sum[c] = ds_add(sum[c], ds_mul(mr3, dx[c]));
        sum[3 + c] = ds_add(sum[3 + c], ds_mul(mr3, ds_add(dv[c], ds_neg(ds_mul(w, dx[c])))));
    }
    sum[6] = ds_add(sum[6], ds_neg(mr));
}

}  // namespace dsa
}  // namespace nb

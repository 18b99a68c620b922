// Device-side steps shared by the single-system and the ensemble kernels:
// the predictor of one component, the corrector of one particle with the
// Aarseth time step and the power-of-two level rule (Portegies Zwart,
// Belleman & Geldof 2007, Sect. 2), and block-wide reductions.
#pragma once

#include "nbody_internal.cuh"

namespace nb {

// Step factors of the predictor: dt/2 (exact) and dt/3.
struct PredDt {
    double dt, half, third;
};
__device__ __forceinline__ PredDt pred_dt(const double dt) { return {dt, 0.5 * dt, __dmul_rn(dt, 1.0 / 3.0)}; }

// Predictor of Sect. 2 for one component, in Horner form with explicit
// roundings so that the predictor and the corrector kernels give the same
// bits:  x_p = x + dt (v + dt/2 (a + dt/3 k)),  v_p = v + dt (a + dt/2 k),
// i.e. x + v dt + a dt^2/2 + k dt^3/6 and v + a dt + k dt^2/2 in five fused
// multiply-adds (GB300's FP64 pipe is ~1/75 of its FP32 pipe).
__device__ __forceinline__ void predict_dim(double x, double v, double a, double k, const PredDt &d,
                                            double &xp, double &vp)
{
    xp = __fma_rn(d.dt, __fma_rn(d.half, __fma_rn(d.third, k, a), v), x);
    vp = __fma_rn(d.dt, __fma_rn(d.half, k, a), v);
}

// Round-to-nearest-even double -> float, and exact float -> double, on the
// integer pipe: GB300 converts at the FP64 rate (~1.8 per clock per SM, the
// predictor's bound).  IEEE 754 binary64 -> binary32: the 52-bit fraction keeps
// its top 23 bits, rounded by the 29 dropped ones (ties to even); a carry out
// of the fraction moves into the exponent, which the addition below does.
// Results outside the normal float range (zero, subnormal, overflow, Inf, NaN)
// take the hardware conversion; every value the predictor writes is normal or
// zero.
__device__ __forceinline__ float d2f_rn(const double d)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
    const int ef = static_cast<int>((b >> 52) & 0x7ffull) - 1023 + 127;
    if (ef < 1 || ef > 254) return __double2float_rn(d);
    const unsigned long long frac = b & ((1ull << 52) - 1);
    unsigned int keep = static_cast<unsigned int>(frac >> 29);
    const unsigned int rest = static_cast<unsigned int>(frac & ((1u << 29) - 1));
    keep += (rest > (1u << 28)) | ((rest == (1u << 28)) & (keep & 1u));
    const unsigned int bits = (static_cast<unsigned int>(b >> 63) << 31) + ((static_cast<unsigned int>(ef) << 23) + keep);
    return __uint_as_float(bits);
}

__device__ __forceinline__ double f2d(const float f)
{
    const unsigned int b = __float_as_uint(f);
    const unsigned int ef = (b >> 23) & 0xffu;
    if (ef == 0u || ef == 255u) return static_cast<double>(f);
    const unsigned long long bits = (static_cast<unsigned long long>(b >> 31) << 63) |
                                    (static_cast<unsigned long long>(ef - 127 + 1023) << 52) |
                                    (static_cast<unsigned long long>(b & 0x7fffffu) << 29);
    return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ double norm3(const double *u)
{
    return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// Level L of the largest power of two 2^-L <= dt, clamped to [lmin, lmax];
// returns -1 for NaN.  *clamped is set when dt < 2^-lmax (incl. dt <= 0).
__device__ __forceinline__ int level_of(double dt, int lmin, int lmax, bool *clamped)
{
    *clamped = false;
    if (isnan(dt)) return -1;
    if (!(dt > 0.0)) {
        *clamped = true;
        return lmax;
    }
    if (isinf(dt)) return lmin;
    int e;
    frexp(dt, &e);  // dt = f 2^e with 1/2 <= f < 1, so 2^(e-1) <= dt < 2^e
    int L = 1 - e;
    if (L < lmin) L = lmin;
    if (L > lmax) {
        L = lmax;
        *clamped = true;
    }
    return L;
}

// State loads: through L2 only (CG, for state that another CTA of the same
// launch may have written since this SM last read it) or plain.
template <bool CG>
__device__ __forceinline__ double ld_state(const double *p)
{
    if constexpr (CG) return __ldcg(p);
    return *p;
}
template <bool CG>
__device__ __forceinline__ int64_t ld_state(const int64_t *p)
{
    if constexpr (CG) return static_cast<int64_t>(__ldcg(reinterpret_cast<const long long *>(p)));
    return *p;
}
template <bool CG>
__device__ __forceinline__ int8_t ld_state(const int8_t *p)
{
    if constexpr (CG) return static_cast<int8_t>(__ldcg(reinterpret_cast<const signed char *>(p)));
    return *p;
}

// Step quantities of the corrector of Sect. 2 for a step of `steps` ticks of
// 2^-lmax: dt, 1/dt, 1/dt^2, dt^3, dt^4 and the predictor's factors.
struct CorrDt {
    double dt, idt, idt2, dt3, dt4;
    PredDt pd;
};
__device__ __forceinline__ CorrDt corr_dt(const int64_t steps, const double tick, const int lmax)
{
    CorrDt d;
    d.dt = static_cast<double>(steps) * tick;
    // 1/dt: when the step is 2^k ticks of 2^-lmax (every particle of a block) it
    // is 2^(lmax - k), built from its exponent bits; otherwise an IEEE division.
    // Both give the same bits.
    d.idt = (steps > 0 && (steps & (steps - 1)) == 0)
                ? __longlong_as_double(static_cast<long long>(1023 + lmax - (__ffsll(steps) - 1)) << 52)
                : 1.0 / d.dt;
    d.idt2 = d.idt * d.idt;
    d.dt3 = d.dt * d.dt * d.dt;
    d.dt4 = d.dt3 * d.dt;
    d.pd = pred_dt(d.dt);
    return d;
}

// One component of the corrector: from x, v, a, k at the start of the step and
// the force ap, kp at the predicted state, the corrected xn, vn and a^(2), a^(3)
// at the end of the step.
__device__ __forceinline__ void corr_dim(const double x, const double v, const double a, const double k,
                                         const double ap, const double kp, const CorrDt &d, double &xn,
                                         double &vn, double &a2e, double &a3)
{
    double xp, vp;
    predict_dim(x, v, a, k, d.pd, xp, vp);
    const double da = a - ap;  // Delta a = a - a_p
    const double a2 = -6.0 * da * d.idt2 - (4.0 * k + 2.0 * kp) * d.idt;
    a3 = 12.0 * da * d.idt2 * d.idt + 6.0 * (k + kp) * d.idt2;
    // the Taylor coefficients 1/24, 1/120, 1/6 as products (an FP64 division
    // is a long dependent sequence on this part's narrow FP64 pipe)
    xn = xp + d.dt4 * (a2 * (1.0 / 24.0) + a3 * d.dt * (1.0 / 120.0));
    vn = vp + d.dt3 * (a2 * (1.0 / 6.0) + a3 * d.dt * (1.0 / 24.0));
    a2e = a2 + a3 * d.dt;  // a^(2) at the end of the step
}

// Eq. (timestep) from |a|, |k|, |a^(2)|, |a^(3)| at the end of the step, then the
// level rule: shrink at once, grow one level when the new time allows.  Raises
// the non-finite and dt_min flags; returns the new level.
__device__ __forceinline__ int corr_level(const double an, const double kn, const double a2n, const double a3n,
                                          const double eta, const int lmin, const int lmax, const int l_old,
                                          const int64_t t_new, const bool finite, DevStatus *st)
{
    const double num = an * a2n + kn * kn;
    const double den = kn * a3n + a2n * a2n;
    const double dtc = den == 0.0 ? static_cast<double>(INFINITY) : sqrt(eta * num / den);
    bool clamped = false;
    const int lc = level_of(dtc, lmin, lmax, &clamped);
    int l_new;
    if (!finite || lc < 0) {
        l_new = lmax;
        atomicOr(&st->flags, kFlagNonfinite);
        atomicAdd(&st->nonfinite, 1ull);
    } else if (lc >= l_old) {
        l_new = lc;  // shrink at once (or keep)
    } else {
        // grow one level, only if the new time is a multiple of twice the old step
        const int64_t two_old = int64_t(2) << (lmax - l_old);
        l_new = (l_old - 1 >= lmin && t_new % two_old == 0) ? l_old - 1 : l_old;
    }
    if (clamped) {
        atomicOr(&st->flags, kFlagDtMin);
        atomicAdd(&st->below_min, 1ull);
    }
    return l_new;
}

// Corrector of Sect. 2 for particle i (its forces at the predicted state in
// ap_in[3], kp_in[3]), then Eq. (timestep) and the new level; the step ends
// at tick t_new.  Updates x, v, a, k, t, level of i and returns the new level.
template <bool CG = false>
__device__ __forceinline__ int correct_row(const State &S, const int64_t i, const double *ap_in,
                                            const double *kp_in, const int64_t t_new, const double tick,
                                            const double eta, const int lmin, const int lmax, DevStatus *st)
{
    const CorrDt d = corr_dt(t_new - ld_state<CG>(S.t + i), tick, lmax);
    double ap[3], kp[3], a2e[3], a3[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ap[c] = ap_in[c];
        kp[c] = kp_in[c];
        double xn, vn;
        corr_dim(ld_state<CG>(S.x[c] + i), ld_state<CG>(S.v[c] + i), ld_state<CG>(S.a[c] + i),
                 ld_state<CG>(S.k[c] + i), ap[c], kp[c], d, xn, vn, a2e[c], a3[c]);
        finite = finite && isfinite(xn) && isfinite(vn) && isfinite(ap[c]) && isfinite(kp[c]);
        S.x[c][i] = xn;
        S.v[c][i] = vn;
        S.a[c][i] = ap[c];
        S.k[c][i] = kp[c];
    }
    // Eq. (timestep) with end-of-step quantities.
    const int l_new = corr_level(norm3(ap), norm3(kp), norm3(a2e), norm3(a3), eta, lmin, lmax,
                                 ld_state<CG>(S.level + i), t_new, finite, st);
    S.t[i] = t_new;
    S.level[i] = static_cast<int8_t>(l_new);
    return l_new;
}

// Block-wide reduction; `id` is the identity of `op` (pads missing warps).
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T *sh, T id)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = static_cast<int>(threadIdx.x) < nw ? sh[threadIdx.x] : id;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

struct MinOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; }
};
struct MaxOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a > b ? a : b; }
};
struct SumOp {
    __device__ long long operator()(long long a, long long b) const { return a + b; }
};

}  // namespace nb

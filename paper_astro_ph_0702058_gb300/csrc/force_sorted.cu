// Sorted-summation force (an ablation of the accumulation order; the paper's
// Sect. 6 proposes adding the pair forces by size, smallest first, to improve
// single-precision accuracy).  One CTA per active row: for each of the 7
// components, every thread forms FP32 pair terms of its j into shared memory,
// the CTA sorts them by magnitude (bitonic network), and one thread adds them
// in that order in FP32.
//
// The pair terms are those of the plain mode (FP32 positions and velocities)
// formed with round-to-nearest intrinsics in a fixed order and the correctly
// rounded reciprocal square root, so a CPU can form, sort and add the same
// terms and obtain the same bits:
//   dx = xj - xi;  dv = vj - vi
//   r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));  rinv = rsqrt_rn(r2)
//   xv = fma(dz, dvz, fma(dy, dvy, dx * dvx))
//   mr = m * rinv;  mr3 = mr * (rinv * rinv);  w = 3 * (xv * (rinv * rinv))
//   terms: mr3 * dx_c,  mr3 * fma(-w, dx_c, dv_c),  -mr
// Sort key: the magnitude bits, then the raw bits (a total order, so equal
// magnitudes of opposite sign always come out in the same order).  Empty
// slots (j = i, j >= n, the power-of-two fill) hold +0 and sort first.
#include "nbody_internal.cuh"

namespace nb {

namespace {

constexpr int kSortThreads = 512;

__device__ __forceinline__ float sorted_term(const int c, const float4 pj, const float4 vj, const float4 xi,
                                             const float4 vi, const float eps2)
{
    const float dx = __fsub_rn(pj.x, xi.x);
    const float dy = __fsub_rn(pj.y, xi.y);
    const float dz = __fsub_rn(pj.z, xi.z);
    const float dvx = __fsub_rn(vj.x, vi.x);
    const float dvy = __fsub_rn(vj.y, vi.y);
    const float dvz = __fsub_rn(vj.z, vi.z);
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, eps2)));
    const float rinv = __frsqrt_rn(r2);
    const float rinv2 = __fmul_rn(rinv, rinv);
    const float mr = __fmul_rn(pj.w, rinv);
    if (c == 6) return -mr;
    const float mr3 = __fmul_rn(mr, rinv2);
    const float d = c % 3 == 0 ? dx : c % 3 == 1 ? dy : dz;
    if (c < 3) return __fmul_rn(mr3, d);
    const float xv = __fmaf_rn(dz, dvz, __fmaf_rn(dy, dvy, __fmul_rn(dx, dvx)));
    const float w = __fmul_rn(3.0f, __fmul_rn(xv, rinv2));
    const float dvc = c == 3 ? dvx : c == 4 ? dvy : dvz;
    return __fmul_rn(mr3, __fmaf_rn(-w, d, dvc));
}

__device__ __forceinline__ bool key_greater(const uint32_t a, const uint32_t b)
{
    const uint32_t ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;
    return ma != mb ? ma > mb : a > b;
}

__global__ void __launch_bounds__(kSortThreads) force_sorted_kernel(const float4 *__restrict__ posm,
                                                                    const float4 *__restrict__ vel,
                                                                    const int32_t *__restrict__ active, int n,
                                                                    int npow2, float eps2, double *__restrict__ acc,
                                                                    double *__restrict__ jerk,
                                                                    double *__restrict__ pot, DevStatus *st)
{
    extern __shared__ uint32_t sk[];
    const int q = blockIdx.x;
    const int tid = threadIdx.x;
    const int i = active[q];
    if (i < 0 || i >= n) {
        if (tid == 0) {
            atomicOr(&st->flags, kFlagBadIndex);
            st->bad_index = q;
        }
        return;
    }
    const float4 xi = posm[i], vi = vel[i];
    float out[7];
    for (int c = 0; c < 7; ++c) {
        for (int j = tid; j < npow2; j += kSortThreads) {
            float t = 0.0f;
            if (j < n && j != i) t = sorted_term(c, posm[j], vel[j], xi, vi, eps2);
            sk[j] = __float_as_uint(t);
        }
        __syncthreads();
        // bitonic sort of npow2 keys, ascending
        for (int k = 2; k <= npow2; k <<= 1) {
            for (int h = k >> 1; h > 0; h >>= 1) {
                for (int t = tid; t < npow2; t += kSortThreads) {
                    const int u = t ^ h;
                    if (u > t) {
                        const uint32_t a = sk[t], b = sk[u];
                        const bool asc = (t & k) == 0;
                        if (key_greater(a, b) == asc) {
                            sk[t] = b;
                            sk[u] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        float s = 0.0f;
        if (tid == 0)
            for (int k = 0; k < npow2; ++k) s = __fadd_rn(s, __uint_as_float(sk[k]));
        out[c] = s;
        __syncthreads();
    }
    if (tid == 0) {
        for (int c = 0; c < 3; ++c) {
            acc[3 * static_cast<size_t>(q) + c] = static_cast<double>(out[c]);
            jerk[3 * static_cast<size_t>(q) + c] = static_cast<double>(out[3 + c]);
        }
        pot[q] = static_cast<double>(out[6]);
    }
}

}  // namespace

cudaError_t force_sorted_launch(const JStream &js, int64_t n, const int32_t *active, int64_t n_act, float eps2,
                                double *acc, double *jerk, double *pot, DevStatus *st, cudaStream_t s)
{
    if (n_act <= 0) return cudaSuccess;
    if (n > kSortedMaxN) return cudaErrorInvalidValue;
    int npow2 = 2;
    while (npow2 < n) npow2 <<= 1;
    const size_t smem = static_cast<size_t>(npow2) * sizeof(uint32_t);
    static size_t smem_set = 0;
    if (smem > 48 * 1024 && smem > smem_set) {
        const cudaError_t e = cudaFuncSetAttribute(force_sorted_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    force_sorted_kernel<<<static_cast<unsigned>(n_act), kSortThreads, smem, s>>>(
        js.posm, js.vel, active, static_cast<int>(n), npow2, eps2, acc, jerk, pot, st);
    return cudaGetLastError();
}

}  // namespace nb

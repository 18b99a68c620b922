// Potential of the energy diagnostic in double-single arithmetic on the FP32
// pipe.  The energy (Sect. 4.2's accuracy measure; E = sum m v^2 / 2 +
// sum m phi / 2 with the softened potential, j = i excluded) is an O(N^2)
// pass.  In FP64 every pair costs an IEEE square root and a division on
// GB300's narrow FP64 pipe, about a minute at N = 2^20; here each pair is
// ~130 FP32 operations instead:
//
//   x_j, x_i, m_j, eps2: (hi, lo) splits of the FP64 values
//   dx = x_j - x_i, r2 = eps2 + dx.dx        (double-single)
//   1/sqrt(r2): MUFU seed and one Newton step with a double-single residual
//   phi_i -= m_j / r                          (double-single product)
//
// The terms of one 256-particle j-tile are added in double-single (they all
// have the same sign), and each tile's sum joins an FP64 running total, so the
// result agrees with the FP64 definition to ~1e-13 at any N.
#include "ds_arith.cuh"
#include "nbody_internal.cuh"

namespace nb {

namespace {

using namespace dsa;

constexpr int kPhiThreads = 256;
constexpr int kPhiTile = 256;

__device__ __forceinline__ ds split(const double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - static_cast<double>(h))};
}

__global__ void __launch_bounds__(kPhiThreads) phi_ds_kernel(const State S, const ds eps2, double *__restrict__ phi)
{
    __shared__ float sh[4][kPhiTile], sl[4][kPhiTile];  // x, y, z, m: hi and lo parts
    const int64_t i = blockIdx.x * static_cast<int64_t>(kPhiThreads) + threadIdx.x;
    const bool live = i < S.n;
    const int64_t li = live ? i : 0;
    const ds xi[3] = {split(S.x[0][li]), split(S.x[1][li]), split(S.x[2][li])};
    double p = 0.0;
    for (int64_t j0 = 0; j0 < S.n; j0 += kPhiTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kPhiTile; t += kPhiThreads) {
            const int64_t j = j0 + t;
            const bool ok = j < S.n;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const ds d = ok ? split(c < 3 ? S.x[c][j] : S.m[j]) : ds{0.0f, 0.0f};
                sh[c][t] = d.h;
                sl[c][t] = d.l;
            }
        }
        __syncthreads();
        const int jn = static_cast<int>(S.n - j0 < kPhiTile ? S.n - j0 : kPhiTile);
        ds tile = {0.0f, 0.0f};
#pragma unroll 2
        for (int t = 0; t < jn; ++t) {
            if (j0 + t == i) continue;  // j = i is not part of the sum
            const ds dx = ds_add({sh[0][t], sl[0][t]}, ds_neg(xi[0]));
            const ds dy = ds_add({sh[1][t], sl[1][t]}, ds_neg(xi[1]));
            const ds dz = ds_add({sh[2][t], sl[2][t]}, ds_neg(xi[2]));
            const ds r2 = ds_add(ds_add(ds_add(eps2, ds_mul(dx, dx)), ds_mul(dy, dy)), ds_mul(dz, dz));
            tile = ds_add(tile, ds_mul({sh[3][t], sl[3][t]}, ds_rsqrt(r2)));
        }
        p -= static_cast<double>(tile.h) + static_cast<double>(tile.l);
    }
    if (live) phi[i] = p;
}

}  // namespace

cudaError_t phi_ds_launch(const State &S, double eps2, double *phi, cudaStream_t s, int64_t *launches)
{
    const float e_hi = static_cast<float>(eps2);
    const ds e2 = {e_hi, static_cast<float>(eps2 - static_cast<double>(e_hi))};
    const unsigned blocks = static_cast<unsigned>((S.n + kPhiThreads - 1) / kPhiThreads);
    phi_ds_kernel<<<blocks, kPhiThreads, 0, s>>>(S, e2, phi);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace nb

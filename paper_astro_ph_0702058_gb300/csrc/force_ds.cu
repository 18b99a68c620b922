// Double-single force: the pair term of Appendix A evaluated entirely in
// double-single arithmetic (an unevaluated sum hi + lo of two floats, ~46
// significant bits) on the FP32 pipe, for a force that agrees with the FP64
// definition to ~1e-12 rather than the ~1e-7 of single-precision pair terms.
//
//   positions, velocities and masses: (hi, lo) splits of the FP64 values
//   dx = x_j - x_i, dv = v_j - v_i        (double-single subtraction)
//   r2 = eps2 + dx.dx                     (double-single products and sums)
//   1/sqrt(r2): single-precision seed y0 (MUFU), then one Newton step with
//               the residual rho = 1 - r2 y0^2 formed in double-single:
//               y = y0 (1 + rho/2 + 3 rho^2/8)
//   a += m r^-3 dx,  k += m r^-3 (dv - 3 (dx.dv) r^-2 dx),  phi -= m r^-1,
//   every product and sum in double-single.
//
// Building blocks in ds_arith.cuh: TwoSum, Fast2Sum and the FMA form of the
// exact product.
//
// One i-particle per thread; the CTA stages each 256-particle j-tile (the
// four float4 streams) in shared memory with ordinary loads, since the pair
// arithmetic (~400 FP32 operations) dwarfs the copy.  j-ranges over gridDim.y
// write (hi, lo) partial sums in the compensated mode's layout, which the
// compensated reduction adds in FP64.
#include "ds_arith.cuh"
#include "force_impl.cuh"

namespace nb {

namespace {

using namespace dsa;

constexpr int kDsThreads = 128;

struct DsParams {
    const float4 *__restrict__ posm;   // (x_hi, y_hi, z_hi, m_hi)
    const float4 *__restrict__ poslo;  // (x_lo, y_lo, z_lo, m_lo)
    const float4 *__restrict__ vel;    // (vx_hi, vy_hi, vz_hi, 0)
    const float4 *__restrict__ vello;  // (vx_lo, vy_lo, vz_lo, 0)
    const int32_t *__restrict__ active;
    int n_act, n, n_tiles;
    ds eps2;
    double *__restrict__ acc, *__restrict__ jerk, *__restrict__ pot;
    float *__restrict__ part;  // [split][14][n_act] when split > 1
    DevStatus *st;
};

__global__ void __launch_bounds__(kDsThreads) force_ds_kernel(const DsParams P)
{
    __shared__ float4 sp[kJTile], sl[kJTile], sv[kJTile], svl[kJTile];
    const int tid = threadIdx.x;
    const int q = blockIdx.x * kDsThreads + tid;
    int gi = -1;
    if (q < P.n_act) {
        gi = P.active[q];
        if (gi < 0 || gi >= P.n) {
            atomicOr(&P.st->flags, kFlagBadIndex);
            P.st->bad_index = q;
            gi = -1;
        }
    }
    const int l = gi >= 0 ? gi : 0;
    const float4 ph = P.posm[l], pl = P.poslo[l], vh = P.vel[l], vl = P.vello[l];
    const ds xi[3] = {{ph.x, pl.x}, {ph.y, pl.y}, {ph.z, pl.z}};
    const ds vi[3] = {{vh.x, vl.x}, {vh.y, vl.y}, {vh.z, vl.z}};
    ds sum[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) sum[c] = {0.0f, 0.0f};

    int t_begin, t_end;
    jrange_tiles(blockIdx.y, gridDim.y, P.n_tiles, t_begin, t_end);
    for (int t = t_begin; t < t_end; ++t) {
        const size_t off = static_cast<size_t>(t) * kJTile;
        __syncthreads();
        for (int e = tid; e < kJTile; e += kDsThreads) {
            sp[e] = P.posm[off + e];
            sl[e] = P.poslo[off + e];
            sv[e] = P.vel[off + e];
            svl[e] = P.vello[off + e];
        }
        __syncthreads();
        const int j0 = t * kJTile;
#pragma unroll 1
        for (int jj = 0; jj < kJTile; ++jj) {
            if (j0 + jj == gi) continue;  // j = i contributes nothing
            ds_pair_term(sp[jj], sl[jj], sv[jj], svl[jj], xi, vi, P.eps2, sum);
        }
    }
    if (q >= P.n_act) return;
    if (gridDim.y == 1) {
        double r[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) r[c] = static_cast<double>(sum[c].h) + static_cast<double>(sum[c].l);
        for (int c = 0; c < 3; ++c) {
            P.acc[3 * static_cast<size_t>(q) + c] = r[c];
            P.jerk[3 * static_cast<size_t>(q) + c] = r[3 + c];
        }
        P.pot[q] = r[6];
    } else {
        float *base = P.part + static_cast<size_t>(blockIdx.y) * 14 * P.n_act + q;
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            base[static_cast<size_t>(c) * P.n_act] = sum[c].h;
            base[static_cast<size_t>(7 + c) * P.n_act] = sum[c].l;
        }
    }
}

}  // namespace

int force_occupancy_ds()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, force_ds_kernel, kDsThreads, 0);
    return b;
}

cudaError_t force_ds_launch(const JStream &js, int64_t n, const int32_t *active, int64_t n_act, double eps2,
                            const ForceConfig &cfg, double *acc, double *jerk, double *pot, void *partials,
                            DevStatus *st, cudaStream_t s)
{
    DsParams P;
    P.posm = js.posm;
    P.poslo = js.poslo;
    P.vel = js.vel;
    P.vello = js.vello;
    P.active = active;
    P.n_act = static_cast<int>(n_act);
    P.n = static_cast<int>(n);
    P.n_tiles = static_cast<int>(js.n_pad / kJTile);
    const float e_hi = static_cast<float>(eps2);
    P.eps2 = {e_hi, static_cast<float>(eps2 - static_cast<double>(e_hi))};
    P.acc = acc;
    P.jerk = jerk;
    P.pot = pot;
    P.part = static_cast<float *>(partials);
    P.st = st;
    dim3 grid(static_cast<unsigned>((n_act + kDsThreads - 1) / kDsThreads), cfg.split);
    force_ds_kernel<<<grid, kDsThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace nb

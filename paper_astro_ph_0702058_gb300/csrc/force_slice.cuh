// The slice shape of the force evaluation (packed plain and compensated modes,
// SoA j-stream): one CTA of 512 threads per SM, CTA g taking the j-stream
// entries [g c, (g+1) c), c = ceil(n_pad / CTAs) rounded up to 4.  It copies
// its slice of every array into shared memory once, then sums the pair terms
// of all of the block's rows over it (rows_force of block_rows.cuh: T threads
// per row, T = 1 from 512 rows on, the packed pair term and 128-term folds,
// the potential included) and writes one partial per row in the layout of the
// j-range partials (range = CTA), which the two-dimensional reduction adds in
// CTA order.  For mid-size blocks this replaces many short (i-block, j-range)
// blocks by one evenly filled wave whose j are read from HBM or L2 once per SM.
#pragma once

#include "block_rows.cuh"

namespace nb {

constexpr int kSliceThreads = 512;

// Entries of the j-stream per CTA of the slice shape (a multiple of 4), or 0
// when that is more than kGrMaxChunk (the largest shared-memory copy).
inline int slice_chunk(const int64_t n_pad, const int ctas)
{
    if (ctas <= 0) return 0;
    const int64_t c = ((n_pad + ctas - 1) / ctas + 3) & ~int64_t(3);
    return c <= kGrMaxChunk ? static_cast<int>(c) : 0;
}

template <int MODE, int SJ>
__global__ void __launch_bounds__(kSliceThreads, 1) force_slice_kernel(const ForceParams P, const int chunk)
{
    constexpr int NA = SoaTile<MODE>::NA;
    constexpr bool DSW = MODE == kModeComp;
    constexpr int NC = DSW ? 14 : 7;  // floats per row of a partial
    extern __shared__ __align__(16) float jsm[];  // NA x SJ: this CTA's slice of each array
    __shared__ float wred[kSliceThreads / 32][7][2];
    const int g = static_cast<int>(blockIdx.x), tid = threadIdx.x;
    const int64_t n_pad = static_cast<int64_t>(P.n_tiles) * kJTile;
    const int lo = g * chunk;
    const int64_t hi = lo + chunk < n_pad ? lo + chunk : n_pad;
    const int L = hi > lo ? static_cast<int>(hi - lo) : 0;  // a multiple of 4
    const int na = P.n_act;
#pragma unroll
    for (int a = 0; a < NA; ++a) {  // 16-byte loads: n_pad and chunk are multiples of 4
        const float4 *src = reinterpret_cast<const float4 *>(P.soa + a * n_pad + lo);
        float4 *dst = reinterpret_cast<float4 *>(jsm + a * SJ);
        for (int k = tid; k < L / 4; k += kSliceThreads) dst[k] = __ldg(src + k);
    }
    __syncthreads();
    // T threads per row: the largest power of two with T na <= threads and at
    // least two groups of 4 j per thread (a CTA past the stream stores zeros)
    int T = kSliceThreads;
    while (T > 1 && (T * na > kSliceThreads || 8 * T > L)) T >>= 1;
    auto load_i = [&](const int rr, const bool live, I2 &I) {
        int idx = -1;
        if (live) {
            idx = P.active[rr];
            if (idx < 0 || idx >= P.n) {
                if (g == 0) {
                    atomicOr(&P.st->flags, kFlagBadIndex);
                    P.st->bad_index = rr;
                }
                idx = -1;
            }
        }
        const float *a = P.soa + (idx >= 0 ? idx : 0);
        const float x = a[0], y = a[n_pad], z = a[2 * n_pad];
        const float vx = a[4 * n_pad], vy = a[5 * n_pad], vz = a[6 * n_pad];
        I.x = f2_pack(x, x);
        I.y = f2_pack(y, y);
        I.z = f2_pack(z, z);
        I.vx = f2_pack(vx, vx);
        I.vy = f2_pack(vy, vy);
        I.vz = f2_pack(vz, vz);
        if (DSW) {
            const float lx = a[7 * n_pad], ly = a[8 * n_pad], lz = a[9 * n_pad];
            I.lx = f2_pack(lx, lx);
            I.ly = f2_pack(ly, ly);
            I.lz = f2_pack(lz, lz);
        }
        return idx;
    };
    auto no_ds = [](const int, const bool, dsa::ds (&)[3], dsa::ds (&)[3]) { return -1; };
    auto store = [&](const int rr, const float *tot, const float *lw) {
        float *d = P.part + static_cast<size_t>(g) * NC * na + rr;
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            d[static_cast<size_t>(c) * na] = tot[c];
            if (DSW) d[static_cast<size_t>(7 + c) * na] = lw[c];
        }
    };
    rows_force<MODE, kSliceThreads, SJ, true>(jsm, SJ, lo, L, na, T, P.eps2, 0.0f, load_i, no_ds, store, wred);
}

template <int MODE, int SJ>
cudaError_t launch_slice_sj(const ForceParams &P, const ForceConfig &cfg, const int chunk, cudaStream_t s)
{
    const size_t smem = static_cast<size_t>(SoaTile<MODE>::NA) * SJ * sizeof(float);
    static const cudaError_t set = cudaFuncSetAttribute(
        force_slice_kernel<MODE, SJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (set != cudaSuccess) return set;
    force_slice_kernel<MODE, SJ><<<cfg.split, kSliceThreads, smem, s>>>(P, chunk);
    return cudaGetLastError();
}

// The slice instance of the smallest shared-memory stride that holds a CTA's slice.
template <int MODE>
cudaError_t launch_force_slice(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s)
{
    if constexpr (NB_PACKED && (MODE == kModePlain || MODE == kModeComp)) {
        const int chunk = slice_chunk(static_cast<int64_t>(P.n_tiles) * kJTile, cfg.split);
        if (!P.soa || chunk == 0 || P.n_act_dev) return cudaErrorInvalidConfiguration;
        if (chunk <= 512) return launch_slice_sj<MODE, 512>(P, cfg, chunk, s);
        if (chunk <= 1024) return launch_slice_sj<MODE, 1024>(P, cfg, chunk, s);
        if (chunk <= 2048) return launch_slice_sj<MODE, 2048>(P, cfg, chunk, s);
        return launch_slice_sj<MODE, kGrMaxChunk>(P, cfg, chunk, s);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace nb

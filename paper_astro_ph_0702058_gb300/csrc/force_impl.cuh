// Direct-summation acceleration, jerk and potential (Eq. Force with the
// softened pair term of Appendix A of Portegies Zwart, Belleman & Geldof
// 2007), FP32 pair arithmetic on the FP32 j-stream.
//
// Kernel layout (one launch):
//   grid  = (i-blocks, j-ranges); block = NT threads; each thread owns IPT
//           active particles (rows q = blockIdx.x*NT*IPT + u*NT + threadIdx.x)
//           and keeps their position/velocity and sums in registers.
//   j     = the block's j-range is streamed through shared memory in tiles of
//           kJTile particles, double-buffered: one thread issues bulk async
//           (TMA) copies of the next tile while all threads work on the
//           current one; completion is tracked by an mbarrier per buffer.
//           Every thread reads the same j at the same time (shared-memory
//           broadcast), so the loop is bound by the FP32 pipe.
//   sums  = per PF pairs, fresh FP32 partial sums; each partial is then
//           folded into the running total: an FP32 add (plain mode) or Knuth's
//           TwoSum into a (hi, lo) double-single pair (compensated mode).
//   split = with more than one j-range, each range writes its sums to scratch
//           and a second kernel adds the ranges in a fixed order (FP64), so
//           results never depend on scheduling.
// The self pair j = i is excluded exactly (Eq. Force sums over j != i): a
// thread whose own i lies in the current tile runs a copy of the tile loop
// that zeroes the term with j == i; all other tiles run without the test.
// This also makes eps2 = 0 safe (r = 0 occurs only for j = i).
#pragma once

#include "nbody_internal.cuh"
#include "ptx.cuh"

// Compile-time tuning of the tile loop: unroll factor of the j loop and the
// number of pairs summed in FP32 before each fold into the running total.
#ifndef NB_JUNROLL
#define NB_JUNROLL 8
#endif
#ifndef NB_FOLD
#define NB_FOLD 128
#endif

namespace nb {

constexpr int kJUnroll = NB_JUNROLL;

struct ForceParams {
    const float4 *__restrict__ posm;
    const float4 *__restrict__ vel;
    const float4 *__restrict__ poslo;
    const float *__restrict__ soa;  // SoA j-stream (kSoaArrays x n_tiles * kJTile), or NULL
    const int32_t *__restrict__ active;
    int n_act;
    const long long *n_act_dev;  // when set, the block size is read here on the device (graph replays);
                                 // n_act then only bounds the launch
    int n;
    int n_tiles;  // j-ranges: jrange_tiles over gridDim.y
    float eps2;
    double *__restrict__ acc;
    double *__restrict__ jerk;
    double *__restrict__ pot;
    float *__restrict__ part;  // [split][7 or 14][n_act] when split > 1
    DevStatus *st;
    int skip_first_copy;       // test hook: leave the first tile's copy out
    unsigned long long opaque_zero;  // always 0; hides values from the assembler (f2_opaque)
};

// One pair term, Appendix A: dx = x_j - x_i, dv = v_j - v_i, r^2 = eps^2 + dx.dx,
// a += m r^-3 dx, k += m r^-3 (dv - 3 (dx.dv) r^-2 dx), phi -= m r^-1.
// Compensated mode forms dx from the hi/lo splits of the FP64 positions.
// 27 FP32 operations + 1 MUFU rsqrt (plain); 33 + 1 (compensated).
template <int MODE, bool SELF>
__device__ __forceinline__ void pair_term(const float4 pj, const float4 vj, const float4 lj,
                                          const float4 xi, const float4 vi, const float4 li,
                                          const float eps2, const int j, const int i, float (&p)[7])
{
    float dx, dy, dz;
    if (is_ds(MODE)) {
        dx = (pj.x - xi.x) + (lj.x - li.x);
        dy = (pj.y - xi.y) + (lj.y - li.y);
        dz = (pj.z - xi.z) + (lj.z - li.z);
    } else {
        dx = pj.x - xi.x;
        dy = pj.y - xi.y;
        dz = pj.z - xi.z;
    }
    const float dvx = vj.x - vi.x;
    const float dvy = vj.y - vi.y;
    const float dvz = vj.z - vi.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
    float rinv = rsqrt_mufu(r2);
    if (SELF) rinv = (j == i) ? 0.0f : rinv;  // j = i contributes nothing
    const float xv = fmaf(dz, dvz, fmaf(dy, dvy, dx * dvx));
    const float rinv2 = rinv * rinv;
    const float mr = pj.w * rinv;
    const float mr3 = mr * rinv2;
    const float w = 3.0f * (xv * rinv2);
    p[0] = fmaf(mr3, dx, p[0]);
    p[1] = fmaf(mr3, dy, p[1]);
    p[2] = fmaf(mr3, dz, p[2]);
    p[3] = fmaf(mr3, fmaf(-w, dx, dvx), p[3]);
    p[4] = fmaf(mr3, fmaf(-w, dy, dvy), p[4]);
    p[5] = fmaf(mr3, fmaf(-w, dz, dvz), p[5]);
    p[6] = p[6] - mr;
}

// Knuth's TwoSum (TAOCP vol. 2, 4.2.2): s + e == hi + x exactly; the error is
// kept in lo, so (hi, lo) carries ~48 significant bits.
__device__ __forceinline__ void fold_ds(float &hi, float &lo, const float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo = lo + e;
}

// The same fold with round-to-nearest intrinsics, which the compiler never
// fuses with the operations around them.
__device__ __forceinline__ void fold_ds_rn(float &hi, float &lo, const float x)
{
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// Adds the double-single sum (h2, l2) to (hi, lo): TwoSum of the high words,
// then the low words and its error (symmetric in its two operands).  On the
// FP32 pipe: GB300's FP64 unit takes ~19 cycles per warp instruction.
__device__ __forceinline__ void ds2_add(float &hi, float &lo, const float h2, const float l2)
{
    const float s = __fadd_rn(hi, h2);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, l2), e);
}

// Summation-check pair term: the compensated pair term with every operation
// written as a round-to-nearest intrinsic in a fixed order and the correctly
// rounded reciprocal square root, each of the 7 terms folded into (tot, lo)
// on its own.  A CPU that follows the same order forms the same FP32 terms,
// so the only difference left is the summation.
//   dx = (xj_hi - xi_hi) + (xj_lo - xi_lo);  dv = vj - vi
//   r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));  rinv = rsqrt_rn(r2)
//   xv = fma(dz, dvz, fma(dy, dvy, dx * dvx))
//   mr = m * rinv;  mr3 = mr * (rinv * rinv);  w = 3 * (xv * (rinv * rinv))
//   terms: mr3 * dx_c,  mr3 * fma(-w, dx_c, dv_c),  -mr
template <bool SELF>
__device__ __forceinline__ void pair_term_check(const float4 pj, const float4 vj, const float4 lj,
                                                const float4 xi, const float4 vi, const float4 li,
                                                const float eps2, const int j, const int i, float (&tot)[7],
                                                float (&lo)[7])
{
    const float dx = __fadd_rn(__fsub_rn(pj.x, xi.x), __fsub_rn(lj.x, li.x));
    const float dy = __fadd_rn(__fsub_rn(pj.y, xi.y), __fsub_rn(lj.y, li.y));
    const float dz = __fadd_rn(__fsub_rn(pj.z, xi.z), __fsub_rn(lj.z, li.z));
    const float dvx = __fsub_rn(vj.x, vi.x);
    const float dvy = __fsub_rn(vj.y, vi.y);
    const float dvz = __fsub_rn(vj.z, vi.z);
    if (SELF && j == i) return;  // j = i contributes nothing
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, eps2)));
    const float rinv = __frsqrt_rn(r2);
    const float xv = __fmaf_rn(dz, dvz, __fmaf_rn(dy, dvy, __fmul_rn(dx, dvx)));
    const float rinv2 = __fmul_rn(rinv, rinv);
    const float mr = __fmul_rn(pj.w, rinv);
    const float mr3 = __fmul_rn(mr, rinv2);
    const float w = __fmul_rn(3.0f, __fmul_rn(xv, rinv2));
    fold_ds_rn(tot[0], lo[0], __fmul_rn(mr3, dx));
    fold_ds_rn(tot[1], lo[1], __fmul_rn(mr3, dy));
    fold_ds_rn(tot[2], lo[2], __fmul_rn(mr3, dz));
    fold_ds_rn(tot[3], lo[3], __fmul_rn(mr3, __fmaf_rn(-w, dx, dvx)));
    fold_ds_rn(tot[4], lo[4], __fmul_rn(mr3, __fmaf_rn(-w, dy, dvy)));
    fold_ds_rn(tot[5], lo[5], __fmul_rn(mr3, __fmaf_rn(-w, dz, dvz)));
    fold_ds_rn(tot[6], lo[6], -mr);
}

// Fold length (pairs per FP32 partial) of each mode.
template <int MODE>
struct FoldLen {
    static constexpr int value = NB_FOLD;
};
template <>
struct FoldLen<kModeCheck> {
    static constexpr int value = 1;
};

// Sums over one staged tile of kJTile j (starting at global index j0).
template <int MODE, int IPT, int PF, bool SELF>
__device__ __forceinline__ void tile_sums(const float4 *sp, const float4 *sv, const float4 *sl, const int j0,
                                          const float4 (&xi)[IPT], const float4 (&vi)[IPT],
                                          const float4 (&li)[IPT], const int (&gi)[IPT], const float eps2,
                                          float (&tot)[IPT][7], float (&lo)[IPT][7])
{
    if constexpr (MODE == kModeCheck) {
#pragma unroll 4
        for (int jj = 0; jj < kJTile; ++jj) {
            const float4 pj = sp[jj], vj = sv[jj], lj = sl[jj];
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                pair_term_check<SELF>(pj, vj, lj, xi[u], vi[u], li[u], eps2, j0 + jj, gi[u], tot[u], lo[u]);
        }
        return;
    }
#pragma unroll 1
    for (int jb = 0; jb < kJTile; jb += PF) {
        float p[IPT][7];
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int c = 0; c < 7; ++c) p[u][c] = 0.0f;
#pragma unroll kJUnroll
        for (int jj = 0; jj < PF; ++jj) {
            const float4 pj = sp[jb + jj];
            const float4 vj = sv[jb + jj];
            const float4 lj = (is_ds(MODE)) ? sl[jb + jj] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                pair_term<MODE, SELF>(pj, vj, lj, xi[u], vi[u], li[u], eps2, j0 + jb + jj, gi[u], p[u]);
        }
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                if (is_ds(MODE))
                    fold_ds(tot[u][c], lo[u][c], p[u][c]);
                else
                    tot[u][c] += p[u][c];
            }
    }
}

template <int MODE, int NT, int IPT, int PF>
__global__ void __launch_bounds__(NT) force_kernel(const ForceParams P)
{
    constexpr int NARR = (is_ds(MODE)) ? 3 : 2;
    constexpr uint32_t kTileBytes = kJTile * sizeof(float4);
    static_assert(kJTile % PF == 0, "fold length must divide the tile");
    __shared__ __align__(128) float4 sj[2][NARR][kJTile];
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    int t_begin, t_end;
    jrange_tiles(blockIdx.y, gridDim.y, P.n_tiles, t_begin, t_end);

    float4 xi[IPT], vi[IPT], li[IPT];
    int gi[IPT];
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        const int q = (blockIdx.x * IPT + u) * NT + tid;
        int idx = -1;
        if (q < P.n_act) {
            idx = P.active[q];
            if (idx < 0 || idx >= P.n) {
                atomicOr(&P.st->flags, kFlagBadIndex);
                P.st->bad_index = q;
                idx = -1;
            }
        }
        gi[u] = idx;
        const int l = idx >= 0 ? idx : 0;
        xi[u] = P.posm[l];
        vi[u] = P.vel[l];
        li[u] = (is_ds(MODE)) ? P.poslo[l] : make_float4(0.f, 0.f, 0.f, 0.f);
    }

    float tot[IPT][7], lo[IPT][7];
#pragma unroll
    for (int u = 0; u < IPT; ++u)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            tot[u][c] = 0.0f;
            lo[u][c] = 0.0f;
        }

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int tile, int b) {
        mbar_arrive_expect_tx(&bar[b], NARR * kTileBytes);
        const size_t off = static_cast<size_t>(tile) * kJTile;
        bulk_g2s(sj[b][0], P.posm + off, kTileBytes, &bar[b]);
        bulk_g2s(sj[b][1], P.vel + off, kTileBytes, &bar[b]);
        if (is_ds(MODE)) bulk_g2s(sj[b][NARR - 1], P.poslo + off, kTileBytes, &bar[b]);
    };

    bool ok = true;
    int it_stop = 0;
    if (tid == 0 && t_begin < t_end && !P.skip_first_copy) issue(t_begin, 0);
    for (int t = t_begin; t < t_end; ++t) {
        const int it = t - t_begin;
        const int b = it & 1;
        if (tid == 0 && t + 1 < t_end) issue(t + 1, b ^ 1);
        ok = mbar_wait_bounded(&bar[b], (it >> 1) & 1);
        if (ok) {
            const int j0 = t * kJTile;
            bool self_tile = false;
#pragma unroll
            for (int u = 0; u < IPT; ++u) self_tile |= static_cast<unsigned>(gi[u] - j0) < static_cast<unsigned>(kJTile);
            if (self_tile)
                tile_sums<MODE, IPT, PF, true>(sj[b][0], sj[b][1], sj[b][NARR - 1], j0, xi, vi, li, gi, P.eps2, tot, lo);
            else
                tile_sums<MODE, IPT, PF, false>(sj[b][0], sj[b][1], sj[b][NARR - 1], j0, xi, vi, li, gi, P.eps2, tot, lo);
        }
        if (__syncthreads_or(!ok)) {
            ok = false;
            it_stop = it;
            break;
        }
    }

    if (!ok) {
        // A tile never arrived.  Drain (with a bound) the copies this block
        // may still have in flight, record the timeout and leave the outputs
        // untouched; the host reports NBODY_ETIMEOUT.
        if (tid == 0) {
            const int b = it_stop & 1;
            mbar_wait_bounded(&bar[b], (it_stop >> 1) & 1);
            if (t_begin + it_stop + 1 < t_end) mbar_wait_bounded(&bar[b ^ 1], ((it_stop + 1) >> 1) & 1);
            atomicOr(&P.st->flags, kFlagTimeout);
        }
        return;
    }

#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        const int q = (blockIdx.x * IPT + u) * NT + tid;
        if (q >= P.n_act) continue;
        if (gridDim.y == 1) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c)
                r[c] = (is_ds(MODE)) ? static_cast<double>(tot[u][c]) + static_cast<double>(lo[u][c])
                                           : static_cast<double>(tot[u][c]);
            double *pa = P.acc + 3 * static_cast<size_t>(q);
            double *pk = P.jerk + 3 * static_cast<size_t>(q);
            pa[0] = r[0];
            pa[1] = r[1];
            pa[2] = r[2];
            pk[0] = r[3];
            pk[1] = r[4];
            pk[2] = r[5];
            P.pot[q] = r[6];
        } else {
            constexpr int NC = (is_ds(MODE)) ? 14 : 7;
            float *base = P.part + static_cast<size_t>(blockIdx.y) * NC * P.n_act + q;
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                base[static_cast<size_t>(c) * P.n_act] = tot[u][c];
                if (is_ds(MODE)) base[static_cast<size_t>(7 + c) * P.n_act] = lo[u][c];
            }
        }
    }
}

// Adds the j-range partial sums of each row in ascending range order (FP64),
// one thread per (row, component): 7 n_act threads, reads coalesced over rows.
template <int MODE>
__global__ void reduce_partials_kernel(const float *__restrict__ part, int split, int n_act,
                                       double *__restrict__ acc, double *__restrict__ jerk,
                                       double *__restrict__ pot, const long long *n_act_dev)
{
    constexpr int NC = (is_ds(MODE)) ? 14 : 7;
    if (n_act_dev) n_act = static_cast<int>(*n_act_dev);
    const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (idx >= 7LL * n_act) return;
    const int c = static_cast<int>(idx / n_act);
    const int q = static_cast<int>(idx - static_cast<int64_t>(c) * n_act);
    double s = 0.0;
    for (int sp = 0; sp < split; ++sp) {
        const float *b = part + static_cast<size_t>(sp) * NC * n_act + q;
        s += static_cast<double>(b[static_cast<size_t>(c) * n_act]);
        if (is_ds(MODE)) s += static_cast<double>(b[static_cast<size_t>(7 + c) * n_act]);
    }
    if (c < 3)
        acc[3 * static_cast<size_t>(q) + c] = s;
    else if (c < 6)
        jerk[3 * static_cast<size_t>(q) + c - 3] = s;
    else
        pot[q] = s;
}

// The same sums for many j-ranges: a block of 256 threads holds 8 consecutive
// rows of one component and 32 lanes per row; lane w adds the ranges w, w + 32,
// ... of its row (ascending), so a warp loads 8 consecutive floats (one 32-byte
// sector) of each of 4 ranges, and a row's ranges are spread over 32 lanes.  The
// lane sums of a row are then added in lane order.  The order depends on the
// split only, not on the number of rows a launch is sized for.  The sums are
// double-single pairs on the FP32 pipe (ds2_add, ~2^-48 relative per addition),
// FP64 in the summation-check mode.  Grid: (ceil(n_act / 8), 7).
template <int MODE, int R>
__global__ void __launch_bounds__(256) reduce_partials_2d_kernel(const float *__restrict__ part, int split,
                                                                 int n_act, double *__restrict__ acc,
                                                                 double *__restrict__ jerk,
                                                                 double *__restrict__ pot, const long long *n_act_dev)
{
    constexpr int NC = (is_ds(MODE)) ? 14 : 7;
    constexpr int L = 256 / R;  // lanes per row
    constexpr bool F64 = MODE == kModeCheck;
    __shared__ double sh[L][R];
    __shared__ float shh[L][R], shl[L][R];
    if (n_act_dev) n_act = static_cast<int>(*n_act_dev);
    const int row = threadIdx.x % R, w = threadIdx.x / R;
    const int c = blockIdx.y;
    const int q = blockIdx.x * R + row;
    if (static_cast<int>(blockIdx.x) * R >= n_act) return;  // a launch sized for more rows
    double r = 0.0;
    float rh = 0.0f, rl = 0.0f;
    if (q < n_act) {
        for (int sp = w; sp < split; sp += L) {
            const float *b = part + (static_cast<size_t>(sp) * NC + c) * n_act + q;
            const float l2 = is_ds(MODE) ? b[static_cast<size_t>(7) * n_act] : 0.0f;
            if constexpr (F64) {
                r += static_cast<double>(b[0]);
                if (is_ds(MODE)) r += static_cast<double>(l2);
            } else {
                ds2_add(rh, rl, b[0], l2);
            }
        }
    }
    if constexpr (F64) {
        sh[w][row] = r;
    } else {
        shh[w][row] = rh;
        shl[w][row] = rl;
    }
    __syncthreads();
    if (w == 0 && q < n_act) {
        double t;
        if constexpr (F64) {
            t = sh[0][row];
            for (int k = 1; k < L; ++k) t += sh[k][row];
        } else {
            float th = shh[0][row], tl = shl[0][row];
            for (int k = 1; k < L; ++k) ds2_add(th, tl, shh[k][row], shl[k][row]);
            t = static_cast<double>(th) + static_cast<double>(tl);
        }
        if (c < 3)
            acc[3 * static_cast<size_t>(q) + c] = t;
        else if (c < 6)
            jerk[3 * static_cast<size_t>(q) + c - 3] = t;
        else
            pot[q] = t;
    }
}

}  // namespace nb

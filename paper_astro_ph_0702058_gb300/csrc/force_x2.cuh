// Packed-FP32 (f32x2) form of the force kernel of force_impl.cuh.
//
// Blackwell executes `fma/mul/add/sub .f32x2` on two FP32 values per lane
// in one instruction.  The pair loop issues ~30 instructions per pair in the
// scalar form and is limited by instruction dispatch, not by the FP32 pipe;
// here two consecutive j share one packed instruction stream:
//   - j-tiles arrive in structure-of-arrays shared memory, one bulk async
//     copy per array from the SoA j-stream, double-buffered, two tiles per
//     mbarrier and block barrier for blocks of 128 threads or more (a
//     float4-only stream, as no-alloc callers pass, is staged and transposed
//     instead); one 128-bit shared load then yields two packed (j, j+1)
//     pairs of a component;
//   - each i-particle is broadcast once into packed registers {x_i, x_i};
//   - the pair term of Appendix A runs on packed operands, with the MUFU
//     reciprocal square root applied to each half;
//   - the two halves hold partial sums of the even and odd j of a fold; they
//     are added at each fold (NB_FOLD pairs), then folded into the running total as in
//     the scalar kernel (FP32 add, or TwoSum into double-single).
#pragma once

#include "force_impl.cuh"

#ifndef NB_PACKED
#define NB_PACKED 1
#endif
// Register cap per thread for the packed kernels (0 = none): the launch
// bounds then ask for 65536 / (NT * cap) resident blocks per SM.
#ifndef NB_X2_REGCAP
#define NB_X2_REGCAP 0
#endif
// Unroll factor of the packed loop over groups of NB_X2_JSTEP j, and the
// group size: 4 (one 128-bit shared load per array gives two packed pairs)
// or 2 (one 64-bit load, half the registers for staged j).
#ifndef NB_X2_UNROLL
#define NB_X2_UNROLL 2
#endif
#ifndef NB_X2_JSTEP
#define NB_X2_JSTEP 4
#endif
// Tiles per barrier in the SoA-tile kernel: each group of NB_X2_TGROUP tiles
// arrives on one mbarrier and ends with one block barrier.
#ifndef NB_X2_TGROUP
#define NB_X2_TGROUP 2
#endif
#define NB_PRAGMA(x) _Pragma(#x)
#define NB_UNROLL(n) NB_PRAGMA(unroll n)

namespace nb {

typedef unsigned long long f2_t;  // two packed floats {lo, hi}

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t r, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

struct I2 {  // one i-particle, broadcast into both halves
    f2_t x, y, z, vx, vy, vz, lx, ly, lz;
};

// Two pair terms (j = 2 consecutive particles, one i) on packed operands.
template <int MODE, bool SELF>
__device__ __forceinline__ void pair_term_x2(const f2_t X, const f2_t Y, const f2_t Z, const f2_t M,
                                             const f2_t VX, const f2_t VY, const f2_t VZ, const f2_t LX,
                                             const f2_t LY, const f2_t LZ, const I2 &I, const f2_t E2,
                                             const f2_t NEG3, const int j_even, const int gi, f2_t (&p)[7])
{
    f2_t dx, dy, dz;
    if (MODE == kModeComp) {
        dx = f2_add(f2_sub(X, I.x), f2_sub(LX, I.lx));
        dy = f2_add(f2_sub(Y, I.y), f2_sub(LY, I.ly));
        dz = f2_add(f2_sub(Z, I.z), f2_sub(LZ, I.lz));
    } else {
        dx = f2_sub(X, I.x);
        dy = f2_sub(Y, I.y);
        dz = f2_sub(Z, I.z);
    }
    const f2_t dvx = f2_sub(VX, I.vx), dvy = f2_sub(VY, I.vy), dvz = f2_sub(VZ, I.vz);
    const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, E2)));
    float r2a, r2b;
    f2_unpack(r2, r2a, r2b);
    float ra = rsqrt_mufu(r2a), rb = rsqrt_mufu(r2b);
    if (SELF) {
        ra = (j_even == gi) ? 0.0f : ra;
        rb = (j_even + 1 == gi) ? 0.0f : rb;
    }
    const f2_t rinv = f2_pack(ra, rb);
    const f2_t xv = f2_fma(dz, dvz, f2_fma(dy, dvy, f2_mul(dx, dvx)));
    const f2_t rinv2 = f2_mul(rinv, rinv);
    const f2_t mr = f2_mul(M, rinv);
    const f2_t mr3 = f2_mul(mr, rinv2);
    const f2_t wn = f2_mul(f2_mul(xv, rinv2), NEG3);  // -3 (dx.dv) r^-2
    p[0] = f2_fma(mr3, dx, p[0]);
    p[1] = f2_fma(mr3, dy, p[1]);
    p[2] = f2_fma(mr3, dz, p[2]);
    p[3] = f2_fma(mr3, f2_fma(wn, dx, dvx), p[3]);
    p[4] = f2_fma(mr3, f2_fma(wn, dy, dvy), p[4]);
    p[5] = f2_fma(mr3, f2_fma(wn, dz, dvz), p[5]);
    p[6] = f2_sub(p[6], mr);
}

// Knuth's TwoSum on both halves at once: hi + x == s + e exactly per half,
// e kept in lo (fold_ds of force_impl.cuh, packed).  Inline PTX is never
// contracted, so every operation rounds as written.
__device__ __forceinline__ void fold_ds_x2(f2_t &hi, f2_t &lo, const f2_t x)
{
    const f2_t s = f2_add(hi, x);
    const f2_t bb = f2_sub(s, hi);
    const f2_t e = f2_add(f2_sub(hi, f2_sub(s, bb)), f2_sub(x, bb));
    hi = s;
    lo = f2_add(lo, e);
}

// x ^ z for a z that is zero at run time but unknown to the compiler: the value
// is unchanged, but it leaves through an integer operation, so the assembler can
// no longer fuse the packed product that formed x into an instruction that
// uses it.  Without this it fuses a term's product into the TwoSum that folds
// the term (even with multiply-add contraction switched off), which keeps the
// product's own rounding error in the low word.
__device__ __forceinline__ f2_t f2_opaque(const f2_t x, const unsigned long long z)
{
    f2_t r;
    asm("xor.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(z));
    return r;
}

// Summation-check form of pair_term_x2 (kModeCheck): the compensated pair term
// with the correctly rounded reciprocal square root (per half), every term
// formed by its own product (no multiply-add into the sums), and each of the
// 7 terms of each half folded at once into packed double-single sums (fold
// length 1).  The operations and their order are those of the CPU's FP32-term
// sums, so both form the same FP32 terms:
//   dx = (xj_hi - xi_hi) + (xj_lo - xi_lo);  dv = vj - vi
//   r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));  rinv = rsqrt_rn(r2)
//   xv = fma(dz, dvz, fma(dy, dvy, dx * dvx));  mr = m rinv;  mr3 = mr (rinv rinv)
//   terms: mr3 dx,  mr3 fma(-3 (xv (rinv rinv)), dx, dv),  -mr
// (x (-3) rounds to the negation of 3 x, so the jerk term is the CPU's bit for bit.)
// Each term passes through f2_opaque (z = 0) before its fold, so it is folded
// as the rounded FP32 value.
template <bool SELF>
__device__ __forceinline__ void pair_term_x2_check(const f2_t X, const f2_t Y, const f2_t Z, const f2_t M,
                                                   const f2_t VX, const f2_t VY, const f2_t VZ, const f2_t LX,
                                                   const f2_t LY, const f2_t LZ, const I2 &I, const f2_t E2,
                                                   const f2_t NEG3, const int j_even, const int gi,
                                                   const unsigned long long z, f2_t (&hi)[7], f2_t (&lo)[7])
{
    const f2_t dx = f2_add(f2_sub(X, I.x), f2_sub(LX, I.lx));
    const f2_t dy = f2_add(f2_sub(Y, I.y), f2_sub(LY, I.ly));
    const f2_t dz = f2_add(f2_sub(Z, I.z), f2_sub(LZ, I.lz));
    const f2_t dvx = f2_sub(VX, I.vx), dvy = f2_sub(VY, I.vy), dvz = f2_sub(VZ, I.vz);
    const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, E2)));
    float r2a, r2b;
    f2_unpack(r2, r2a, r2b);
    float ra = __frsqrt_rn(r2a), rb = __frsqrt_rn(r2b);
    if (SELF) {  // j = i: every term becomes an exact zero, and folding a zero changes nothing
        ra = (j_even == gi) ? 0.0f : ra;
        rb = (j_even + 1 == gi) ? 0.0f : rb;
    }
    const f2_t rinv = f2_pack(ra, rb);
    const f2_t xv = f2_fma(dz, dvz, f2_fma(dy, dvy, f2_mul(dx, dvx)));
    const f2_t rinv2 = f2_mul(rinv, rinv);
    const f2_t mr = f2_mul(M, rinv);
    const f2_t mr3 = f2_mul(mr, rinv2);
    const f2_t wn = f2_mul(f2_mul(xv, rinv2), NEG3);
    fold_ds_x2(hi[0], lo[0], f2_opaque(f2_mul(mr3, dx), z));
    fold_ds_x2(hi[1], lo[1], f2_opaque(f2_mul(mr3, dy), z));
    fold_ds_x2(hi[2], lo[2], f2_opaque(f2_mul(mr3, dz), z));
    fold_ds_x2(hi[3], lo[3], f2_opaque(f2_mul(mr3, f2_fma(wn, dx, dvx)), z));
    fold_ds_x2(hi[4], lo[4], f2_opaque(f2_mul(mr3, f2_fma(wn, dy, dvy)), z));
    fold_ds_x2(hi[5], lo[5], f2_opaque(f2_mul(mr3, f2_fma(wn, dz, dvz)), z));
    fold_ds_x2(hi[6], lo[6], f2_opaque(f2_sub(0ull, mr), z));
}

// Structure-of-arrays copy of one tile: x y z m vx vy vz (lx ly lz).
template <int MODE>
struct SoaTile {
    static constexpr int NA = is_ds(MODE) ? 10 : 7;
    float a[NA][kJTile];
};

// Summation-check sums over one tile: every pair term of each half folded
// into the packed double-single sums ph, pl.
template <int IPT, bool SELF>
__device__ __forceinline__ void tile_sums_x2_check(const SoaTile<kModeCheck> &T, const int j0, const I2 (&I)[IPT],
                                                   const int (&gi)[IPT], const f2_t E2, const f2_t NEG3,
                                                   const unsigned long long z, f2_t (&ph)[IPT][7],
                                                   f2_t (&pl)[IPT][7])
{
#pragma unroll 2
    for (int jj = 0; jj < kJTile; jj += 4) {
        f2_t v[10][2];
#pragma unroll
        for (int a = 0; a < 10; ++a) {
            const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(&T.a[a][jj]);
            v[a][0] = q.x;
            v[a][1] = q.y;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                pair_term_x2_check<SELF>(v[0][h], v[1][h], v[2][h], v[3][h], v[4][h], v[5][h], v[6][h], v[7][h],
                                         v[8][h], v[9][h], I[u], E2, NEG3, j0 + jj + 2 * h, gi[u], z, ph[u],
                                         pl[u]);
    }
}

// Sums over the j of one staged tile (starting at global index j0), or over
// the JL of them from jstart on (a j-subgroup's share of the tile).
template <int MODE, int IPT, int PF, bool SELF, int JL = kJTile>
__device__ __forceinline__ void tile_sums_x2(const SoaTile<MODE> &T, const int j0, const I2 (&I)[IPT],
                                             const int (&gi)[IPT], const f2_t E2, const f2_t NEG3,
                                             float (&tot)[IPT][7], float (&lo)[IPT][7], const int jstart = 0)
{
    static_assert(JL % PF == 0 || PF % JL == 0, "fold length and j share");
#pragma unroll 1
    for (int jb = jstart; jb < jstart + JL; jb += (PF < JL ? PF : JL)) {
        f2_t p[IPT][7];
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int c = 0; c < 7; ++c) p[u][c] = 0ull;
        constexpr int JS = NB_X2_JSTEP;
        static_assert(JS == 2 || JS == 4, "j group of 2 or 4");
NB_UNROLL(NB_X2_UNROLL)
        for (int jj = 0; jj < (PF < JL ? PF : JL); jj += JS) {
            f2_t v[SoaTile<MODE>::NA][JS / 2];
#pragma unroll
            for (int a = 0; a < SoaTile<MODE>::NA; ++a) {
                if constexpr (JS == 4) {
                    const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(&T.a[a][jb + jj]);
                    v[a][0] = q.x;
                    v[a][JS / 2 - 1] = q.y;
                } else {
                    v[a][0] = *reinterpret_cast<const f2_t *>(&T.a[a][jb + jj]);
                }
            }
#pragma unroll
            for (int h = 0; h < JS / 2; ++h)
#pragma unroll
                for (int u = 0; u < IPT; ++u)
                    pair_term_x2<MODE, SELF>(v[0][h], v[1][h], v[2][h], v[3][h], v[4][h], v[5][h], v[6][h],
                                             is_ds(MODE) ? v[SoaTile<MODE>::NA - 3][h] : 0ull,
                                             is_ds(MODE) ? v[SoaTile<MODE>::NA - 2][h] : 0ull,
                                             is_ds(MODE) ? v[SoaTile<MODE>::NA - 1][h] : 0ull, I[u], E2,
                                             NEG3, j0 + jb + jj + 2 * h, gi[u], p[u]);
        }
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                float e, o;
                f2_unpack(p[u][c], e, o);
                const float part = e + o;
                if (MODE == kModeComp)
                    fold_ds(tot[u][c], lo[u][c], part);
                else
                    tot[u][c] += part;
            }
    }
}

#if NB_X2_REGCAP > 0
#define NB_X2_BOUNDS(NT) __launch_bounds__(NT, (65536 / ((NT) * NB_X2_REGCAP) > 0 ? 65536 / ((NT) * NB_X2_REGCAP) : 1))
#else
#define NB_X2_BOUNDS(NT) __launch_bounds__(NT)
#endif

template <int MODE, int NT, int IPT, int PF, bool SOAIN, int JSUB = 1>
__global__ void NB_X2_BOUNDS(NT) force_kernel_x2(const ForceParams P)
{
    // SOAIN: the tiles come straight from the SoA j-stream into the SoA tile
    // buffers (one bulk copy per array, one barrier per tile); otherwise the
    // float4 stream is staged and transposed (two barriers per tile).
    // JSUB > 1: a block holds NT / JSUB rows, each with JSUB threads that take
    // consecutive quarters (JSUB = 4) of every tile; at the end the JSUB sums of a
    // row are added in shared memory in subgroup order (double-single, on the
    // FP32 pipe: GB300's FP64 unit would take ~19 cycles per warp instruction).  The same rows
    // per block as JSUB = 1 with NT / JSUB threads, but blocks JSUB times shorter:
    // more, evenly filled waves for mid-size blocks, and each tile copy serves
    // JSUB times the pairs.
    static_assert(JSUB == 1 || (IPT == 1 && SOAIN && NT % (32 * JSUB) == 0), "j-subgroups: one row per thread");
    constexpr int RB = NT / JSUB;          // rows of a block (per i of a thread)
    constexpr int JL = kJTile / JSUB;      // j of a tile per subgroup
    constexpr int NARR = is_ds(MODE) ? 3 : 2;
    constexpr int NA = SoaTile<MODE>::NA;
    constexpr uint32_t kTileBytes = kJTile * sizeof(float4);
    constexpr uint32_t kArrBytes = kJTile * sizeof(float);
    static_assert(MODE == kModeCheck || (kJTile % PF == 0 && PF % 4 == 0), "fold length");
    __shared__ __align__(128) float4 sj[SOAIN ? 1 : 2][SOAIN ? 1 : NARR][SOAIN ? 1 : kJTile];
    // small blocks keep one tile per group: their occupancy is set by shared memory
    constexpr int TG = (SOAIN && NT >= 128) ? NB_X2_TGROUP : 1;
    __shared__ __align__(128) SoaTile<MODE> soa[SOAIN ? 2 * TG : 1];
    __shared__ __align__(8) uint64_t bar[2];

    const int n_act = P.n_act_dev ? static_cast<int>(*P.n_act_dev) : P.n_act;
    if (static_cast<int>(blockIdx.x) * RB * IPT >= n_act) return;  // a launch sized for more rows
    const int tid = threadIdx.x;
    const int row = tid % RB, sub = tid / RB;
    int t_begin, t_end;
    jrange_tiles(blockIdx.y, gridDim.y, P.n_tiles, t_begin, t_end);
    const f2_t E2 = f2_pack(P.eps2, P.eps2);
    const f2_t NEG3 = f2_pack(-3.0f, -3.0f);
    const size_t n_pad = static_cast<size_t>(P.n_tiles) * kJTile;

    I2 I[IPT];
    int gi[IPT];
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        const int q = (blockIdx.x * IPT + u) * RB + row;
        int idx = -1;
        if (q < n_act) {
            idx = P.active[q];
            if (idx < 0 || idx >= P.n) {
                atomicOr(&P.st->flags, kFlagBadIndex);
                P.st->bad_index = q;
                idx = -1;
            }
        }
        gi[u] = idx;
        const int l = idx >= 0 ? idx : 0;
        float4 xp, vp, lp = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (SOAIN) {  // the rows from the structure-of-arrays stream, as the tiles
            const float *a = P.soa + l;
            xp = make_float4(a[0], a[n_pad], a[2 * n_pad], 0.f);
            vp = make_float4(a[4 * n_pad], a[5 * n_pad], a[6 * n_pad], 0.f);
            if (is_ds(MODE)) lp = make_float4(a[7 * n_pad], a[8 * n_pad], a[9 * n_pad], 0.f);
        } else {
            xp = P.posm[l];
            vp = P.vel[l];
            if (is_ds(MODE)) lp = P.poslo[l];
        }
        I[u].x = f2_pack(xp.x, xp.x);
        I[u].y = f2_pack(xp.y, xp.y);
        I[u].z = f2_pack(xp.z, xp.z);
        I[u].vx = f2_pack(vp.x, vp.x);
        I[u].vy = f2_pack(vp.y, vp.y);
        I[u].vz = f2_pack(vp.z, vp.z);
        if (is_ds(MODE)) {
            I[u].lx = f2_pack(lp.x, lp.x);
            I[u].ly = f2_pack(lp.y, lp.y);
            I[u].lz = f2_pack(lp.z, lp.z);
        }
    }
    float tot[IPT][7], lo[IPT][7];
    f2_t ph[IPT][7], pl[IPT][7];  // summation check: packed even/odd double-single sums
#pragma unroll
    for (int u = 0; u < IPT; ++u)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            tot[u][c] = 0.0f;
            lo[u][c] = 0.0f;
            ph[u][c] = 0ull;
            pl[u][c] = 0ull;
        }

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // group g holds tiles t_begin + g TG .. (at most TG of them)
    const int n_g = t_end > t_begin ? (t_end - t_begin + TG - 1) / TG : 0;
    auto issue = [&](int gidx, int b) {
        const int t0 = t_begin + gidx * TG;
        const size_t off = static_cast<size_t>(t0) * kJTile;
        if constexpr (SOAIN) {
            const int nt = min(TG, t_end - t0);
            if (!NB_CHECK(static_cast<size_t>(t0 + nt) * kJTile <= n_pad, P.st, 1)) return;  // no copy, the wait gives up
            mbar_arrive_expect_tx(&bar[b], nt * NA * kArrBytes);
            for (int k = 0; k < nt; ++k)
#pragma unroll
                for (int a = 0; a < NA; ++a)
                    bulk_g2s(soa[b * TG + k].a[a], P.soa + a * n_pad + off + k * kJTile, kArrBytes, &bar[b]);
        } else {
            mbar_arrive_expect_tx(&bar[b], NARR * kTileBytes);
            bulk_g2s(sj[b][0], P.posm + off, kTileBytes, &bar[b]);
            bulk_g2s(sj[b][1], P.vel + off, kTileBytes, &bar[b]);
            if (is_ds(MODE)) bulk_g2s(sj[b][NARR - 1], P.poslo + off, kTileBytes, &bar[b]);
        }
    };

    bool ok = true;
    int it_stop = 0;
    if (tid == 0 && n_g > 0 && !P.skip_first_copy) issue(0, 0);
    for (int it = 0; it < n_g; ++it) {
        const int b = it & 1;
        if (tid == 0 && it + 1 < n_g) issue(it + 1, b ^ 1);
        ok = mbar_wait_bounded(&bar[b], (it >> 1) & 1);
        if constexpr (!SOAIN) {
            if (ok) {
                for (int e = tid; e < kJTile; e += NT) {
                    const float4 pv = sj[b][0][e], vv = sj[b][1][e];
                    soa[0].a[0][e] = pv.x;
                    soa[0].a[1][e] = pv.y;
                    soa[0].a[2][e] = pv.z;
                    soa[0].a[3][e] = pv.w;
                    soa[0].a[4][e] = vv.x;
                    soa[0].a[5][e] = vv.y;
                    soa[0].a[6][e] = vv.z;
                    if (is_ds(MODE)) {
                        const float4 lv = sj[b][NARR - 1][e];
                        soa[0].a[7][e] = lv.x;
                        soa[0].a[8][e] = lv.y;
                        soa[0].a[9][e] = lv.z;
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                ok = false;
                it_stop = it;
                break;
            }
        }
        // (with SOAIN a thread whose wait gave up computes on a partial tile; the
        // barrier below stops every thread before any result is written)
        const int t0 = t_begin + it * TG;
        const int nt = min(TG, t_end - t0);
#pragma unroll 1
        for (int k = 0; k < nt; ++k) {
            const SoaTile<MODE> &T = soa[SOAIN ? b * TG + k : 0];
            const int j0 = (t0 + k) * kJTile;
            bool self_tile = false;
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                self_tile |= static_cast<unsigned>(gi[u] - j0 - sub * JL) < static_cast<unsigned>(JL);
            if constexpr (JSUB > 1) {
                if (self_tile)
                    tile_sums_x2<MODE, IPT, PF, true, JL>(T, j0, I, gi, E2, NEG3, tot, lo, sub * JL);
                else
                    tile_sums_x2<MODE, IPT, PF, false, JL>(T, j0, I, gi, E2, NEG3, tot, lo, sub * JL);
            } else if constexpr (MODE == kModeCheck) {
                if (self_tile)
                    tile_sums_x2_check<IPT, true>(T, j0, I, gi, E2, NEG3, P.opaque_zero, ph, pl);
                else
                    tile_sums_x2_check<IPT, false>(T, j0, I, gi, E2, NEG3, P.opaque_zero, ph, pl);
            } else if (self_tile) {
                tile_sums_x2<MODE, IPT, PF, true>(T, j0, I, gi, E2, NEG3, tot, lo);
            } else {
                tile_sums_x2<MODE, IPT, PF, false>(T, j0, I, gi, E2, NEG3, tot, lo);
            }
        }
        if constexpr (SOAIN) {
            if (__syncthreads_or(!ok)) {
                ok = false;
                it_stop = it;
                break;
            }
        } else {
            __syncthreads();
        }
    }

    if (!ok) {
        if (tid == 0) {
            const int b = it_stop & 1;
            mbar_wait_bounded(&bar[b], (it_stop >> 1) & 1);
            if (it_stop + 1 < n_g) mbar_wait_bounded(&bar[b ^ 1], ((it_stop + 1) >> 1) & 1);
            atomicOr(&P.st->flags, kFlagTimeout);
        }
        return;
    }

    if constexpr (JSUB > 1) {
        // the JSUB sums of each row, through shared memory (the tile buffers are
        // free: every copy issued has been waited for), added in subgroup order
        constexpr int NCS = is_ds(MODE) ? 14 : 7;
        static_assert(sizeof(soa) >= sizeof(float) * NCS * NT, "combine buffer");
        float *red = reinterpret_cast<float *>(soa);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            red[(sub * NCS + c) * RB + row] = tot[0][c];
            if (is_ds(MODE)) red[(sub * NCS + 7 + c) * RB + row] = lo[0][c];
        }
        __syncthreads();
        const int q = blockIdx.x * RB + row;
        if (sub != 0 || q >= n_act) return;
        float hs[7], ls[7];  // the JSUB sums as double-single pairs, added in subgroup order
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            hs[c] = red[c * RB + row];
            ls[c] = is_ds(MODE) ? red[(7 + c) * RB + row] : 0.0f;
#pragma unroll
            for (int g = 1; g < JSUB; ++g) {
                ds2_add(hs[c], ls[c], red[(g * NCS + c) * RB + row],
                        is_ds(MODE) ? red[(g * NCS + 7 + c) * RB + row] : 0.0f);
            }
        }
        if (gridDim.y == 1) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) r[c] = static_cast<double>(hs[c]) + static_cast<double>(ls[c]);
            double *pa = P.acc + 3 * static_cast<size_t>(q);
            double *pk = P.jerk + 3 * static_cast<size_t>(q);
            pa[0] = r[0];
            pa[1] = r[1];
            pa[2] = r[2];
            pk[0] = r[3];
            pk[1] = r[4];
            pk[2] = r[5];
            P.pot[q] = r[6];
        } else {  // a partial sum: the (hi, lo) pair, or in plain mode its rounded sum
            float *base = P.part + static_cast<size_t>(blockIdx.y) * NCS * n_act + q;
            if (!NB_CHECK(q < n_act, P.st, 2)) return;
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                if (is_ds(MODE)) {
                    base[static_cast<size_t>(c) * n_act] = hs[c];
                    base[static_cast<size_t>(7 + c) * n_act] = ls[c];
                } else {
                    base[static_cast<size_t>(c) * n_act] = __fadd_rn(hs[c], ls[c]);
                }
            }
        }
        return;
    }
    if constexpr (MODE == kModeCheck) {
        // even and odd sums into one double-single pair: TwoSum of the high
        // words, the low words and the error added (all round to nearest)
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                float he, ho, le, lo2;
                f2_unpack(ph[u][c], he, ho);
                f2_unpack(pl[u][c], le, lo2);
                tot[u][c] = he;
                lo[u][c] = __fadd_rn(le, lo2);
                fold_ds_rn(tot[u][c], lo[u][c], ho);
            }
    }
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        const int q = (blockIdx.x * IPT + u) * RB + row;
        if (q >= n_act) continue;
        if (gridDim.y == 1) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c)
                r[c] = is_ds(MODE) ? static_cast<double>(tot[u][c]) + static_cast<double>(lo[u][c])
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
            constexpr int NC = is_ds(MODE) ? 14 : 7;
            float *base = P.part + static_cast<size_t>(blockIdx.y) * NC * n_act + q;
            if (!NB_CHECK(static_cast<int>(blockIdx.y) < static_cast<int>(gridDim.y) && q < n_act, P.st, 2)) continue;
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                base[static_cast<size_t>(c) * n_act] = tot[u][c];
                if (is_ds(MODE)) base[static_cast<size_t>(7 + c) * n_act] = lo[u][c];
            }
        }
    }
}

}  // namespace nb

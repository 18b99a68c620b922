// Pieces shared by the one-launch block-step kernels (cluster_step.cu,
// grid_step.cu): the forces of a block's rows over j-particles held in shared
// memory, and the corrector of a few rows packed into as few warps as the
// lanes allow.
#pragma once

#include "ds_arith.cuh"
#include "force_x2.cuh"
#include "step_impl.cuh"

namespace nb {

// Pair terms of NG groups of 4 j (g T + sub) 4, g = g0 .. g0 + NG - 1 (NG = 0:
// ng of them), of the shared-memory copy, into the packed partials p.  ONE:
// T = 1 (consecutive groups).  A fixed NG gives the loop a compile-time trip
// count.
template <int MODE, bool SELF, int STRIDE, bool ONE, int NG>
__device__ __forceinline__ void rows_groups_x2(const float *jsm, const int stride, const int j0, const int g0,
                                               const int ng, const int T, const int sub, const I2 &I, const int gi,
                                               const f2_t E2, const f2_t NEG3, f2_t (&p)[7])
{
    constexpr bool DSW = MODE == kModeComp;
    constexpr int NA = SoaTile<MODE>::NA;
    const int n_it = NG > 0 ? NG : ng;
#pragma unroll 2
    for (int u = 0; u < n_it; ++u) {
        const int g = g0 + u;
        const int jj = ONE ? 4 * g : (g * T + sub) * 4;
        f2_t v[NA][2];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(&jsm[a * (STRIDE > 0 ? STRIDE : stride) + jj]);
            v[a][0] = q.x;
            v[a][1] = q.y;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
            pair_term_x2<MODE, SELF>(v[0][h], v[1][h], v[2][h], v[3][h], v[4][h], v[5][h], v[6][h],
                                     DSW ? v[NA - 3][h] : 0ull, DSW ? v[NA - 2][h] : 0ull, DSW ? v[NA - 1][h] : 0ull,
                                     I, E2, NEG3, j0 + jj + 2 * h, gi, p);
    }
}

// One thread's part of a row in rows_force: the groups of 4 j (g T + sub) 4,
// g < my, of the shared-memory copy, folded every 128 terms (32 groups) into
// (tot, lo): acceleration and jerk, and with POT the potential.
template <int MODE, bool SELF, int STRIDE, bool POT>
__device__ __forceinline__ void rows_sums_x2(const float *jsm, const int stride_rt, const int j0, const int my,
                                             const int T, const int sub, const I2 &I, const int gi, const f2_t E2,
                                             const f2_t NEG3, float (&tot)[7], float (&lo)[7])
{
    constexpr bool DSW = MODE == kModeComp;
    constexpr int NS = POT ? 7 : 6;
    const int stride = STRIDE > 0 ? STRIDE : stride_rt;
    for (int g0 = 0; g0 < my; g0 += 32) {  // folds of 128 terms
        f2_t p[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) p[c] = 0ull;
        // a full fold with a compile-time trip count: 2-3 % faster in plain mode; the compensated mode's
        // 128-register kernels measured slower with it (the C2 free run 1.74 -> 1.78 s)
        if (MODE == kModePlain && g0 + 32 <= my) {
            if (T == 1)
                rows_groups_x2<MODE, SELF, STRIDE, true, 32>(jsm, stride, j0, g0, 32, T, sub, I, gi, E2, NEG3, p);
            else
                rows_groups_x2<MODE, SELF, STRIDE, false, 32>(jsm, stride, j0, g0, 32, T, sub, I, gi, E2, NEG3, p);
        } else {
            rows_groups_x2<MODE, SELF, STRIDE, false, 0>(jsm, stride, j0, g0, min(32, my - g0), T, sub, I, gi, E2,
                                                         NEG3, p);
        }
#pragma unroll
        for (int c = 0; c < NS; ++c) {
            float e, o;
            f2_unpack(p[c], e, o);
            const float part = e + o;
            if (DSW)
                fold_ds_rn(tot[c], lo[c], part);
            else
                tot[c] = __fadd_rn(tot[c], part);
        }
    }
}

// Sums of the acceleration and jerk terms of Eq. (Force) for rows 0 .. cnt-1
// over the first L entries (a multiple of 4) of a copy of j-particles in shared
// memory, entry e holding particle j0 + e.  Layout: structure of arrays of
// `stride` floats each (STRIDE when it is positive, else stride_rt; x, y, z, m,
// vx, vy, vz, and the lo parts of x, y, z in
// compensated mode), or in the double-single mode four float4 arrays (x, m),
// (x_lo, m_lo), v, v_lo.  T threads per row (a power of two; NT / T rows per
// pass): thread `sub` of a row takes the groups of 4 entries 4 (g T + sub),
// g = 0, 1, ... (one entry g T + sub at a time in the double-single mode), so the
// lanes of a warp read consecutive 16-byte words.  The packed pair term is that
// of force_x2.cuh, folded every 128 terms into (hi, lo) (compensated) or an FP32
// sum (plain); the double-single mode takes ds_pair_term one j at a time.  The T
// sums of a row are added in a fixed tree: a butterfly within the warp, then warp
// by warp through wred.  load_i(r, live, I) fills the packed i-data of row r
// (row 0's when !live) and returns its particle index (-1 when !live); in the
// double-single mode load_ds(r, live, xi, vi) does the same with double-single
// i-data.  store(r, tot, lo) takes the row's sums (one thread per row): six,
// and with POT (packed modes) the potential as the seventh.  The pair j = i is
// masked in the warps holding a row whose particle lies in the entries, where
// it matters: for the potential, or for a softening too small to keep its
// zero terms finite.  Every thread of the block calls this function: it holds
// block barriers.
template <int MODE, int NT, int STRIDE = 0, bool POT = false, class LoadI, class LoadDS, class Store>
__device__ __forceinline__ void rows_force(const float *jsm, const int stride_rt, const int j0, const int L,
                                           const int cnt, const int T, const float eps2, const float eps2_lo,
                                           LoadI &&load_i, LoadDS &&load_ds, Store &&store,
                                           float (*wred)[7][2])
{
    constexpr int NS = POT ? 7 : 6;
    constexpr bool DSM = MODE == kModeDS;
    constexpr bool DSW = MODE == kModeComp || DSM;  // two-word sums
    const int stride = STRIDE > 0 ? STRIDE : stride_rt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rpp = NT / T;
    const int TW = T < 32 ? T : 32;
    const f2_t E2 = f2_pack(eps2, eps2);
    const f2_t NEG3 = f2_pack(-3.0f, -3.0f);
    for (int q0 = 0; q0 < cnt; q0 += rpp) {
        const int rr = q0 + tid / T;
        const int sub = tid % T;
        const bool live = rr < cnt;
        const bool warp_live = q0 + warp * 32 / T < cnt;  // a warp with no row skips the sums
        float tot[7], lo[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) tot[c] = lo[c] = 0.0f;
        if constexpr (DSM) {
            const float4 *sp = reinterpret_cast<const float4 *>(jsm);
            dsa::ds xi[3], vi[3];
            const int gi = load_ds(rr, live, xi, vi);
            const dsa::ds e2 = {eps2, eps2_lo};
            dsa::ds sum[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) sum[c] = {0.0f, 0.0f};
            const int my = warp_live ? (L - sub + T - 1) / T : 0;
#pragma unroll 1
            for (int g = 0; g < my; ++g) {
                const int e = g * T + sub;
                if (j0 + e == gi) continue;  // j = i contributes nothing
                dsa::ds_pair_term(sp[e], sp[stride + e], sp[2 * stride + e], sp[3 * stride + e], xi, vi, e2, sum);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                tot[c] = sum[c].h;
                lo[c] = sum[c].l;
            }
        } else {
            I2 I;
            const int gi = load_i(rr, live, I);
            const int my = warp_live ? (L / 4 - sub + T - 1) / T : 0;  // this thread's groups of 4 j
            // with eps > 0 the pair j = i adds exact zeros to the acceleration and jerk (dx = dv = 0,
            // r^2 = eps^2, m r^-3 finite for eps^2 >= 1e-12 and m < 1e20), so only the potential or a
            // tiny or zero eps needs the mask, and only in a warp with a row whose particle is among the
            // entries; the choice is the same for every lane of a warp
            const bool own_row = live && static_cast<unsigned>(gi - j0) < static_cast<unsigned>(L);
            if (__any_sync(0xffffffffu, own_row) && (POT || eps2 < 1e-12f))
                rows_sums_x2<MODE, true, STRIDE, POT>(jsm, stride, j0, my, T, sub, I, gi, E2, NEG3, tot, lo);
            else
                rows_sums_x2<MODE, false, STRIDE, POT>(jsm, stride, j0, my, T, sub, I, gi, E2, NEG3, tot, lo);
        }
        // the T sums of a row: a butterfly within the warp, then warp by warp
        for (int o = 1; o < (warp_live ? TW : 1); o <<= 1) {
#pragma unroll
            for (int c = 0; c < NS; ++c) {
                const float h2 = __shfl_xor_sync(0xffffffffu, tot[c], o);
                if (DSW) {
                    const float l2 = __shfl_xor_sync(0xffffffffu, lo[c], o);
                    ds2_add(tot[c], lo[c], h2, l2);
                } else {
                    tot[c] = __fadd_rn(tot[c], h2);
                }
            }
        }
        if (T > 32) {
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < NS; ++c) {
                    wred[warp][c][0] = tot[c];
                    wred[warp][c][1] = lo[c];
                }
            __syncthreads();
            if (sub == 0)
                for (int w = warp + 1; w < warp + T / 32; ++w)
#pragma unroll
                    for (int c = 0; c < NS; ++c) {
                        if (DSW)
                            ds2_add(tot[c], lo[c], wred[w][c][0], wred[w][c][1]);
                        else
                            tot[c] = __fadd_rn(tot[c], wred[w][c][0]);
                    }
        }
        if (live && sub == 0) store(rr, tot, lo);
        __syncthreads();  // wred and the sums of this pass are done
    }
}

// The corrector of Sect. 2 and Eq. (timestep) for rows q < cnt at tick tb: row q
// is particle idx[q], its forces fh[q][0..5] (+ fl[q][0..5], two-word sums).  Up
// to 8 rows run in warp 0 with 4 lanes per row (lanes 0-2 one component each,
// then the four norms of Eq. (timestep) one per lane: the operations of
// correct_row, in parallel); more rows one per thread q < cnt.  GB300's FP64
// unit is one per SM and takes ~19 cycles per warp instruction whatever the
// number of active lanes, so rows are packed into as few warps as possible.
// The state is read through L2 (another CTA of the launch may have written it).
// due(q, r, t) receives each row's new due tick t (from one thread per row).
template <bool DSW, class Due>
__device__ __forceinline__ void rows_correct(const State &S, const int *idx, const float (*fh)[6],
                                             const float (*fl)[6], const int cnt, const unsigned long long tb,
                                             const double tick, const double eta, const int lmin, const int lmax,
                                             DevStatus *st, Due &&due)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (cnt <= 8) {
        if (warp == 0) {
            const int q = lane >> 2, part = lane & 3, base = lane & ~3;
            const bool live = q < cnt;
            const int qq = live ? q : 0;
            const int r = idx[qq];
            double f[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] = DSW ? f2d(fh[qq][c]) + f2d(fl[qq][c]) : f2d(fh[qq][c]);
            const CorrDt d = corr_dt(static_cast<int64_t>(tb) - ld_state<true>(S.t + r), tick, lmax);
            double a2e = 0.0, a3 = 0.0;
            bool finite = true;
            if (part < 3) {
                const double fa = part == 0 ? f[0] : part == 1 ? f[1] : f[2];
                const double fk = part == 0 ? f[3] : part == 1 ? f[4] : f[5];
                double xn, vn;
                corr_dim(ld_state<true>(S.x[part] + r), ld_state<true>(S.v[part] + r), ld_state<true>(S.a[part] + r),
                         ld_state<true>(S.k[part] + r), fa, fk, d, xn, vn, a2e, a3);
                finite = isfinite(xn) && isfinite(vn) && isfinite(fa) && isfinite(fk);
                if (live) {
                    S.x[part][r] = xn;
                    S.v[part][r] = vn;
                    S.a[part][r] = fa;
                    S.k[part][r] = fk;
                }
            }
            double u[3][2];  // a^(2) and a^(3) of the row, every component
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                u[c][0] = __shfl_sync(0xffffffffu, a2e, base + c);
                u[c][1] = __shfl_sync(0xffffffffu, a3, base + c);
            }
            // all four lanes' finiteness (every lane takes part in every shuffle)
            const int f1 = __shfl_xor_sync(0xffffffffu, static_cast<int>(finite), 1);
            const int f2 = __shfl_xor_sync(0xffffffffu, static_cast<int>(finite), 2);
            finite = finite && f1 && f2;
            const int f3 = __shfl_xor_sync(0xffffffffu, static_cast<int>(finite), 1);
            finite = finite && f3;
            double w[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) w[c] = part == 0 ? f[c] : part == 1 ? f[3 + c] : part == 2 ? u[c][0] : u[c][1];
            const double nrm = norm3(w);  // |ap|, |kp|, |a^(2)|, |a^(3)| on lanes 0-3
            const double an = __shfl_sync(0xffffffffu, nrm, base), kn = __shfl_sync(0xffffffffu, nrm, base + 1);
            const double a2n = __shfl_sync(0xffffffffu, nrm, base + 2);
            const double a3n = __shfl_sync(0xffffffffu, nrm, base + 3);
            if (live && part == 0) {
                const int l_new = corr_level(an, kn, a2n, a3n, eta, lmin, lmax, ld_state<true>(S.level + r),
                                             static_cast<int64_t>(tb), finite, st);
                S.t[r] = static_cast<int64_t>(tb);
                S.level[r] = static_cast<int8_t>(l_new);
                due(q, r, tb + (1ull << (lmax - l_new)));
            }
        }
    } else if (tid < cnt) {
        double f[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) f[c] = DSW ? f2d(fh[tid][c]) + f2d(fl[tid][c]) : f2d(fh[tid][c]);
        const int r = idx[tid];
        const int l_new = correct_row<true>(S, r, f, f + 3, static_cast<int64_t>(tb), tick, eta, lmin, lmax, st);
        due(tid, r, tb + (1ull << (lmax - l_new)));
    }
}

}  // namespace nb

// Batched ensembles of independent clusters: every cluster runs the block-step
// Hermite scheme of Sect. 2 (Portegies Zwart, Belleman & Geldof 2007) with its
// own block schedule, and one batched step advances every unfinished cluster by
// one of its own block steps.
//
// A batched step is five kernels, all sized from device-side counts so the
// step can be captured once in a CUDA graph and replayed without host syncs:
//   ens_schedule  one block per cluster: t_blk = min(t_i + dt_i), ordered list
//   ens_plan      one block: prefix sums of the work items (cluster, i-block,
//                 j-range) and of the active rows; resets the work counter
//   ens_predict   every particle of a cluster with a block, to its t_blk
//   ens_force     persistent blocks take work items from an atomic counter;
//                 each item sums one i-block of one cluster over one j-range
//                 with the single-system tile code (j-tiles double-buffered
//                 through shared memory by bulk async copies)
//   ens_correct   per active row: the j-range partial sums in a fixed order,
//                 then the shared corrector and time-step rule
// With one j-range per cluster a row's sums are bit-identical to the single-
// system kernel with one j-range.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "force_x2.cuh"
#include "step_impl.cuh"

namespace nb {

struct EnsDev {
    int n_cl;
    int s_max;
    int64_t n_tot;
    const int64_t *off;    // [n_cl + 1] first row of each cluster
    const int64_t *joff;   // [n_cl] first j-stream entry (multiple of kJTile)
    const int32_t *cl_of;  // [n_tot] cluster of each row
    State S;
    JStream J;
    long long *t_blk;      // [n_cl]
    int *n_act;            // [n_cl] rows in this step's block (0: nothing to do)
    int32_t *act;          // [n_tot] block lists: cluster c's at act[off[c] ..]
    long long *item_pfx;   // [n_cl + 1] exclusive prefix of work items
    long long *row_pfx;    // [n_cl + 1] exclusive prefix of active rows
    int *nsplit;           // [n_cl] j-ranges this step
    int *tpr;              // [n_cl] tiles per j-range
    unsigned int *work;    // work-item counter of the force kernel
    int *live;             // [2]: clusters with a block this step, batched steps with work
    long long *blocks;     // [n_cl] block steps taken per cluster
    long long *pairs;      // [n_cl] pair interactions evaluated per cluster
    float *part;           // partial sums [row][s_max][7 or 14]
    DevStatus *st;
};

namespace {

constexpr int kEnsThreads = 256;

__device__ __forceinline__ unsigned long long ens_due(const State &S, int64_t i, int lmax)
{
    return static_cast<unsigned long long>(S.t[i] + (int64_t(1) << (lmax - S.level[i])));
}

// Block scheduler of Sect. 2 for one cluster per block.
__global__ void ens_schedule_kernel(const EnsDev E, long long t_end, int lmax)
{
    __shared__ unsigned long long shm[32];
    __shared__ int warp_tot[32];
    const int c = blockIdx.x;
    const int64_t lo = E.off[c], hi = E.off[c + 1];
    unsigned long long m = ~0ull;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const unsigned long long d = ens_due(E.S, i, lmax);
        m = d < m ? d : m;
    }
    m = block_reduce(m, MinOp(), shm, ~0ull);
    if (static_cast<long long>(m) > t_end) {
        if (threadIdx.x == 0) E.n_act[c] = 0;
        return;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    int count = 0;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool hit = i < hi && ens_due(E.S, i, lmax) == m;
        const unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (l == 0) warp_tot[w] = __popc(mask);
        __syncthreads();
        int before = 0, round = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) before += warp_tot[k];
            round += warp_tot[k];
        }
        if (hit) E.act[lo + count + before + __popc(mask & ((1u << l) - 1u))] = static_cast<int32_t>(i);
        count += round;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        E.n_act[c] = count;
        E.t_blk[c] = static_cast<long long>(m);
        E.blocks[c] += 1;
        E.pairs[c] += static_cast<long long>(count) * (hi - lo - 1);
    }
}

// Work items and row offsets of this step (one block, fixed summation order).
__global__ void ens_plan_kernel(const EnsDev E, int rows_per_item, int tiles_per_range)
{
    __shared__ long long s_items[1024], s_rows[1024];
    __shared__ int s_live[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (E.n_cl + nt - 1) / nt;
    const int c0 = t * chunk, c1 = min(c0 + chunk, E.n_cl);
    long long items = 0, rows = 0;
    int live = 0;
    for (int c = c0; c < c1; ++c) {
        const int na = E.n_act[c];
        int S = 0, tpr = 1;
        if (na > 0) {
            const int ntl = static_cast<int>((E.off[c + 1] - E.off[c] + kJTile - 1) / kJTile);
            S = min((ntl + tiles_per_range - 1) / tiles_per_range, E.s_max);
            tpr = (ntl + S - 1) / S;
            S = (ntl + tpr - 1) / tpr;
            items += static_cast<long long>((na + rows_per_item - 1) / rows_per_item) * S;
            rows += na;
            live += 1;
        }
        E.nsplit[c] = S;
        E.tpr[c] = tpr;
    }
    s_items[t] = items;
    s_rows[t] = rows;
    s_live[t] = live;
    __syncthreads();
    if (t == 0) {  // sequential exclusive scan over the (<= 1024) per-thread sums
        long long ai = 0, ar = 0;
        int al = 0;
        for (int k = 0; k < nt; ++k) {
            const long long xi = s_items[k], xr = s_rows[k];
            s_items[k] = ai;
            s_rows[k] = ar;
            ai += xi;
            ar += xr;
            al += s_live[k];
        }
        E.item_pfx[E.n_cl] = ai;
        E.row_pfx[E.n_cl] = ar;
        E.live[0] = al;
        if (al > 0) E.live[1] += 1;
        E.work[0] = 0u;
    }
    __syncthreads();
    long long pi = s_items[t], pr = s_rows[t];
    for (int c = c0; c < c1; ++c) {
        E.item_pfx[c] = pi;
        E.row_pfx[c] = pr;
        const int na = E.n_act[c];
        if (na > 0) {
            pi += static_cast<long long>((na + rows_per_item - 1) / rows_per_item) * E.nsplit[c];
            pr += na;
        }
    }
}

// Start of a run: every particle in the block of its cluster at t = 0.
__global__ void ens_all_active_kernel(const EnsDev E)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < E.n_tot;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        E.act[i] = static_cast<int32_t>(i);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < E.n_cl; c += gridDim.x * blockDim.x) {
        E.n_act[c] = static_cast<int>(E.off[c + 1] - E.off[c]);
        E.t_blk[c] = 0;
    }
}

__global__ void ens_predict_kernel(const EnsDev E, double tick, int comp)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < E.n_tot;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = E.cl_of[i];
        if (E.n_act[c] == 0) continue;
        const double dt = static_cast<double>(E.t_blk[c] - E.S.t[i]) * tick;
        double xp[3], vp[3];
        const PredDt pd = pred_dt(dt);
#pragma unroll
        for (int q = 0; q < 3; ++q) predict_dim(E.S.x[q][i], E.S.v[q][i], E.S.a[q][i], E.S.k[q][i], pd, xp[q], vp[q]);
        const int64_t j = E.joff[c] + (i - E.off[c]);
        // the roundings on the integer pipe (d2f_rn: the same bits as the hardware conversion)
        const float hx = d2f_rn(xp[0]), hy = d2f_rn(xp[1]), hz = d2f_rn(xp[2]);
        const float hm = d2f_rn(E.S.m[i]);
        const float hvx = d2f_rn(vp[0]), hvy = d2f_rn(vp[1]), hvz = d2f_rn(vp[2]);
        E.J.posm[j] = make_float4(hx, hy, hz, hm);
        E.J.vel[j] = make_float4(hvx, hvy, hvz, 0.f);
        float lx = 0.f, ly = 0.f, lz = 0.f;
        if (comp) {
            lx = d2f_rn(xp[0] - f2d(hx));
            ly = d2f_rn(xp[1] - f2d(hy));
            lz = d2f_rn(xp[2] - f2d(hz));
            E.J.poslo[j] = make_float4(lx, ly, lz, 0.f);
        }
        float *a = E.J.soa + j;
        const int64_t np = E.J.n_pad;
        a[0] = hx;
        a[np] = hy;
        a[2 * np] = hz;
        a[3 * np] = hm;
        a[4 * np] = hvx;
        a[5 * np] = hvy;
        a[6 * np] = hvz;
        if (comp) {
            a[7 * np] = lx;
            a[8 * np] = ly;
            a[9 * np] = lz;
        }
    }
}

// Persistent force blocks over the work list of this step.
template <int MODE, int NT, int IPT>
__global__ void __launch_bounds__(NT) ens_force_kernel(const EnsDev E, const float eps2)
{
    constexpr int NARR = (MODE == kModeComp) ? 3 : 2;
    constexpr int NC = (MODE == kModeComp) ? 14 : 7;
    constexpr int PF = FoldLen<MODE>::value;
    constexpr uint32_t kTileBytes = kJTile * sizeof(float4);
    constexpr bool kPacked = NB_PACKED != 0;
    constexpr int NA = SoaTile<MODE>::NA;
    constexpr uint32_t kArrBytes = kJTile * sizeof(float);
    // packed: tiles copied from the SoA j-stream into two SoA buffers; scalar: float4 staging
    __shared__ __align__(128) float4 sj[kPacked ? 1 : 2][kPacked ? 1 : NARR][kPacked ? 1 : kJTile];
    __shared__ __align__(128) typename std::conditional<kPacked, SoaTile<MODE>, char>::type soa[2];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ long long s_w;
    const int tid = threadIdx.x;
    const f2_t E2 = f2_pack(eps2, eps2);
    const f2_t NEG3 = f2_pack(-3.0f, -3.0f);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int64_t tile, int b) {
        const size_t off = static_cast<size_t>(tile) * kJTile;
        if constexpr (kPacked) {
            mbar_arrive_expect_tx(&bar[b], NA * kArrBytes);
#pragma unroll
            for (int a = 0; a < NA; ++a)
                bulk_g2s(soa[b].a[a], E.J.soa + a * static_cast<size_t>(E.J.n_pad) + off, kArrBytes, &bar[b]);
        } else {
            mbar_arrive_expect_tx(&bar[b], NARR * kTileBytes);
            bulk_g2s(sj[b][0], E.J.posm + off, kTileBytes, &bar[b]);
            bulk_g2s(sj[b][1], E.J.vel + off, kTileBytes, &bar[b]);
            if (MODE == kModeComp) bulk_g2s(sj[b][NARR - 1], E.J.poslo + off, kTileBytes, &bar[b]);
        }
    };
    const long long W = E.item_pfx[E.n_cl];
    unsigned int g = 0;  // tiles this block has consumed: buffer g & 1, phase (g >> 1) & 1
    for (;;) {
        if (tid == 0) s_w = static_cast<long long>(atomicAdd(E.work, 1u));
        __syncthreads();
        const long long w = s_w;
        __syncthreads();
        if (w >= W) break;
        int lo = 0, hi = E.n_cl;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (E.item_pfx[mid] <= w) lo = mid;
            else hi = mid;
        }
        const int c = lo;
        const long long local = w - E.item_pfx[c];
        const int S = E.nsplit[c];
        const int blk = static_cast<int>(local / S), s = static_cast<int>(local % S);
        const int nact = E.n_act[c];
        const int64_t roff = E.off[c], jo = E.joff[c];
        const int ntl = static_cast<int>((E.off[c + 1] - roff + kJTile - 1) / kJTile);
        const int t_begin = s * E.tpr[c];
        const int t_end = min(t_begin + E.tpr[c], ntl);

        float4 xi[IPT], vi[IPT], li[IPT];
        int gi[IPT];
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int q = (blk * IPT + u) * NT + tid;
            int jidx = -1;
            if (q < nact) {
                const int64_t i = E.act[roff + q];
                if (i < roff || i >= E.off[c + 1]) {
                    atomicOr(&E.st->flags, kFlagBadIndex);
                    E.st->bad_index = q;
                } else {
                    jidx = static_cast<int>(jo + (i - roff));
                }
            }
            gi[u] = jidx;
            const int64_t l = jidx >= 0 ? jidx : jo;
            xi[u] = E.J.posm[l];
            vi[u] = E.J.vel[l];
            li[u] = (MODE == kModeComp) ? E.J.poslo[l] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        I2 I[IPT];
        if constexpr (kPacked) {
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                I[u].x = f2_pack(xi[u].x, xi[u].x);
                I[u].y = f2_pack(xi[u].y, xi[u].y);
                I[u].z = f2_pack(xi[u].z, xi[u].z);
                I[u].vx = f2_pack(vi[u].x, vi[u].x);
                I[u].vy = f2_pack(vi[u].y, vi[u].y);
                I[u].vz = f2_pack(vi[u].z, vi[u].z);
                I[u].lx = f2_pack(li[u].x, li[u].x);
                I[u].ly = f2_pack(li[u].y, li[u].y);
                I[u].lz = f2_pack(li[u].z, li[u].z);
            }
        }
        float tot[IPT][7], lo_[IPT][7];
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                tot[u][k] = 0.0f;
                lo_[u][k] = 0.0f;
            }
        const int64_t jt0 = jo / kJTile;
        bool ok = true;
        if (tid == 0 && t_begin < t_end) issue(jt0 + t_begin, g & 1);
        for (int t = t_begin; t < t_end; ++t, ++g) {
            const int b = g & 1;
            if (tid == 0 && t + 1 < t_end) issue(jt0 + t + 1, b ^ 1);
            ok = mbar_wait_bounded(&bar[b], (g >> 1) & 1);
            if constexpr (kPacked) {
                // the single-system packed kernel's tile loop: SoA tile, packed pairs, one barrier
                // (a thread whose wait gave up computes on a partial tile; the barrier stops all
                // threads before anything is written)
                const int j0 = static_cast<int>(jo) + t * kJTile;
                bool self_tile = false;
#pragma unroll
                for (int u = 0; u < IPT; ++u)
                    self_tile |= static_cast<unsigned>(gi[u] - j0) < static_cast<unsigned>(kJTile);
                if (self_tile)
                    tile_sums_x2<MODE, IPT, PF, true>(soa[b], j0, I, gi, E2, NEG3, tot, lo_);
                else
                    tile_sums_x2<MODE, IPT, PF, false>(soa[b], j0, I, gi, E2, NEG3, tot, lo_);
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) {
                        mbar_wait_bounded(&bar[b], (g >> 1) & 1);
                        if (t + 1 < t_end) mbar_wait_bounded(&bar[b ^ 1], ((g + 1) >> 1) & 1);
                        atomicOr(&E.st->flags, kFlagTimeout);
                    }
                    return;
                }
                continue;
            }
            if (ok) {
                const int j0 = static_cast<int>(jo) + t * kJTile;
                bool self_tile = false;
#pragma unroll
                for (int u = 0; u < IPT; ++u)
                    self_tile |= static_cast<unsigned>(gi[u] - j0) < static_cast<unsigned>(kJTile);
                if (self_tile)
                    tile_sums<MODE, IPT, PF, true>(sj[b][0], sj[b][1], sj[b][NARR - 1], j0, xi, vi, li, gi, eps2, tot, lo_);
                else
                    tile_sums<MODE, IPT, PF, false>(sj[b][0], sj[b][1], sj[b][NARR - 1], j0, xi, vi, li, gi, eps2, tot, lo_);
            }
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    mbar_wait_bounded(&bar[b], (g >> 1) & 1);
                    if (t + 1 < t_end) mbar_wait_bounded(&bar[b ^ 1], ((g + 1) >> 1) & 1);
                    atomicOr(&E.st->flags, kFlagTimeout);
                }
                return;
            }
        }
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int q = (blk * IPT + u) * NT + tid;
            if (q >= nact) continue;
            float *base = E.part + ((static_cast<size_t>(E.row_pfx[c] + q) * E.s_max) + s) * NC;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                base[k] = tot[u][k];
                if (MODE == kModeComp) base[7 + k] = lo_[u][k];
            }
        }
    }
}

// Sums a row's j-range partials in ascending range order, as double-single
// pairs on the FP32 pipe (ds2_add; GB300's FP64 unit is narrow), then hi + lo in
// FP64.  With one range the result is the range's hi + lo, as the
// single-system kernel writes it.
template <int NC>
__device__ __forceinline__ void ens_row_sums(const EnsDev &E, long long r, int S, double (&f)[7])
{
    float h[7], l[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) h[k] = l[k] = 0.0f;
    for (int s = 0; s < S; ++s) {
        const float *base = E.part + ((static_cast<size_t>(r) * E.s_max) + s) * NC;
#pragma unroll
        for (int k = 0; k < 7; ++k) ds2_add(h[k], l[k], base[k], NC == 14 ? base[7 + k] : 0.0f);
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = static_cast<double>(h[k]) + static_cast<double>(l[k]);
}

__device__ __forceinline__ int ens_row_cluster(const EnsDev &E, long long r)
{
    int lo = 0, hi = E.n_cl;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (E.row_pfx[mid] <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int NC>
__global__ void ens_correct_kernel(const EnsDev E, double tick, double eta, int lmin, int lmax)
{
    const long long R = E.row_pfx[E.n_cl];
    for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = ens_row_cluster(E, r);
        const int64_t i = E.act[E.off[c] + (r - E.row_pfx[c])];
        double f[7];
        ens_row_sums<NC>(E, r, E.nsplit[c], f);
        correct_row(E.S, i, f, f + 3, E.t_blk[c], tick, eta, lmin, lmax, E.st);
    }
}

// t = 0: a, k from the force on every particle, first levels from Eq. (initTimestep).
template <int NC>
__global__ void ens_init_kernel(const EnsDev E, double eta_init, int lmin, int lmax)
{
    const long long R = E.row_pfx[E.n_cl];
    for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = ens_row_cluster(E, r);
        const int64_t i = E.act[E.off[c] + (r - E.row_pfx[c])];
        double f[7];
        ens_row_sums<NC>(E, r, E.nsplit[c], f);
        bool finite = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            E.S.a[q][i] = f[q];
            E.S.k[q][i] = f[3 + q];
            finite = finite && isfinite(f[q]) && isfinite(f[3 + q]);
        }
        const double kn = norm3(f + 3);
        const double dt0 = kn == 0.0 ? static_cast<double>(INFINITY) : eta_init * norm3(f) / kn;
        bool clamped = false;
        int L = level_of(dt0, lmin, lmax, &clamped);
        if (!finite || L < 0) {
            L = lmax;
            atomicOr(&E.st->flags, kFlagNonfinite);
            atomicAdd(&E.st->nonfinite, 1ull);
        }
        if (clamped) {
            atomicOr(&E.st->flags, kFlagDtMin);
            atomicAdd(&E.st->below_min, 1ull);
        }
        E.S.t[i] = 0;
        E.S.level[i] = static_cast<int8_t>(L);
    }
}

// phi_i over the particle's own cluster (FP64, ascending j), then per-cluster sums.
__global__ void ens_phi_kernel(const EnsDev E, double eps2, double *__restrict__ phi)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < E.n_tot;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = E.cl_of[i];
        const double xi = E.S.x[0][i], yi = E.S.x[1][i], zi = E.S.x[2][i];
        double p = 0.0;
        for (int64_t j = E.off[c]; j < E.off[c + 1]; ++j) {
            if (j == i) continue;
            const double dx = E.S.x[0][j] - xi, dy = E.S.x[1][j] - yi, dz = E.S.x[2][j] - zi;
            const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(eps2, __dmul_rn(dx, dx)), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz));
            p = __dsub_rn(p, __ddiv_rn(E.S.m[j], __dsqrt_rn(r2)));
        }
        phi[i] = p;
    }
}

__global__ void ens_energy_sum_kernel(const EnsDev E, const double *__restrict__ phi, double *out)
{
    __shared__ double sk[kEnsThreads], sp[kEnsThreads];
    const int c = blockIdx.x;
    double k = 0.0, p = 0.0;
    for (int64_t i = E.off[c] + threadIdx.x; i < E.off[c + 1]; i += blockDim.x) {
        const double vx = E.S.v[0][i], vy = E.S.v[1][i], vz = E.S.v[2][i];
        k += 0.5 * E.S.m[i] * (vx * vx + vy * vy + vz * vz);
        p += 0.5 * E.S.m[i] * phi[i];
    }
    sk[threadIdx.x] = k;
    sp[threadIdx.x] = p;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (static_cast<int>(threadIdx.x) < s) {
            sk[threadIdx.x] += sk[threadIdx.x + s];
            sp[threadIdx.x] += sp[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * c] = sk[0];
        out[2 * c + 1] = sp[0];
    }
}

__global__ void ens_time_range_kernel(const EnsDev E, long long *out)
{
    // out[2c] = min t, out[2c+1] = max t of cluster c (one block per cluster)
    __shared__ unsigned long long sh[32];
    const int c = blockIdx.x;
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t i = E.off[c] + threadIdx.x; i < E.off[c + 1]; i += blockDim.x) {
        const unsigned long long t = static_cast<unsigned long long>(E.S.t[i]);
        lo = t < lo ? t : lo;
        hi = t > hi ? t : hi;
    }
    lo = block_reduce(lo, MinOp(), sh, ~0ull);
    hi = block_reduce(hi, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0) {
        out[2 * c] = static_cast<long long>(lo);
        out[2 * c + 1] = static_cast<long long>(hi);
    }
}

__global__ void ens_pad_kernel(const EnsDev E)
{
    // padding entries of every cluster's j-segment: massless, far away
    for (int c = blockIdx.x; c < E.n_cl; c += gridDim.x) {
        const int64_t n_c = E.off[c + 1] - E.off[c];
        const int64_t pad = (n_c + kJTile - 1) / kJTile * kJTile;
        for (int64_t k = n_c + threadIdx.x; k < pad; k += blockDim.x) {
            const int64_t j = E.joff[c] + k;
            E.J.posm[j] = make_float4(kPadPosition, kPadPosition, kPadPosition, 0.f);
            E.J.vel[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            E.J.poslo[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int a = 0; a < kSoaArrays; ++a) E.J.soa[a * E.J.n_pad + j] = a < 3 ? kPadPosition : 0.f;
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
using EnsForceFn = void (*)(EnsDev, float);

template <int MODE, int NT, int IPT>
void ens_force_instance(const EnsDev &E, float eps2, int grid, cudaStream_t s)
{
    ens_force_kernel<MODE, NT, IPT><<<grid, NT, 0, s>>>(E, eps2);
}

// Resident blocks per SM of one force instance (queried once, before any
// graph capture, and cached).
template <int MODE, int NT, int IPT>
int ens_force_occupancy()
{
    static const int cached = [] {  // a function-local static: thread-safe initialisation
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ens_force_kernel<MODE, NT, IPT>, NT, 0);
        return b;
    }();
    return cached;
}

// Launch shapes the ensemble can use (the tuner picks among them).
struct EnsShape {
    int threads, ipt;
};
constexpr EnsShape kEnsShapes[] = {{32, 1}, {64, 1}, {64, 2}, {128, 1}, {128, 2}};

void ens_prefetch_occupancy()
{
    ens_force_occupancy<kModePlain, 32, 1>();
    ens_force_occupancy<kModePlain, 64, 1>();
    ens_force_occupancy<kModePlain, 64, 2>();
    ens_force_occupancy<kModePlain, 128, 1>();
    ens_force_occupancy<kModePlain, 128, 2>();
    ens_force_occupancy<kModeComp, 32, 1>();
    ens_force_occupancy<kModeComp, 64, 1>();
    ens_force_occupancy<kModeComp, 64, 2>();
    ens_force_occupancy<kModeComp, 128, 1>();
    ens_force_occupancy<kModeComp, 128, 2>();
}

cudaError_t ens_force_launch(int mode, int threads, int ipt, const EnsDev &E, float eps2, int sm_count,
                             cudaStream_t s, int64_t *launches)
{
#define NB_ENS(M, T, I)                                                    \
    if (mode == M && threads == T && ipt == I) {                            \
        const int grid = sm_count * std::max(1, ens_force_occupancy<M, T, I>()); \
        ens_force_instance<M, T, I>(E, eps2, grid, s);                      \
        ++*launches;                                                        \
        return cudaGetLastError();                                          \
    }
    NB_ENS(kModePlain, 32, 1)
    NB_ENS(kModePlain, 64, 1)
    NB_ENS(kModePlain, 64, 2)
    NB_ENS(kModePlain, 128, 1)
    NB_ENS(kModePlain, 128, 2)
    NB_ENS(kModeComp, 32, 1)
    NB_ENS(kModeComp, 64, 1)
    NB_ENS(kModeComp, 64, 2)
    NB_ENS(kModeComp, 128, 1)
    NB_ENS(kModeComp, 128, 2)
#undef NB_ENS
    return cudaErrorInvalidConfiguration;
}

}  // namespace nb

// ======================================================================= C ABI
using namespace nb;

struct nbody_ens {
    int n_cl = 0;
    int64_t n_tot = 0, j_tot = 0;
    double eps2 = 0.0;
    nbody_params p{};
    cudaStream_t s = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int s_max = 8;
    int threads = 64, ipt = 1, tiles_per_range = 4;
    std::vector<int64_t> off_h;
    // device memory
    double *state = nullptr;
    int64_t *t = nullptr;
    int8_t *level = nullptr;
    float4 *jbuf = nullptr;
    int64_t *off = nullptr, *joff = nullptr;
    int32_t *cl_of = nullptr, *act = nullptr;
    long long *t_blk = nullptr, *item_pfx = nullptr, *row_pfx = nullptr, *blocks = nullptr, *pairs = nullptr;
    int *n_act = nullptr, *nsplit = nullptr, *tpr = nullptr, *live = nullptr;
    unsigned int *work = nullptr;
    float *part = nullptr;
    DevStatus *st = nullptr;
    double *phi = nullptr, *e_out = nullptr, *stage = nullptr;
    long long *trange = nullptr;
    // pinned host mirrors
    int *live_h = nullptr;
    DevStatus *st_h = nullptr;
    EnsDev E{};
    cudaGraphExec_t graph = nullptr;
    long long graph_t_end = -1;
    int graph_shape[3] = {0, 0, 0};
    int64_t kernel_launches = 0;
};

namespace {

int efail(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return report_error(code, buf);
}

int ecuda(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return efail(e == cudaErrorMemoryAllocation ? NBODY_ENOMEM : NBODY_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define NB_ECUDA(call, what)                               \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return ecuda(e_, what);     \
    } while (0)

void ens_release(nbody_ens *e)
{
    if (e->graph) cudaGraphExecDestroy(e->graph);
    void *dev[] = {e->state, e->t, e->level, e->jbuf, e->off, e->joff, e->cl_of, e->act, e->t_blk, e->item_pfx,
                   e->row_pfx, e->blocks, e->pairs, e->n_act, e->nsplit, e->tpr, e->live, e->work, e->part, e->st, e->phi,
                   e->e_out, e->stage, e->trange};
    for (void *d : dev)
        if (d) cudaFree(d);
    if (e->live_h) cudaFreeHost(e->live_h);
    if (e->st_h) cudaFreeHost(e->st_h);
    if (e->own_stream && e->s) cudaStreamDestroy(e->s);
    delete e;
}

int ens_check(nbody_ens *e)
{
    NB_ECUDA(cudaMemcpyAsync(e->st_h, e->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, e->s), "status read-back");
    NB_ECUDA(cudaStreamSynchronize(e->s), "stream synchronise");
    const unsigned f = e->st_h->flags;
    if (!f) return NBODY_OK;
    NB_ECUDA(cudaMemsetAsync(&e->st->flags, 0, sizeof(unsigned), e->s), "status clear");
    if (f & kFlagTimeout) return efail(NBODY_ETIMEOUT, "ensemble: a bounded tile wait gave up");
    if (f & kFlagBadIndex) return efail(NBODY_EINVAL, "ensemble: block list index outside its cluster");
    if (f & kFlagNonfinite) return efail(NBODY_ENONFINITE, "ensemble: non-finite force or state");
    if ((f & kFlagDtMin) && e->p.strict) return efail(NBODY_EDTMIN, "ensemble: time step below dt_min");
    return NBODY_OK;
}

// Enqueues one batched step (schedule, plan, predict, force, correct).
int ens_enqueue_step(nbody_ens *e, long long t_end_tick)
{
    const int lmax = e->p.lmax;
    const double tick = std::ldexp(1.0, -lmax);
    const int rows = e->threads * e->ipt;
    ens_schedule_kernel<<<e->n_cl, kEnsThreads, 0, e->s>>>(e->E, t_end_tick, lmax);
    ens_plan_kernel<<<1, 1024, 0, e->s>>>(e->E, rows, e->tiles_per_range);
    const int pg = static_cast<int>(std::min<int64_t>((e->n_tot + 255) / 256, e->sm_count * 16));
    ens_predict_kernel<<<pg, 256, 0, e->s>>>(e->E, tick, e->p.mode == kModeComp);
    NB_ECUDA(cudaGetLastError(), "ensemble step launch");
    NB_ECUDA(ens_force_launch(e->p.mode, e->threads, e->ipt, e->E, static_cast<float>(e->eps2), e->sm_count, e->s,
                              &e->kernel_launches),
             "ensemble force launch");
    if (e->p.mode == kModeComp)
        ens_correct_kernel<14><<<pg, 256, 0, e->s>>>(e->E, tick, e->p.eta, e->p.lmin, lmax);
    else
        ens_correct_kernel<7><<<pg, 256, 0, e->s>>>(e->E, tick, e->p.eta, e->p.lmin, lmax);
    NB_ECUDA(cudaGetLastError(), "ensemble step launch");
    e->kernel_launches += 4;
    return NBODY_OK;
}

int ens_ticks(const nbody_ens *e, double t, long long *out)
{
    const double tt = std::ldexp(t, e->p.lmax);
    if (!std::isfinite(tt) || tt < 0.0 || tt > 4.0e18 || tt != std::floor(tt))
        return efail(NBODY_EINVAL, "time %.17g is not a multiple of dt_min", t);
    *out = static_cast<long long>(tt);
    const long long dtmax = 1ll << (e->p.lmax - e->p.lmin);
    if (*out % dtmax != 0) return efail(NBODY_EINVAL, "end time must be a multiple of dt_max");
    return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_ens_init(nbody_ens **out, int64_t n_clusters, const int64_t *sizes, const double *m, const double *x,
                   const double *v, double eps2, const nbody_params *p)
{
    report_error(NBODY_OK, "");
    if (!out || !sizes || !m || !x || !v) return efail(NBODY_EINVAL, "nbody_ens_init: null pointer argument");
    *out = nullptr;
    if (n_clusters < 1 || n_clusters > (1 << 20)) return efail(NBODY_EINVAL, "nbody_ens_init: bad cluster count");
    nbody_params prm;
    if (p) prm = *p;
    else nbody_default_params(&prm);
    if (prm.eta_init <= 0.0) prm.eta_init = prm.eta;
    if (!(prm.eta > 0.0) || prm.lmin < 0 || prm.lmax > 40 || prm.lmin > prm.lmax ||
        (prm.mode != NBODY_MODE_PLAIN && prm.mode != NBODY_MODE_COMP) || !(eps2 >= 0.0))
        return efail(NBODY_EINVAL, "nbody_ens_init: bad parameters");
    std::vector<int64_t> sz(static_cast<size_t>(n_clusters));
    if (cudaMemcpy(sz.data(), sizes, sz.size() * sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess)
        return ecuda(cudaGetLastError(), "sizes read");
    std::vector<int64_t> off(sz.size() + 1, 0), joff(sz.size(), 0);
    int64_t jt = 0;
    for (size_t c = 0; c < sz.size(); ++c) {
        if (sz[c] < 1) return efail(NBODY_EINVAL, "nbody_ens_init: cluster %zu is empty", c);
        off[c + 1] = off[c] + sz[c];
        joff[c] = jt;
        jt += (sz[c] + kJTile - 1) / kJTile * kJTile;
    }
    const int64_t n = off.back();
    if (n > 2147483647LL || jt > 2147483647LL) return efail(NBODY_EINVAL, "nbody_ens_init: too many particles");

    const int sh_t = prm.j_tile ? prm.j_tile : 64, sh_i = prm.i_block ? prm.i_block : 1;
    const int sh_p = prm.j_split > 0 ? prm.j_split : 4;
    bool shape_ok = false;
    for (const EnsShape &sh : kEnsShapes) shape_ok |= sh.threads == sh_t && sh.ipt == sh_i;
    if (!shape_ok) return efail(NBODY_EINVAL, "nbody_ens_init: unsupported force shape %d x %d", sh_t, sh_i);
    nbody_ens *e = new (std::nothrow) nbody_ens;
    if (!e) return efail(NBODY_ENOMEM, "nbody_ens_init: host allocation failed");
    e->threads = sh_t;
    e->ipt = sh_i;
    e->tiles_per_range = sh_p;
    e->n_cl = static_cast<int>(n_clusters);
    e->n_tot = n;
    e->j_tot = jt;
    e->eps2 = eps2;
    e->p = prm;
    e->off_h = off;
    auto bail = [&](int code) {
        ens_release(e);
        return code;
    };
#define NB_EI(call, what)                                            \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return bail(ecuda(e_, what));         \
    } while (0)
    if (prm.stream) {
        e->s = static_cast<cudaStream_t>(prm.stream);
    } else {
        NB_EI(cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking), "stream create");
        e->own_stream = true;
    }
    int dev = 0;
    NB_EI(cudaGetDevice(&dev), "cudaGetDevice");
    NB_EI(cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const size_t nd = static_cast<size_t>(n), nc = static_cast<size_t>(n_clusters);
    const size_t NC = prm.mode == NBODY_MODE_COMP ? 14 : 7;
    NB_EI(cudaMalloc(&e->state, 13 * nd * sizeof(double)), "state allocation");
    NB_EI(cudaMalloc(&e->t, nd * sizeof(int64_t)), "time allocation");
    NB_EI(cudaMalloc(&e->level, nd), "level allocation");
    const size_t jbytes = static_cast<size_t>(jt) * (3 * sizeof(float4) + kSoaArrays * sizeof(float));
    NB_EI(cudaMalloc(&e->jbuf, jbytes), "j-stream allocation");
    NB_EI(cudaMalloc(&e->off, (nc + 1) * sizeof(int64_t)), "offsets");
    NB_EI(cudaMalloc(&e->joff, nc * sizeof(int64_t)), "offsets");
    NB_EI(cudaMalloc(&e->cl_of, nd * sizeof(int32_t)), "cluster map");
    NB_EI(cudaMalloc(&e->act, nd * sizeof(int32_t)), "block lists");
    NB_EI(cudaMalloc(&e->t_blk, nc * sizeof(long long)), "cluster times");
    NB_EI(cudaMalloc(&e->item_pfx, (nc + 1) * sizeof(long long)), "plan");
    NB_EI(cudaMalloc(&e->row_pfx, (nc + 1) * sizeof(long long)), "plan");
    NB_EI(cudaMalloc(&e->blocks, nc * sizeof(long long)), "block counters");
    NB_EI(cudaMalloc(&e->pairs, nc * sizeof(long long)), "pair counters");
    NB_EI(cudaMalloc(&e->n_act, nc * sizeof(int)), "plan");
    NB_EI(cudaMalloc(&e->nsplit, nc * sizeof(int)), "plan");
    NB_EI(cudaMalloc(&e->tpr, nc * sizeof(int)), "plan");
    NB_EI(cudaMalloc(&e->live, 2 * sizeof(int)), "plan");
    NB_EI(cudaMalloc(&e->work, sizeof(unsigned int)), "work counter");
    NB_EI(cudaMalloc(&e->part, nd * e->s_max * NC * sizeof(float)), "partial sums");
    NB_EI(cudaMalloc(&e->st, sizeof(DevStatus)), "status");
    NB_EI(cudaMalloc(&e->phi, nd * sizeof(double)), "energy scratch");
    NB_EI(cudaMalloc(&e->e_out, 2 * nc * sizeof(double)), "energy");
    NB_EI(cudaMalloc(&e->stage, 3 * nd * sizeof(double)), "staging");
    NB_EI(cudaMalloc(&e->trange, 2 * nc * sizeof(long long)), "time range");
    NB_EI(cudaMallocHost(&e->live_h, 2 * sizeof(int)), "pinned");
    NB_EI(cudaMallocHost(&e->st_h, sizeof(DevStatus)), "pinned");
    std::vector<int32_t> clmap(nd);
    for (size_t c = 0; c < nc; ++c)
        for (int64_t i = off[c]; i < off[c + 1]; ++i) clmap[static_cast<size_t>(i)] = static_cast<int32_t>(c);

    EnsDev &E = e->E;
    E.n_cl = e->n_cl;
    E.s_max = e->s_max;
    E.n_tot = n;
    E.off = e->off;
    E.joff = e->joff;
    E.cl_of = e->cl_of;
    E.S.n = n;
    E.S.m = e->state;
    for (int q = 0; q < 3; ++q) {
        E.S.x[q] = e->state + (1 + q) * nd;
        E.S.v[q] = e->state + (4 + q) * nd;
        E.S.a[q] = e->state + (7 + q) * nd;
        E.S.k[q] = e->state + (10 + q) * nd;
    }
    E.S.t = e->t;
    E.S.level = e->level;
    E.J.posm = e->jbuf;
    E.J.vel = e->jbuf + jt;
    E.J.poslo = e->jbuf + 2 * jt;
    E.J.soa = reinterpret_cast<float *>(e->jbuf + 3 * jt);
    E.J.n_pad = jt;
    E.t_blk = e->t_blk;
    E.n_act = e->n_act;
    E.act = e->act;
    E.item_pfx = e->item_pfx;
    E.row_pfx = e->row_pfx;
    E.nsplit = e->nsplit;
    E.tpr = e->tpr;
    E.work = e->work;
    E.live = e->live;
    E.blocks = e->blocks;
    E.pairs = e->pairs;
    E.part = e->part;
    E.st = e->st;

    cudaStream_t s = e->s;
    NB_EI(cudaMemcpyAsync(e->off, off.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s), "upload");
    NB_EI(cudaMemcpyAsync(e->joff, joff.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice, s), "upload");
    NB_EI(cudaMemcpyAsync(e->cl_of, clmap.data(), nd * sizeof(int32_t), cudaMemcpyHostToDevice, s), "upload");
    NB_EI(cudaMemsetAsync(e->jbuf, 0, jbytes, s), "memset");
    NB_EI(cudaMemsetAsync(e->state + 7 * nd, 0, 6 * nd * sizeof(double), s), "memset");
    NB_EI(cudaMemsetAsync(e->t, 0, nd * sizeof(int64_t), s), "memset");
    NB_EI(cudaMemsetAsync(e->blocks, 0, nc * sizeof(long long), s), "memset");
    NB_EI(cudaMemsetAsync(e->live, 0, 2 * sizeof(int), s), "memset");
    NB_EI(cudaMemsetAsync(e->st, 0, sizeof(DevStatus), s), "memset");
    NB_EI(cudaMemcpyAsync(e->state, m, nd * sizeof(double), cudaMemcpyDefault, s), "mass upload");
    NB_EI(cudaMemcpyAsync(e->stage, x, 3 * nd * sizeof(double), cudaMemcpyDefault, s), "position upload");
    NB_EI(aos_to_soa_launch(e->stage, E.S.x[0], E.S.x[1], E.S.x[2], n, s, &e->kernel_launches), "layout");
    NB_EI(cudaMemcpyAsync(e->stage, v, 3 * nd * sizeof(double), cudaMemcpyDefault, s), "velocity upload");
    NB_EI(aos_to_soa_launch(e->stage, E.S.v[0], E.S.v[1], E.S.v[2], n, s, &e->kernel_launches), "layout");
    ens_prefetch_occupancy();
    ens_pad_kernel<<<std::min(e->n_cl, 1024), 256, 0, s>>>(E);
    // t = 0: everything active, full force per cluster, first levels
    const int pg = static_cast<int>(std::min<int64_t>((n + 255) / 256, e->sm_count * 16));
    ens_all_active_kernel<<<pg, 256, 0, s>>>(E);
    ens_plan_kernel<<<1, 1024, 0, s>>>(E, e->threads * e->ipt, e->tiles_per_range);
    ens_predict_kernel<<<pg, 256, 0, s>>>(E, std::ldexp(1.0, -prm.lmax), prm.mode == NBODY_MODE_COMP);
    NB_EI(cudaGetLastError(), "init launch");
    NB_EI(ens_force_launch(prm.mode, e->threads, e->ipt, E, static_cast<float>(eps2), e->sm_count, s,
                           &e->kernel_launches),
          "init force");
    if (prm.mode == NBODY_MODE_COMP)
        ens_init_kernel<14><<<pg, 256, 0, s>>>(E, prm.eta_init, prm.lmin, prm.lmax);
    else
        ens_init_kernel<7><<<pg, 256, 0, s>>>(E, prm.eta_init, prm.lmin, prm.lmax);
    NB_EI(cudaGetLastError(), "init launch");
    NB_EI(cudaMemsetAsync(e->blocks, 0, nc * sizeof(long long), s), "memset");
    NB_EI(cudaMemsetAsync(e->pairs, 0, nc * sizeof(long long), s), "memset");
    NB_EI(cudaMemsetAsync(e->live, 0, 2 * sizeof(int), s), "memset");
    e->kernel_launches += 5;
    int r = ens_check(e);
    if (r == NBODY_EDTMIN) r = NBODY_OK;
    if (r != NBODY_OK) return bail(r);
#undef NB_EI
    *out = e;
    return NBODY_OK;
}

int nbody_ens_set_shape(nbody_ens *e, int threads, int i_block, int tiles_per_range)
{
    if (!e) return efail(NBODY_EINVAL, "nbody_ens_set_shape: null ensemble");
    bool known = false;
    for (const EnsShape &sh : kEnsShapes) known |= sh.threads == threads && sh.ipt == i_block;
    if (!known || tiles_per_range < 1) return efail(NBODY_EINVAL, "nbody_ens_set_shape: unsupported shape");
    e->threads = threads;
    e->ipt = i_block;
    e->tiles_per_range = tiles_per_range;
    return NBODY_OK;
}

int nbody_ens_step(nbody_ens *e, double t_end, int64_t *n_live)
{
    if (!e) return efail(NBODY_EINVAL, "nbody_ens_step: null ensemble");
    long long tend;
    int r = ens_ticks(e, t_end, &tend);
    if (r != NBODY_OK) return r;
    r = ens_enqueue_step(e, tend);
    if (r != NBODY_OK) return r;
    NB_ECUDA(cudaMemcpyAsync(e->live_h, e->live, 2 * sizeof(int), cudaMemcpyDeviceToHost, e->s), "live read-back");
    r = ens_check(e);
    if (r != NBODY_OK) return r;
    if (n_live) *n_live = e->live_h[0];
    return NBODY_OK;
}

int nbody_ens_run(nbody_ens *e, double t_end, int64_t check_every, int64_t *n_steps)
{
    if (!e) return efail(NBODY_EINVAL, "nbody_ens_run: null ensemble");
    long long tend;
    int r = ens_ticks(e, t_end, &tend);
    if (r != NBODY_OK) return r;
    if (check_every <= 0) check_every = 16;
    const bool stale = !e->graph || e->graph_t_end != tend || e->graph_shape[0] != e->threads ||
                       e->graph_shape[1] != e->ipt || e->graph_shape[2] != e->tiles_per_range;
    if (stale) {
        if (e->graph) {
            cudaGraphExecDestroy(e->graph);
            e->graph = nullptr;
        }
        cudaGraph_t g;
        NB_ECUDA(cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal), "graph capture begin");
        r = ens_enqueue_step(e, tend);
        const cudaError_t ec = cudaMemcpyAsync(e->live_h, e->live, 2 * sizeof(int), cudaMemcpyDeviceToHost, e->s);
        cudaError_t ee = cudaStreamEndCapture(e->s, &g);
        if (r != NBODY_OK) return r;
        if (ec != cudaSuccess) return ecuda(ec, "graph capture copy");
        if (ee != cudaSuccess) return ecuda(ee, "graph capture end");
        ee = cudaGraphInstantiate(&e->graph, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) return ecuda(ee, "graph instantiate");
        e->graph_t_end = tend;
        e->graph_shape[0] = e->threads;
        e->graph_shape[1] = e->ipt;
        e->graph_shape[2] = e->tiles_per_range;
    }
    NB_ECUDA(cudaMemsetAsync(e->live + 1, 0, sizeof(int), e->s), "memset");
    for (;;) {
        for (int64_t k = 0; k < check_every; ++k) {
            NB_ECUDA(cudaGraphLaunch(e->graph, e->s), "graph launch");
            e->kernel_launches += 5;
        }
        r = ens_check(e);
        if (r != NBODY_OK) return r;
        if (e->live_h[0] == 0) break;
    }
    if (n_steps) *n_steps = e->live_h[1];
    return NBODY_OK;
}

int nbody_ens_tune(nbody_ens *e, double t_end, int steps, int *threads, int *i_block, int *tiles_per_range,
                   double *best_ms)
{
    if (!e) return efail(NBODY_EINVAL, "nbody_ens_tune: null ensemble");
    long long tend;
    int r = ens_ticks(e, t_end, &tend);
    if (r != NBODY_OK) return r;
    if (steps < 1) steps = 4;
    const size_t nd = static_cast<size_t>(e->n_tot), nc = static_cast<size_t>(e->n_cl);
    const size_t bytes = 13 * nd * sizeof(double) + nd * sizeof(int64_t) + nd + 2 * nc * sizeof(long long);
    char *save = nullptr;
    NB_ECUDA(cudaMalloc(&save, bytes), "tuner save buffer");
    auto copy_state = [&](bool to_save) -> cudaError_t {
        char *p = save;
        const void *src[5] = {e->state, e->t, e->level, e->blocks, e->pairs};
        const size_t len[5] = {13 * nd * sizeof(double), nd * sizeof(int64_t), nd, nc * sizeof(long long),
                               nc * sizeof(long long)};
        void *dst[5] = {e->state, e->t, e->level, e->blocks, e->pairs};
        for (int q = 0; q < 5; ++q) {
            const cudaError_t ce = to_save ? cudaMemcpyAsync(p, src[q], len[q], cudaMemcpyDeviceToDevice, e->s)
                                           : cudaMemcpyAsync(dst[q], p, len[q], cudaMemcpyDeviceToDevice, e->s);
            if (ce != cudaSuccess) return ce;
            p += len[q];
        }
        return cudaSuccess;
    };
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int tprs[] = {1, 2, 4, 8, 16};
    float best = 1e30f;
    int bt = e->threads, bi = e->ipt, bp = e->tiles_per_range;
    cudaError_t ce = copy_state(true);
    for (const EnsShape &sh : kEnsShapes) {
        for (int tp : tprs) {
            if (ce != cudaSuccess || r != NBODY_OK) break;
            e->threads = sh.threads;
            e->ipt = sh.ipt;
            e->tiles_per_range = tp;
            cudaEventRecord(a, e->s);
            for (int k = 0; k < steps && r == NBODY_OK; ++k) r = ens_enqueue_step(e, tend);
            cudaEventRecord(b, e->s);
            ce = cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) {
                best = ms;
                bt = sh.threads;
                bi = sh.ipt;
                bp = tp;
            }
            if (ce == cudaSuccess) ce = copy_state(false);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->s);
    cudaFree(save);
    if (ce != cudaSuccess) return ecuda(ce, "tuner");
    if (r != NBODY_OK) return r;
    e->threads = bt;
    e->ipt = bi;
    e->tiles_per_range = bp;
    if (threads) *threads = bt;
    if (i_block) *i_block = bi;
    if (tiles_per_range) *tiles_per_range = bp;
    if (best_ms) *best_ms = best / steps;
    return ens_check(e);
}

int nbody_ens_energy(nbody_ens *e, double *ekin, double *epot)
{
    if (!e || !ekin || !epot) return efail(NBODY_EINVAL, "nbody_ens_energy: null argument");
    const size_t nc = static_cast<size_t>(e->n_cl);
    ens_time_range_kernel<<<e->n_cl, 256, 0, e->s>>>(e->E, e->trange);
    std::vector<long long> tr(2 * nc);
    NB_ECUDA(cudaMemcpyAsync(tr.data(), e->trange, 2 * nc * sizeof(long long), cudaMemcpyDeviceToHost, e->s),
             "time range");
    int r = ens_check(e);
    if (r != NBODY_OK) return r;
    for (size_t c = 0; c < nc; ++c)
        if (tr[2 * c] != tr[2 * c + 1]) return efail(NBODY_ENOTSYNC, "cluster %zu is not at one time", c);
    const int pg = static_cast<int>(std::min<int64_t>((e->n_tot + 127) / 128, e->sm_count * 32));
    ens_phi_kernel<<<pg, 128, 0, e->s>>>(e->E, e->eps2, e->phi);
    ens_energy_sum_kernel<<<e->n_cl, kEnsThreads, 0, e->s>>>(e->E, e->phi, e->e_out);
    NB_ECUDA(cudaGetLastError(), "energy kernels");
    std::vector<double> out(2 * nc);
    NB_ECUDA(cudaMemcpyAsync(out.data(), e->e_out, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, e->s),
             "energy read-back");
    r = ens_check(e);
    if (r != NBODY_OK) return r;
    for (size_t c = 0; c < nc; ++c) {
        ekin[c] = out[2 * c];
        epot[c] = out[2 * c + 1];
    }
    e->kernel_launches += 3;
    return NBODY_OK;
}

int nbody_ens_get_state(nbody_ens *e, double *x, double *v, double *a, double *k, int64_t *t_tick, int8_t *level)
{
    if (!e) return efail(NBODY_EINVAL, "nbody_ens_get_state: null ensemble");
    const size_t nd = static_cast<size_t>(e->n_tot);
    double *const *src[4] = {e->E.S.x, e->E.S.v, e->E.S.a, e->E.S.k};
    double *dst[4] = {x, v, a, k};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        NB_ECUDA(soa_to_aos_launch(src[q][0], src[q][1], src[q][2], e->stage, e->n_tot, e->s, &e->kernel_launches),
                 "layout");
        NB_ECUDA(cudaMemcpyAsync(dst[q], e->stage, 3 * nd * sizeof(double), cudaMemcpyDefault, e->s), "copy");
        NB_ECUDA(cudaStreamSynchronize(e->s), "stream synchronise");
    }
    if (t_tick) NB_ECUDA(cudaMemcpyAsync(t_tick, e->t, nd * sizeof(int64_t), cudaMemcpyDefault, e->s), "copy");
    if (level) NB_ECUDA(cudaMemcpyAsync(level, e->level, nd, cudaMemcpyDefault, e->s), "copy");
    return ens_check(e);
}

int nbody_ens_get_stats(nbody_ens *e, int64_t *blocks_per_cluster, int64_t *pairs_per_cluster,
                        int64_t *kernel_launches)
{
    if (!e) return efail(NBODY_EINVAL, "nbody_ens_get_stats: null ensemble");
    int64_t *outs[2] = {blocks_per_cluster, pairs_per_cluster};
    const long long *srcs[2] = {e->blocks, e->pairs};
    for (int q = 0; q < 2; ++q) {
        if (!outs[q]) continue;
        std::vector<long long> b(static_cast<size_t>(e->n_cl));
        NB_ECUDA(cudaMemcpyAsync(b.data(), srcs[q], b.size() * sizeof(long long), cudaMemcpyDeviceToHost, e->s),
                 "stats");
        NB_ECUDA(cudaStreamSynchronize(e->s), "stream synchronise");
        for (size_t c = 0; c < b.size(); ++c) outs[q][c] = b[c];
    }
    if (kernel_launches) *kernel_launches = e->kernel_launches;
    return NBODY_OK;
}

void nbody_ens_free(nbody_ens *e)
{
    if (!e) return;
    cudaStreamSynchronize(e->s);
    ens_release(e);
}

}  // extern "C"

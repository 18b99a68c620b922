// FP64 parts of the block-step Hermite integrator of Portegies Zwart,
// Belleman & Geldof (2007), Sect. 2: predictor, corrector with the Aarseth
// time step, power-of-two levels, the block scheduler, and the energy
// diagnostic.  All of them are memory- or latency-bound; FP64 never enters
// the O(N^2) pair loop (except in the energy diagnostic).
#include <cfloat>

#include "nbody_internal.cuh"
#include "step_impl.cuh"

namespace nb {

namespace {

constexpr int kThreads = 256;

int blocks_for(int64_t n, int threads, int cap = 1 << 20)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return static_cast<int>(b < cap ? b : cap);
}

// Predictor of Sect. 2 for every particle, FP64, and the FP32 j-stream the
// force reads.  FP64-pipe work per particle: the step, 15 fused multiply-adds
// and the lo differences; the roundings to float run on the integer pipe
// (d2f_rn) and the masses' were done once at set-up (mass_jstream_kernel).
// The structure-of-arrays stream is always written; the float4 streams only
// when a kernel of this context reads them (J.aos).
template <bool INTCONV>
__device__ __forceinline__ float to_f32(const double d)
{
    return INTCONV ? d2f_rn(d) : __double2float_rn(d);
}
template <bool INTCONV>
__device__ __forceinline__ double to_f64(const float f)
{
    return INTCONV ? f2d(f) : static_cast<double>(f);
}

// INTCONV: the roundings on the integer pipe (throughput, large n) or by the
// hardware conversion (latency, small n); both give the same bits.
template <bool INTCONV>
__global__ void predict_kernel(const State S, const JStream J, int64_t t_new, double tick, int lo_parts,
                               const long long *t_dev)
{
    if (t_dev) t_new = *t_dev;
    const int64_t np = J.n_pad;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < S.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const PredDt pd = pred_dt(static_cast<double>(t_new - S.t[i]) * tick);
        double xp[3], vp[3];
        float h[3], hv[3], lx[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            predict_dim(S.x[c][i], S.v[c][i], S.a[c][i], S.k[c][i], pd, xp[c], vp[c]);
            h[c] = to_f32<INTCONV>(xp[c]);
            hv[c] = to_f32<INTCONV>(vp[c]);
            lx[c] = lo_parts ? to_f32<INTCONV>(xp[c] - to_f64<INTCONV>(h[c])) : 0.f;  // the difference is exact
        }
        float *a = J.soa + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c * np] = h[c];
            a[(4 + c) * np] = hv[c];
            if (lo_parts) a[(7 + c) * np] = lx[c];
        }
        if (J.aos) {
            const float hm = a[3 * np];
            J.posm[i] = make_float4(h[0], h[1], h[2], hm);
            J.vel[i] = make_float4(hv[0], hv[1], hv[2], 0.f);
            if (lo_parts)
                J.poslo[i] = make_float4(lx[0], lx[1], lx[2],
                                         lo_parts > 1 ? d2f_rn(S.m[i] - f2d(hm)) : 0.f);
            if (lo_parts > 1)
                J.vello[i] = make_float4(d2f_rn(vp[0] - f2d(hv[0])), d2f_rn(vp[1] - f2d(hv[1])),
                                         d2f_rn(vp[2] - f2d(hv[2])), 0.f);
        }
    }
}

// The masses of the j-stream (structure-of-arrays and float4 forms), once at set-up.
__global__ void mass_jstream_kernel(const State S, const JStream J)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < S.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float hm = __double2float_rn(S.m[i]);
        J.soa[3 * J.n_pad + i] = hm;
        J.posm[i].w = hm;
    }
}

// The float4 streams from the structure-of-arrays stream (on demand, for
// readers of the float4 form when the predictor did not write it).
__global__ void aos_from_soa_kernel(const JStream J, int64_t n)
{
    const int64_t np = J.n_pad;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float *a = J.soa + i;
        J.posm[i] = make_float4(a[0], a[np], a[2 * np], a[3 * np]);
        J.vel[i] = make_float4(a[4 * np], a[5 * np], a[6 * np], 0.f);
        J.poslo[i] = make_float4(a[7 * np], a[8 * np], a[9 * np], 0.f);
    }
}

// Corrector of Sect. 2 plus Eq. (timestep), one block row per thread.
__global__ void correct_kernel(const State S, const int32_t *__restrict__ active, int64_t n_act,
                               const double *__restrict__ acc, const double *__restrict__ jerk,
                               int64_t t_new, double tick, double eta, int lmin, int lmax,
                               DevStatus *st, const SchedOut *sched_dev, const float *__restrict__ part,
                               int split, int two_word)
{
    if (sched_dev) {
        t_new = sched_dev->t_blk;
        n_act = sched_dev->n_act;
    }
    const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (q >= n_act) return;
    const int64_t i = active[q];
    if (i < 0 || i >= S.n) {
        atomicOr(&st->flags, kFlagBadIndex);
        st->bad_index = static_cast<int>(q);
        return;
    }
    if (part) {  // the block's j-range partials, added as reduce_partials_kernel does
        const int nc = two_word ? 14 : 7;
        if (!NB_CHECK(split > 1 && split < kFusedSplitMax, st, 3)) return;
        // all loads first (unrolled over the largest fused split, predicated), so
        // their latencies overlap; then the sums in ascending range order
        float hv[kFusedSplitMax - 1][6], lv[kFusedSplitMax - 1][6];
#pragma unroll
        for (int sp = 0; sp < kFusedSplitMax - 1; ++sp)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float *b = part + static_cast<size_t>(sp) * nc * n_act + q;
                hv[sp][c] = sp < split ? b[static_cast<size_t>(c) * n_act] : 0.0f;
                lv[sp][c] = (sp < split && two_word) ? b[static_cast<size_t>(7 + c) * n_act] : 0.0f;
            }
        double f[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double s = 0.0;
#pragma unroll
            for (int sp = 0; sp < kFusedSplitMax - 1; ++sp) {
                if (sp < split) {
                    s += static_cast<double>(hv[sp][c]);
                    if (two_word) s += static_cast<double>(lv[sp][c]);
                }
            }
            f[c] = s;
        }
        correct_row(S, i, f, f + 3, t_new, tick, eta, lmin, lmax, st);
        return;
    }
    correct_row(S, i, acc + 3 * q, jerk + 3 * q, t_new, tick, eta, lmin, lmax, st);
}

// Start of a run: a, k from the full force at t = 0, t = 0 and the first level
// from Eq. (initTimestep), dt = eta_init |a| / |k|.
__global__ void init_levels_kernel(const State S, const double *__restrict__ acc,
                                   const double *__restrict__ jerk, double eta_init, int lmin,
                                   int lmax, DevStatus *st)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= S.n) return;
    double a[3], k[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = acc[3 * i + c];
        k[c] = jerk[3 * i + c];
        S.a[c][i] = a[c];
        S.k[c][i] = k[c];
        finite = finite && isfinite(a[c]) && isfinite(k[c]);
    }
    const double kn = norm3(k);
    const double dt0 = kn == 0.0 ? static_cast<double>(INFINITY) : eta_init * norm3(a) / kn;
    bool clamped = false;
    int L = level_of(dt0, lmin, lmax, &clamped);
    if (!finite || L < 0) {
        L = lmax;
        atomicOr(&st->flags, kFlagNonfinite);
        atomicAdd(&st->nonfinite, 1ull);
    }
    if (clamped) {
        atomicOr(&st->flags, kFlagDtMin);
        atomicAdd(&st->below_min, 1ull);
    }
    S.t[i] = 0;
    S.level[i] = static_cast<int8_t>(L);
}

// ------------------------------------------------------------------ scheduler
// Three passes over contiguous chunks (one per block): (1) per-chunk minimum
// of t_i + dt_i, (2) global minimum and per-chunk match count, (3) ordered
// compaction of the matching indices at the prefix offset of each chunk.
struct SchedGeom {
    int64_t chunk;
    int blocks;
};

SchedGeom sched_geom(int64_t n)
{
    int64_t chunk = 2048;
    if ((n + chunk - 1) / chunk > 1024) chunk = ((n + 1023) / 1024 + kThreads - 1) / kThreads * kThreads;
    SchedGeom g;
    g.chunk = chunk;
    g.blocks = static_cast<int>((n + chunk - 1) / chunk);
    if (g.blocks < 1) g.blocks = 1;
    return g;
}

__device__ __forceinline__ unsigned long long due_tick(const State &S, int64_t i, int lmax)
{
    return static_cast<unsigned long long>(S.t[i] + (int64_t(1) << (lmax - S.level[i])));
}

__global__ void sched_min_kernel(const State S, int lmax, int64_t chunk, unsigned long long *bmin)
{
    __shared__ unsigned long long sh[32];
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = min(lo + chunk, S.n);
    unsigned long long m = ~0ull;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const unsigned long long d = due_tick(S, i, lmax);
        m = d < m ? d : m;
    }
    m = block_reduce(m, MinOp(), sh, ~0ull);
    if (threadIdx.x == 0) bmin[blockIdx.x] = m;
}

__global__ void sched_count_kernel(const State S, int lmax, int64_t chunk, int nblk,
                                   const unsigned long long *bmin, long long *bcnt, SchedOut *out)
{
    __shared__ unsigned long long shm[32];
    __shared__ long long shc[32];
    unsigned long long g = ~0ull;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) g = bmin[b] < g ? bmin[b] : g;
    g = block_reduce(g, MinOp(), shm, ~0ull);
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = min(lo + chunk, S.n);
    long long c = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += due_tick(S, i, lmax) == g;
    c = block_reduce(c, SumOp(), shc, 0ll);
    if (threadIdx.x == 0) {
        bcnt[blockIdx.x] = c;
        if (blockIdx.x == 0) out->t_blk = static_cast<long long>(g);
    }
}

__global__ void sched_write_kernel(const State S, int lmax, int64_t chunk, int nblk,
                                   const long long *bcnt, SchedOut *out, int32_t *active)
{
    __shared__ long long shc[32];
    __shared__ int warp_tot[32];
    const unsigned long long g = static_cast<unsigned long long>(out->t_blk);
    long long off = 0, total = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        if (b < static_cast<int>(blockIdx.x)) off += bcnt[b];
        total += bcnt[b];
    }
    off = block_reduce(off, SumOp(), shc, 0ll);
    total = block_reduce(total, SumOp(), shc, 0ll);
    if (blockIdx.x == 0 && threadIdx.x == 0) out->n_act = total;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = min(lo + chunk, S.n);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool hit = i < hi && due_tick(S, i, lmax) == g;
        const unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (l == 0) warp_tot[w] = __popc(mask);
        __syncthreads();
        int before = 0, round = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) before += warp_tot[k];
            round += warp_tot[k];
        }
        if (hit) active[off + before + __popc(mask & ((1u << l) - 1u))] = static_cast<int32_t>(i);
        off += round;
        __syncthreads();
    }
}

// Decision of the device-side block loop on the scheduled block (t, na); one thread.
__device__ __forceinline__ void loop_decide(const LoopArgs &la, long long t, long long na)
{
    StepLoop *L = la.L;
    const bool go = L->budget > 0 && (la.st->flags & la.stop_flags) == 0u && t <= L->t_end && na > 0 &&
                    na < la.n_fits && la.fits[na] != 0;
    if (go) {
        L->budget -= 1;
        L->blocks += 1;
        L->rows += na;
        L->last_t = t;
    }
    cudaGraphSetConditional(la.h, go ? 1u : 0u);
}

// n <= one chunk: the three passes in one block and one launch (same list);
// inside the block loop (LOOP) thread 0 then takes the loop's decision.
constexpr int kSchedSingleThreads = 1024;

template <bool LOOP>
__global__ void sched_single_kernel(const State S, int lmax, SchedOut *out, int32_t *active, const LoopArgs la)
{
    __shared__ unsigned long long shm[32];
    __shared__ int warp_tot[32];
    unsigned long long m = ~0ull;
    for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) {
        const unsigned long long d = due_tick(S, i, lmax);
        m = d < m ? d : m;
    }
    const unsigned long long g = block_reduce(m, MinOp(), shm, ~0ull);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    long long off = 0;
    for (int64_t base = 0; base < S.n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool hit = i < S.n && due_tick(S, i, lmax) == g;
        const unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (l == 0) warp_tot[w] = __popc(mask);
        __syncthreads();
        int before = 0, round = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) before += warp_tot[k];
            round += warp_tot[k];
        }
        if (hit) active[off + before + __popc(mask & ((1u << l) - 1u))] = static_cast<int32_t>(i);
        off += round;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->t_blk = static_cast<long long>(g);
        out->n_act = off;
        if (LOOP) loop_decide(la, static_cast<long long>(g), off);
    }
}

// The loop's decision after the multi-block scheduler; one thread.
__global__ void step_loop_kernel(const SchedOut *next, const LoopArgs la)
{
    loop_decide(la, next->t_blk, next->n_act);
}

// ------------------------------------------------------------------ energy
// phi_i = -sum_{j != i} m_j / sqrt(r^2 + eps^2) in FP64, j in ascending order.
constexpr int kETile = 128;

__global__ void phi_kernel(const State S, double eps2, double *__restrict__ phi)
{
    __shared__ double sx[kETile], sy[kETile], sz[kETile], sm[kETile];
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const bool live = i < S.n;
    const double xi = live ? S.x[0][i] : 0.0;
    const double yi = live ? S.x[1][i] : 0.0;
    const double zi = live ? S.x[2][i] : 0.0;
    double p = 0.0;
    for (int64_t j0 = 0; j0 < S.n; j0 += kETile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kETile; t += blockDim.x) {
            const int64_t j = j0 + t;
            const bool ok = j < S.n;
            sx[t] = ok ? S.x[0][j] : 0.0;
            sy[t] = ok ? S.x[1][j] : 0.0;
            sz[t] = ok ? S.x[2][j] : 0.0;
            sm[t] = ok ? S.m[j] : 0.0;
        }
        __syncthreads();
        const int jn = static_cast<int>(S.n - j0 < kETile ? S.n - j0 : kETile);
        for (int t = 0; t < jn; ++t) {
            if (j0 + t == i) continue;
            const double dx = sx[t] - xi, dy = sy[t] - yi, dz = sz[t] - zi;
            const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(eps2, __dmul_rn(dx, dx)), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz));
            p = __dsub_rn(p, __ddiv_rn(sm[t], __dsqrt_rn(r2)));
        }
    }
    if (live) phi[i] = p;
}

// One block: E_kin = sum m v^2 / 2, E_pot = sum m phi / 2 (fixed summation order).
__global__ void energy_sum_kernel(const State S, const double *__restrict__ phi, double *out)
{
    __shared__ double sk[1024], sp[1024];
    double k = 0.0, p = 0.0;
    for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) {
        const double vx = S.v[0][i], vy = S.v[1][i], vz = S.v[2][i];
        k += 0.5 * S.m[i] * (vx * vx + vy * vy + vz * vz);
        p += 0.5 * S.m[i] * phi[i];
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
        out[0] = sk[0];
        out[1] = sp[0];
    }
}

__global__ void time_range_kernel(const State S, unsigned long long *out)
{
    __shared__ unsigned long long sh[32];
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < S.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const unsigned long long t = static_cast<unsigned long long>(S.t[i]);
        lo = t < lo ? t : lo;
        hi = t > hi ? t : hi;
    }
    lo = block_reduce(lo, MinOp(), sh, ~0ull);
    hi = block_reduce(hi, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0) {
        atomicMin(&out[0], lo);
        atomicMax(&out[1], hi);
    }
}

__global__ void aos_to_soa_kernel(const double *__restrict__ aos, double *c0, double *c1, double *c2, int64_t n)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        c0[i] = aos[3 * i];
        c1[i] = aos[3 * i + 1];
        c2[i] = aos[3 * i + 2];
    }
}

__global__ void soa_to_aos_kernel(const double *c0, const double *c1, const double *c2, double *__restrict__ aos,
                                  int64_t n)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        aos[3 * i] = c0[i];
        aos[3 * i + 1] = c1[i];
        aos[3 * i + 2] = c2[i];
    }
}

// Padding of the j-stream: massless particles far away (r^2 ~ 3e30), so a
// padding pair adds exactly zero even with eps = 0 and a particle at the origin.
__global__ void pad_jstream_kernel(float4 *posm, float4 *vel, float4 *poslo, float *soa, int64_t n, int64_t n_pad)
{
    for (int64_t i = n + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_pad;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        posm[i] = make_float4(kPadPosition, kPadPosition, kPadPosition, 0.f);
        vel[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        poslo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (soa)
            for (int a = 0; a < kSoaArrays; ++a) soa[a * n_pad + i] = a < 3 ? kPadPosition : 0.f;
    }
}

__global__ void iota_kernel(int32_t *a, int64_t n)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        a[i] = static_cast<int32_t>(i);
}

}  // namespace

cudaError_t pad_jstream_launch(const JStream &J, int64_t n, cudaStream_t s, int64_t *launches)
{
    if (J.n_pad <= n) return cudaSuccess;
    pad_jstream_kernel<<<1, kThreads, 0, s>>>(J.posm, J.vel, J.poslo, J.soa, n, J.n_pad);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t iota_launch(int32_t *a, int64_t n, cudaStream_t s, int64_t *launches)
{
    iota_kernel<<<blocks_for(n, kThreads, 152 * 32), kThreads, 0, s>>>(a, n);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t mass_jstream_launch(const State &S, const JStream &J, cudaStream_t s, int64_t *launches)
{
    mass_jstream_kernel<<<blocks_for(S.n, kThreads, 152 * 8), kThreads, 0, s>>>(S, J);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t aos_from_soa_launch(const JStream &J, int64_t n, cudaStream_t s, int64_t *launches)
{
    aos_from_soa_kernel<<<blocks_for(n, kThreads, 152 * 8), kThreads, 0, s>>>(J, n);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t predict_launch(const State &S, const JStream &J, int64_t t_new, int lmax, int lo_parts,
                           cudaStream_t s, int64_t *launches, const long long *t_dev)
{
    // FP64 per particle: small n spread over more SMs (GB300's FP64 rate per SM is low)
    const int tpb = S.n >= 152 * 128 ? kThreads : 32;
    const unsigned grid = static_cast<unsigned>(blocks_for(S.n, tpb, 152 * 64 * (kThreads / tpb)));
    if (S.n >= 152 * 128)
        predict_kernel<true><<<grid, tpb, 0, s>>>(S, J, t_new, ldexp(1.0, -lmax), lo_parts, t_dev);
    else
        predict_kernel<false><<<grid, tpb, 0, s>>>(S, J, t_new, ldexp(1.0, -lmax), lo_parts, t_dev);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t correct_launch(const State &S, const int32_t *active, int64_t n_act, const double *acc,
                           const double *jerk, int64_t t_new, double eta, int lmin, int lmax, DevStatus *st,
                           cudaStream_t s, int64_t *launches, const SchedOut *sched_dev, const float *part,
                           int split, bool two_word)
{
    if (n_act <= 0) return cudaSuccess;
    // FP64-heavy rows: small blocks spread over more SMs (GB300's FP64 rate per SM is low)
    const int tpb = n_act >= 152 * 128 ? 128 : 32;
    correct_kernel<<<blocks_for(n_act, tpb), tpb, 0, s>>>(S, active, n_act, acc, jerk, t_new, ldexp(1.0, -lmax),
                                                          eta, lmin, lmax, st, sched_dev, part, split,
                                                          two_word ? 1 : 0);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t init_levels_launch(const State &S, const double *acc, const double *jerk, double eta_init, int lmin,
                               int lmax, DevStatus *st, cudaStream_t s, int64_t *launches)
{
    init_levels_kernel<<<blocks_for(S.n, kThreads), kThreads, 0, s>>>(S, acc, jerk, eta_init, lmin, lmax, st);
    ++*launches;
    return cudaGetLastError();
}

size_t sched_scratch_bytes(int64_t n)
{
    const SchedGeom g = sched_geom(n);
    return static_cast<size_t>(g.blocks) * (sizeof(unsigned long long) + sizeof(long long));
}

cudaError_t schedule_launch(const State &S, int lmax, int32_t *active, SchedOut *out, void *scratch,
                            cudaStream_t s, int64_t *launches)
{
    const SchedGeom g = sched_geom(S.n);
    if (g.blocks == 1) {
        sched_single_kernel<false><<<1, kSchedSingleThreads, 0, s>>>(S, lmax, out, active, LoopArgs{});
        ++*launches;
        return cudaGetLastError();
    }
    unsigned long long *bmin = static_cast<unsigned long long *>(scratch);
    long long *bcnt = reinterpret_cast<long long *>(bmin + g.blocks);
    sched_min_kernel<<<g.blocks, kThreads, 0, s>>>(S, lmax, g.chunk, bmin);
    sched_count_kernel<<<g.blocks, kThreads, 0, s>>>(S, lmax, g.chunk, g.blocks, bmin, bcnt, out);
    sched_write_kernel<<<g.blocks, kThreads, 0, s>>>(S, lmax, g.chunk, g.blocks, bcnt, out, active);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t schedule_loop_launch(const State &S, int lmax, int32_t *active, SchedOut *out, void *scratch,
                                 const LoopArgs &la, cudaStream_t s, int64_t *launches)
{
    if (sched_geom(S.n).blocks == 1) {
        sched_single_kernel<true><<<1, kSchedSingleThreads, 0, s>>>(S, lmax, out, active, la);
        ++*launches;
        return cudaGetLastError();
    }
    cudaError_t e = schedule_launch(S, lmax, active, out, scratch, s, launches);
    if (e != cudaSuccess) return e;
    step_loop_kernel<<<1, 1, 0, s>>>(out, la);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t energy_launch(const State &S, double eps2, double *phi, double *out, cudaStream_t s,
                          int64_t *launches, bool ds_potential)
{
    if (ds_potential) {
        const cudaError_t e = phi_ds_launch(S, eps2, phi, s, launches);
        if (e != cudaSuccess) return e;
    } else {
        phi_kernel<<<blocks_for(S.n, kETile), kETile, 0, s>>>(S, eps2, phi);
        ++*launches;
    }
    energy_sum_kernel<<<1, 1024, 0, s>>>(S, phi, out);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t time_range_launch(const State &S, unsigned long long *out, cudaStream_t s, int64_t *launches)
{
    cudaError_t e = cudaMemsetAsync(out, 0xff, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(out + 1, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    time_range_kernel<<<blocks_for(S.n, kThreads, 152 * 8), kThreads, 0, s>>>(S, out);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t aos_to_soa_launch(const double *aos, double *c0, double *c1, double *c2, int64_t n, cudaStream_t s,
                              int64_t *launches)
{
    aos_to_soa_kernel<<<blocks_for(n, kThreads, 152 * 32), kThreads, 0, s>>>(aos, c0, c1, c2, n);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t soa_to_aos_launch(const double *c0, const double *c1, const double *c2, double *aos, int64_t n,
                              cudaStream_t s, int64_t *launches)
{
    soa_to_aos_kernel<<<blocks_for(n, kThreads, 152 * 32), kThreads, 0, s>>>(c0, c1, c2, aos, n);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace nb

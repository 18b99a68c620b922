// Block steps of a small system inside one thread-block cluster: the block
// time-step scheme of Sect. 2 (the next block time and its active particles,
// the predictor, the force of Eq. (Force) on the active particles, the
// corrector and Eq. (timestep)) repeated by one launch, the CTAs of the
// cluster meeting at two hardware cluster barriers per block.
//
// At small n a block is latency: separate kernels for the schedule, the
// predictor, the force and the corrector cost a few microseconds each even when
// they have almost nothing to do.  Here CTA r of C owns the particles
// [r chunk, (r+1) chunk), chunk = n_pad / C.  Per block:
//   1. each CTA takes the earliest due tick t_i + dt_i over its particles that
//      were not in the last block and the rows it corrected in the last block,
//      and stores it into every CTA's shared memory; barrier A; every CTA takes
//      the minimum, the block time (each CTA keeps the due ticks of its own
//      particles in shared memory; a corrector stores a row's new one into its
//      owner's);
//   2. each CTA predicts all of its particles into the j-stream in global
//      memory (structure of arrays; the float4 streams in the double-single
//      mode) and stores its active particles (ascending) and their count into
//      every CTA's shared memory; barrier C;
//   3. each CTA copies the predicted j-stream into shared memory (asynchronous
//      copies through L2, while it finds its rows): the block's rows, in list
//      order, cut into C equal contiguous shares.  It computes the force on its
//      share over all n j (T threads per row, T a power of two, taking groups of
//      4 j in turn; the T sums added in a fixed tree), and corrects its share:
//      up to 8 rows in one warp, 4 lanes per row, else one row per lane of as
//      few warps as possible.
// GB300's FP64 unit is one per SM and takes ~19 cycles per warp instruction
// whatever the number of active lanes (64-cycle latency, ~650-700 for a
// division or square root), so the FP64 corrector packs its rows into as few
// warps as the lanes allow, and the rows are spread evenly over the cluster's
// SMs; the predictor rounds to float on the integer pipe (d2f_rn, f2d: the
// same bits).  State written by
// one CTA and read by another in a later block is read through L2 only.  The
// masses of the j-stream are copied once.
//
// Every decision to go on or stop (block time past t_end, budget spent, a stop
// flag, an empty block or one larger than rows_max) is taken from values every
// CTA holds alike after a barrier, so all CTAs leave the loop together; the
// status flags are read by CTA 0 between barriers A and C, when no corrector
// runs, and passed on with its count.  No wait spins: the barriers are the
// hardware's, and the loop runs at most `budget` blocks.
//
// The pair term and its 128-term folds are those of the packed force kernel
// (force_x2.cuh); the per-thread sums of a row are added in double-single
// (compensated) or FP32 (plain) arithmetic in a fixed order.  The double-single
// mode (n_pad <= kClMaxPadDS) takes the pair term of force_ds.cu (ds_pair_term)
// one j at a time over the float4 streams (x, m), (x_lo, m_lo), v, v_lo.  The
// predictor and the corrector are those of step_impl.cuh, so the state a block
// leaves differs from the separate kernels' only by the summation order of its
// forces.
#include <cooperative_groups.h>

#include "block_rows.cuh"

namespace cg = cooperative_groups;

namespace nb {

namespace {

constexpr int kClThreads = 512;
constexpr int kClWarps = kClThreads / 32;
constexpr int kClMaxC = 16;
static_assert(kClMaxChunk <= kClThreads, "one own particle per thread");

struct ClArgs {
    State S;
    float *soa;  // the predicted j-stream (kSoaArrays x n_pad); padding entries stay as set up
    float4 *posm, *poslo, *vel, *vello;  // its float4 form (double-single mode)
    int64_t n_pad;
    float eps2, eps2_lo;  // eps^2 and, for the double-single mode, its low part
    double tick, eta;
    int lmin, lmax;
    long long t_end, budget, rows_max, last_t;
    unsigned stop_flags;
    DevStatus *st;
    SchedOut *sched_out;
    StepLoop *L;
    int32_t *act_out;  // the block's list (n), for the host
};

// Bytes of shared memory the mode's copy of the j-stream takes per particle.
template <int MODE>
constexpr int cl_jbytes()
{
    return MODE == kModeDS ? 4 * static_cast<int>(sizeof(float4)) : SoaTile<MODE>::NA * static_cast<int>(sizeof(float));
}

template <int MODE>
__global__ void __launch_bounds__(kClThreads, 1) cluster_step_kernel(const ClArgs A)
{
    constexpr bool DSM = MODE == kModeDS;
    constexpr int NA = SoaTile<MODE>::NA;
    constexpr bool DSW = MODE == kModeComp || DSM;  // two-word sums
    // the predicted j-stream: NA x n_pad floats (structure of arrays), or in the
    // double-single mode 4 x n_pad float4: (x, m), (x_lo, m_lo), v, v_lo
    extern __shared__ __align__(16) float jsm[];
    __shared__ unsigned long long x_min[kClMaxC];  // earliest due tick of each CTA (stored by that CTA)
    __shared__ int x_cnt[kClMaxC];                 // active count of each CTA (stored by that CTA)
    __shared__ unsigned x_flags;                   // status flags of this block (stored by CTA 0)
    __shared__ int row_idx[kClMaxChunk];           // this CTA's share of the block's rows
    __shared__ float f_hi[kClMaxChunk][6], f_lo[kClMaxChunk][6];  // their acc and jerk sums
    __shared__ int warp_tot[kClWarps];
    __shared__ float wred[kClWarps][7][2];
    __shared__ unsigned long long red_u64[32];
    __shared__ int b_pre[kClMaxC + 1];
    __shared__ int lists[kClMaxPad];  // CTA r's active particles at r chunk .. (stored by CTA r)
    __shared__ unsigned long long due_c[kClMaxChunk];  // due ticks of this CTA's particles
    __shared__ unsigned long long due_r[kClMaxChunk];  // new due ticks of the rows it corrected last

    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks());
    const int rank = static_cast<int>(cl.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const State &S = A.S;
    const int64_t n = S.n;
    const int np = static_cast<int>(A.n_pad);
    const int chunk = np / C;
    const int lo_i = rank * chunk;
    const int hi_i = static_cast<int>(min(static_cast<int64_t>(lo_i + chunk), n));

    const int i = lo_i + tid;  // this thread's own particle
    const bool mine = tid < chunk && i < hi_i;
    if (mine)
        due_c[tid] = static_cast<unsigned long long>(ld_state<true>(S.t + i) +
                                                     (int64_t(1) << (A.lmax - ld_state<true>(S.level + i))));
    float m_hi = 0.0f, m_lo = 0.0f;  // double-single mode: this thread's mass split
    if constexpr (DSM) {
        if (mine) {
            const double mm = S.m[i];
            m_hi = d2f_rn(mm);
            m_lo = d2f_rn(mm - f2d(m_hi));
        }
    } else {  // the j-stream's masses (the rest is copied before each block's forces)
        const float4 *src = reinterpret_cast<const float4 *>(A.soa + 3 * np);
        float4 *dst = reinterpret_cast<float4 *>(jsm + 3 * np);
        for (int k = tid; k < np / 4; k += kClThreads) dst[k] = src[k];
    }
    cl.sync();  // every CTA of the cluster runs before any stores into another's shared memory
    long long done = 0, rows = 0, last_t = A.last_t;
    unsigned long long tb = 0;
    int na = 0, cnt_last = 0;
    bool hit = false;  // this thread's particle was in the last block
    for (;;) {
        // 1. the earliest due tick over this CTA's particles that were not in the last
        //    block (unchanged) and the rows it corrected (their new ones), stored into every CTA
        unsigned long long m = (mine && !hit) ? due_c[tid] : ~0ull;
        if (tid < cnt_last) m = due_r[tid] < m ? due_r[tid] : m;
        m = block_reduce(m, MinOp(), red_u64, ~0ull);
        if (warp == 0 && lane < C) *cl.map_shared_rank(&x_min[rank], lane) = m;
        cl.sync();  // barrier A: every corrector of the last block has finished
        if (rank == 0 && tid == 0) x_flags = __ldcg(&A.st->flags);  // stored into the others below
        tb = ~0ull;
        for (int r = 0; r < C; ++r) tb = x_min[r] < tb ? x_min[r] : tb;

        // 2. this CTA's active particles (ascending) and its particles predicted to tb
        {
            hit = mine && due_c[tid] == tb;
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) warp_tot[warp] = __popc(mask);
            if (mine) {  // the state through L2: another CTA may have corrected it
                const PredDt pd = pred_dt(static_cast<double>(static_cast<int64_t>(tb) - ld_state<true>(S.t + i)) * A.tick);
                float h[3], hl[3], hv[3], hvl[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double xp, vp;
                    predict_dim(ld_state<true>(S.x[c] + i), ld_state<true>(S.v[c] + i), ld_state<true>(S.a[c] + i),
                                ld_state<true>(S.k[c] + i), pd, xp, vp);
                    h[c] = d2f_rn(xp);
                    hv[c] = d2f_rn(vp);
                    hl[c] = DSW ? d2f_rn(xp - f2d(h[c])) : 0.0f;  // the differences are exact
                    hvl[c] = DSM ? d2f_rn(vp - f2d(hv[c])) : 0.0f;
                }
                if constexpr (DSM) {
                    A.posm[i] = make_float4(h[0], h[1], h[2], m_hi);
                    A.poslo[i] = make_float4(hl[0], hl[1], hl[2], m_lo);
                    A.vel[i] = make_float4(hv[0], hv[1], hv[2], 0.0f);
                    A.vello[i] = make_float4(hvl[0], hvl[1], hvl[2], 0.0f);
                } else {
                    float *a = A.soa + i;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        a[c * np] = h[c];
                        a[(4 + c) * np] = hv[c];
                        if (DSW) a[(7 + c) * np] = hl[c];
                    }
                }
            }
            __syncthreads();
            int before = 0, total = 0;
            for (int k = 0; k < kClWarps; ++k) {
                before += k < warp ? warp_tot[k] : 0;
                total += warp_tot[k];
            }
            if (hit) {
                const int slot = lo_i + before + __popc(mask & ((1u << lane) - 1u));
                if (NB_CHECK(slot < hi_i, A.st, 4))
                    for (int r = 0; r < C; ++r) *cl.map_shared_rank(&lists[slot], r) = i;
            }
            if (warp == 0 && lane < C) {
                *cl.map_shared_rank(&x_cnt[rank], lane) = total;
                if (rank == 0) *cl.map_shared_rank(&x_flags, lane) = x_flags;
            }
        }
        cl.sync();  // barrier C: the j-stream, the lists, the counts and the flags are stored
        if constexpr (DSM) {  // the four float4 streams into shared memory, while the rows are found
            float4 *dst = reinterpret_cast<float4 *>(jsm);
            const float4 *srcs[4] = {A.posm, A.poslo, A.vel, A.vello};
            for (int k = tid; k < 4 * np; k += kClThreads) {
                const int a = k / np, e = k - a * np;
                cp_async16_cg(dst + k, srcs[a] + e);
            }
            cp_async_commit();
        } else {  // the j-stream's positions and velocities into shared memory, while the rows are found
            const int nq = np / 4;
            for (int k = tid; k < (NA - 1) * nq; k += kClThreads) {
                const int a = k / nq, off = 4 * (k - a * nq) + (a >= 3 ? a + 1 : a) * np;  // every array but m
                cp_async16_cg(jsm + off, A.soa + off);
            }
            cp_async_commit();
        }
        if (warp == 0) {  // where each CTA's list starts in the block's list
            const int v = lane < C ? x_cnt[lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane <= C) b_pre[lane] = incl - v;
        }
        __syncthreads();
        na = b_pre[C];
        const bool go = done < A.budget && (x_flags & A.stop_flags) == 0u && static_cast<long long>(tb) <= A.t_end &&
                        na > 0 && na <= A.rows_max;
        // this CTA's share of the rows in list order, and the list for the host
        const int p0 = static_cast<int>(static_cast<long long>(rank) * na / C);
        const int p1 = static_cast<int>(static_cast<long long>(rank + 1) * na / C);
        const int cnt = p1 - p0;
        if (tid < cnt) {
            const int p = p0 + tid;
            int o = 0;
            while (o + 1 < C && b_pre[o + 1] <= p) ++o;
            const int e = o * chunk + (p - b_pre[o]);
            const int r = NB_CHECK(e >= o * chunk && e < min((o + 1) * chunk, np), A.st, 5) ? lists[e] : 0;
            row_idx[tid] = r;
            A.act_out[p] = r;
        }
        cp_async_wait_all();
        __syncthreads();
        if (!go) break;

        // 3. forces on this CTA's share of the rows, then their correction
        if (cnt > 0) {
            // T threads per row: the largest power of two with T cnt <= threads whose
            // j-share n_pad / T is a multiple of 8
            int T = kClThreads;
            while (T > 1 && (T * cnt > kClThreads || (np / 8) % T != 0)) T >>= 1;
            auto load_i = [&](const int rr, const bool live, I2 &I) {
                const int gi = live ? row_idx[rr] : -1;
                const int li = live ? gi : 0;
                I.x = f2_pack(jsm[li], jsm[li]);
                I.y = f2_pack(jsm[np + li], jsm[np + li]);
                I.z = f2_pack(jsm[2 * np + li], jsm[2 * np + li]);
                I.vx = f2_pack(jsm[4 * np + li], jsm[4 * np + li]);
                I.vy = f2_pack(jsm[5 * np + li], jsm[5 * np + li]);
                I.vz = f2_pack(jsm[6 * np + li], jsm[6 * np + li]);
                if (DSW && !DSM) {
                    I.lx = f2_pack(jsm[7 * np + li], jsm[7 * np + li]);
                    I.ly = f2_pack(jsm[8 * np + li], jsm[8 * np + li]);
                    I.lz = f2_pack(jsm[9 * np + li], jsm[9 * np + li]);
                }
                return gi;
            };
            auto load_ds = [&](const int rr, const bool live, dsa::ds (&xi)[3], dsa::ds (&vi)[3]) {
                const int gi = live ? row_idx[rr] : -1;
                const int li = live ? gi : 0;
                const float4 *sp = reinterpret_cast<const float4 *>(jsm);
                const float4 ph = sp[li], pl = sp[np + li], vh = sp[2 * np + li], vl = sp[3 * np + li];
                xi[0] = {ph.x, pl.x};
                xi[1] = {ph.y, pl.y};
                xi[2] = {ph.z, pl.z};
                vi[0] = {vh.x, vl.x};
                vi[1] = {vh.y, vl.y};
                vi[2] = {vh.z, vl.z};
                return gi;
            };
            auto store = [&](const int rr, const float *tot, const float *lo) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    f_hi[rr][c] = tot[c];
                    f_lo[rr][c] = DSW ? lo[c] : 0.0f;
                }
            };
            rows_force<MODE, kClThreads>(jsm, np, 0, np, cnt, T, A.eps2, A.eps2_lo, load_i, load_ds, store, wred);
            // the new due tick of each row: kept for this CTA's next minimum and stored into
            // the owner's shared memory for its schedule after barrier A
            auto due = [&](const int q, const int r, const unsigned long long dd) {
                due_r[q] = dd;
                const int o = r / chunk;
                if (NB_CHECK(o < C && r - o * chunk < chunk, A.st, 6)) *cl.map_shared_rank(&due_c[r - o * chunk], o) = dd;
            };
            rows_correct<DSW>(S, row_idx, f_hi, f_lo, cnt, tb, A.tick, A.eta, A.lmin, A.lmax, A.st, due);
        }
        cnt_last = cnt;
        ++done;
        rows += na;
        last_t = static_cast<long long>(tb);
    }
    if (rank == 0 && tid == 0) {
        A.sched_out->t_blk = static_cast<long long>(tb);
        A.sched_out->n_act = na;
        A.L->blocks = done;
        A.L->rows = rows;
        A.L->last_t = last_t;
    }
    cl.sync();  // no CTA leaves while another may still store into its shared memory
}

int cl_max_pad(int mode) { return mode == kModeDS ? kClMaxPadDS : kClMaxPad; }

template <int MODE>
int cluster_size_for()
{
    // 16 CTAs where the device takes that non-portable size, else the portable 8, else 0;
    // found once per mode (a function-local static: thread-safe initialisation)
    static const int size = [] {
        auto kern = cluster_step_kernel<MODE>;
        const size_t smem = static_cast<size_t>(cl_jbytes<MODE>()) * cl_max_pad(MODE);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        for (int C : {16, 8}) {
            if (C > 8 &&
                cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(kClThreads);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters >= 1) return C;
            cudaGetLastError();
        }
        return 0;
    }();
    return size;
}

}  // namespace

int cluster_step_size(int mode)
{
    if (mode == kModePlain) return cluster_size_for<kModePlain>();
    if (mode == kModeComp) return cluster_size_for<kModeComp>();
    if (mode == kModeDS) return cluster_size_for<kModeDS>();
    return 0;
}

cudaError_t cluster_step_launch(int mode, const State &S, const JStream &J, double eps2, double eta, int lmin,
                                int lmax, long long t_end, long long budget, long long rows_max, long long last_t,
                                unsigned stop_flags, DevStatus *st, SchedOut *sched_out, StepLoop *L,
                                int32_t *act_out, cudaStream_t s, int64_t *launches)
{
    const int C = cluster_step_size(mode);
    if (C == 0 || C > kClMaxC || J.n_pad > cl_max_pad(mode) || J.n_pad % kJTile != 0 || J.n_pad / C > kClMaxChunk ||
        !J.soa)
        return cudaErrorInvalidValue;
    ClArgs A;
    A.S = S;
    A.soa = J.soa;
    A.posm = J.posm;
    A.poslo = J.poslo;
    A.vel = J.vel;
    A.vello = J.vello;
    A.n_pad = J.n_pad;
    A.eps2 = static_cast<float>(eps2);
    A.eps2_lo = static_cast<float>(eps2 - static_cast<double>(A.eps2));
    A.tick = ldexp(1.0, -lmax);
    A.eta = eta;
    A.lmin = lmin;
    A.lmax = lmax;
    A.t_end = t_end;
    A.budget = budget;
    A.rows_max = rows_max;
    A.last_t = last_t;
    A.stop_flags = stop_flags;
    A.st = st;
    A.sched_out = sched_out;
    A.L = L;
    A.act_out = act_out;
    const int jbytes = mode == kModeDS ? cl_jbytes<kModeDS>() : mode == kModeComp ? cl_jbytes<kModeComp>()
                                                                                 : cl_jbytes<kModePlain>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = static_cast<size_t>(jbytes) * J.n_pad;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = mode == kModeDS     ? cudaLaunchKernelEx(&cfg, cluster_step_kernel<kModeDS>, A)
                          : mode == kModeComp ? cudaLaunchKernelEx(&cfg, cluster_step_kernel<kModeComp>, A)
                                              : cudaLaunchKernelEx(&cfg, cluster_step_kernel<kModePlain>, A);
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace nb

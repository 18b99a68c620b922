// Block steps of a larger system as one cooperative launch over the whole GPU:
// the block time-step scheme of Sect. 2 (the next block time and its active
// particles, the predictor, the force of Eq. (Force) on the active particles,
// the corrector and Eq. (timestep)) repeated on the device, the CTAs meeting at
// three bounded grid barriers per block.
//
// Past the one-cluster kernel's sizes, a block of a few hundred rows costs more
// in the separate kernels' latency (three scheduler passes, the predictor, the
// force and its reduction, the corrector: ~60 us at N = 65536) than in its pair
// interactions.  Here CTA g of G (one per SM) owns the particles
// [g ch, (g+1) ch), ch = ceil(n / G) rounded up to 4, keeps their due ticks
// t_i + dt_i and, each block, their prediction in shared memory.  Per block:
//   1. each CTA takes the earliest due tick over its particles and lists its
//      particles due then (ascending); it publishes the tick, the count and the
//      status flags it sees; barrier;
//   2. every CTA takes the block time (the minimum), the block size and where
//      its own rows start in the block's list (the counts of the CTAs before it
//      that hold the minimum), all alike, and decides alike whether the block
//      runs; it writes its rows into the list, predicts all of its particles to
//      the block time into shared memory (structure of arrays) and copies its
//      rows' predicted data into a row buffer; barrier;
//   3. every CTA sums the pair terms of all of the block's rows over its own
//      particles (T threads per row, rows_force) and writes one partial per row;
//      barrier;
//   4. each CTA adds the G partials of each of its own rows in CTA order (lanes
//      over CTAs, then a butterfly: double-single in compensated mode) and
//      corrects them (rows_correct), keeping their new due ticks.
// The state of a particle is read and written by its owner only; what crosses
// CTAs (published ticks, the list, the row buffer, the partials) is read through
// L2 after a barrier.  The barriers count arrivals on one counter in global
// memory (zeroed before each launch) and give up after ~1 s, raising the
// timeout flag; the cooperative launch guarantees that all CTAs are resident.
// The loop stops, every CTA alike, at a block past t_end, a raised stop flag, a
// spent budget or a block larger than rows_max; that block's list and size are
// left for the host, and for a larger block also the j-stream predicted to its
// time (each CTA its particles), so that the host runs it through the separate
// force kernel and corrector alone.
//
// The forces of a block are the separate kernels' pair terms summed in another
// order (per CTA, then across CTAs), so the state differs from theirs by
// rounding only; the order depends on the block size and G alone, so runs repeat
// bit for bit.
#include "block_rows.cuh"

namespace nb {

namespace {

constexpr int kGrThreads = 512;
constexpr int kGrWarps = kGrThreads / 32;

// What each CTA publishes before the barrier of step 1.
struct GrPub {
    unsigned long long m;  // earliest due tick of its particles
    int cnt;               // its particles due then
    unsigned flags;        // the status flags it saw
};

struct GrArgs {
    State S;
    float *soa;           // the j-stream (kSoaArrays x n_pad floats, structure of arrays)
    int64_t n_pad;
    const float *mass_j;  // the j-stream's masses (float), n entries
    int chunk;            // particles per CTA, a multiple of 4
    int rows_max;         // largest block this launch runs; rows of the row buffer
    float eps2;
    double tick, eta;
    int lmin, lmax;
    long long t_end, budget, last_t;
    unsigned stop_flags;
    int skip_arrival;  // test hook: the last CTA leaves before its first barrier (the others' wait gives up)
    DevStatus *st;
    SchedOut *sched_out;
    StepLoop *L;
    int32_t *act_out;         // the block's list (n), for the host too
    float *ri;                // predicted data of the block's rows: (NA - 1) x rows_max (no masses)
    float *part;              // partials: rows_max x G x (12 or 6) floats
    GrPub *pub;               // G records
    unsigned long long *bar;  // barrier counter, zero at launch
};

// Dynamic shared memory of a CTA: the prediction of its particles (NA arrays of
// SJ >= chunk floats: a compile-time stride folds into the force loop's load
// offsets; the kernel is built for a few strides, the smallest that holds the
// chunk is launched), their due ticks and its rows of a block.
constexpr int kGrStrides[4] = {512, 1024, 2048, kGrMaxChunk};
template <int MODE, int SJ>
constexpr size_t gr_smem()
{
    return static_cast<size_t>(SJ) * (SoaTile<MODE>::NA * sizeof(float) + sizeof(unsigned long long) + sizeof(int));
}

template <int MODE, int SJ>
__global__ void __launch_bounds__(kGrThreads, 1) grid_step_kernel(const GrArgs A)
{
    constexpr int NA = SoaTile<MODE>::NA;
    constexpr bool DSW = MODE == kModeComp;
    constexpr int PW = DSW ? 12 : 6;  // floats per partial
    extern __shared__ __align__(16) float jsm[];  // NA x SJ: x, y, z, m, vx, vy, vz (, x_lo, y_lo, z_lo)
    __shared__ float f_hi[kGrThreads][6], f_lo[kGrThreads][6];  // forces of up to kGrThreads own rows
    __shared__ float wred[kGrWarps][7][2];
    __shared__ unsigned long long red_u64[32];
    __shared__ int warp_tot[kGrWarps];
    __shared__ unsigned long long s_tb;
    __shared__ int s_na, s_off, s_ok;
    __shared__ unsigned s_flags;

    const int CH = A.chunk;
    unsigned long long *due_c = reinterpret_cast<unsigned long long *>(jsm + NA * SJ);  // CH used (16-byte aligned)
    int *own = reinterpret_cast<int *>(due_c + SJ);  // this CTA's rows of the block (particle indices, ascending)
    const int G = static_cast<int>(gridDim.x), g = static_cast<int>(blockIdx.x);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const State &S = A.S;
    const int n = static_cast<int>(S.n);
    const int lo = g * CH;
    const int nown = max(0, min(lo + CH, n) - lo);
    const int L = (nown + 3) & ~3;  // entries the force reads: own particles, then massless padding
    const int RM = A.rows_max;

    for (int k = tid; k < CH; k += kGrThreads) {
        const bool in = k < nown;
        due_c[k] = in ? static_cast<unsigned long long>(ld_state<true>(S.t + lo + k) +
                                                        (int64_t(1) << (A.lmax - ld_state<true>(S.level + lo + k))))
                      : ~0ull;
#pragma unroll
        for (int a = 0; a < NA; ++a) jsm[a * SJ + k] = in ? 0.0f : (a < 3 ? kPadPosition : 0.0f);
        if (in) jsm[3 * SJ + k] = A.mass_j[lo + k];
    }
    __syncthreads();

    unsigned long long target = 0;  // thread 0: arrivals the barriers have waited for
    auto barrier = [&]() {  // false: a barrier gave up (recorded); every CTA then leaves
        if (grid_barrier(A.bar, target, G, &s_ok)) return true;
        if (tid == 0) atomicOr(&A.st->flags, static_cast<unsigned>(kFlagTimeout));
        return false;
    };
    // this CTA's particles predicted to tick t: array a of particle lo + k at dst[a * stride + base + k]
    // (x, y, z, vx, vy, vz and, compensated, the lo parts of x, y, z: the predictor kernel's values)
    auto predict_own = [&](const unsigned long long t, float *dst, const int64_t stride, const int64_t base) {
        for (int k = tid; k < nown; k += kGrThreads) {
            const int i = lo + k;
            const PredDt pd = pred_dt(static_cast<double>(static_cast<int64_t>(t) - ld_state<true>(S.t + i)) * A.tick);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double xp, vp;
                predict_dim(ld_state<true>(S.x[c] + i), ld_state<true>(S.v[c] + i), ld_state<true>(S.a[c] + i),
                            ld_state<true>(S.k[c] + i), pd, xp, vp);
                const float h = d2f_rn(xp);
                dst[c * stride + base + k] = h;
                dst[(4 + c) * stride + base + k] = d2f_rn(vp);
                if (DSW) dst[(7 + c) * stride + base + k] = d2f_rn(xp - f2d(h));  // the difference is exact
            }
        }
    };
    long long done = 0, rows = 0, last_t = A.last_t, predicted = -1;
    unsigned long long tb = ~0ull;
    int na = 0;
    for (;;) {
        // 1. this CTA's earliest due tick, its particles due then (ascending), published
        unsigned long long m = ~0ull;
        for (int k = tid; k < nown; k += kGrThreads) m = due_c[k] < m ? due_c[k] : m;
        m = block_reduce(m, MinOp(), red_u64, ~0ull);
        int cnt = 0;
        for (int base = 0; base < nown; base += kGrThreads) {
            const int k = base + tid;
            const bool h = k < nown && due_c[k] == m;
            const unsigned mask = __ballot_sync(0xffffffffu, h);
            if (lane == 0) warp_tot[warp] = __popc(mask);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < kGrWarps; ++w) {
                before += w < warp ? warp_tot[w] : 0;
                total += warp_tot[w];
            }
            if (h) {
                const int slot = cnt + before + __popc(mask & ((1u << lane) - 1u));
                if (NB_CHECK(slot < CH, A.st, 7)) own[slot] = lo + k;
            }
            cnt += total;
            __syncthreads();  // warp_tot is read before the next round stores it
        }
        if (tid == 0) {
            A.pub[g].m = m;
            A.pub[g].cnt = cnt;
            A.pub[g].flags = __ldcg(&A.st->flags);
        }
        if (A.skip_arrival && done == 0 && g == G - 1) break;
        if (!barrier()) break;

        // 2. the block time and size, where this CTA's rows start, the decision (all alike)
        if (warp == 0) {
            unsigned long long mm = ~0ull;
            for (int r = lane; r < G; r += 32) {
                const unsigned long long v = __ldcg(&A.pub[r].m);
                mm = v < mm ? v : mm;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long v = __shfl_xor_sync(0xffffffffu, mm, o);
                mm = v < mm ? v : mm;
            }
            int before = 0, total = 0;
            unsigned fl = 0;
            for (int r = lane; r < G; r += 32) {
                const int c = __ldcg(&A.pub[r].m) == mm ? __ldcg(&A.pub[r].cnt) : 0;
                total += c;
                before += r < g ? c : 0;
                fl |= __ldcg(&A.pub[r].flags);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                total += __shfl_xor_sync(0xffffffffu, total, o);
                before += __shfl_xor_sync(0xffffffffu, before, o);
                fl |= __shfl_xor_sync(0xffffffffu, fl, o);
            }
            if (lane == 0) {
                s_tb = mm;
                s_na = total;
                s_off = before;
                s_flags = fl;
            }
        }
        __syncthreads();
        tb = s_tb;
        na = s_na;
        const int off = s_off;
        const int mine = m == tb ? cnt : 0;
        const bool go = done < A.budget && (s_flags & A.stop_flags) == 0u && static_cast<long long>(tb) <= A.t_end &&
                        na > 0 && na <= RM;
        for (int q = tid; q < mine; q += kGrThreads)
            if (NB_CHECK(off + q < n, A.st, 8)) A.act_out[off + q] = own[q];
        if (!go) {
            if (done < A.budget && (s_flags & A.stop_flags) == 0u && static_cast<long long>(tb) <= A.t_end &&
                na > RM) {  // the separate kernels run this block: leave them the prediction
                predict_own(tb, A.soa, A.n_pad, lo);
                predicted = static_cast<long long>(tb);
            }
            break;
        }
        predict_own(tb, jsm, SJ, 0);  // this CTA's particles predicted to tb, into shared memory
        __syncthreads();
        for (int q = tid; q < mine; q += kGrThreads) {  // the rows' predicted data for every CTA
            const int k = own[q] - lo;
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a != 3 && NB_CHECK(off + q < RM, A.st, 9))
                    A.ri[(a < 3 ? a : a - 1) * RM + off + q] = jsm[a * SJ + k];
        }
        if (!barrier()) break;

        // 3. the pair terms of every row of the block over this CTA's particles: one partial per row
        {
            // T threads per row: the largest power of two with T na <= threads and at
            // least two groups of 4 j per thread (a CTA without particles stores zeros)
            int T = kGrThreads;
            while (T > 1 && (T * na > kGrThreads || 8 * T > L)) T >>= 1;
            auto load_i = [&](const int rr, const bool live, I2 &I) {
                const int p = live ? rr : 0;
                const float *r = A.ri + p;
                const float x = __ldcg(r), y = __ldcg(r + RM), z = __ldcg(r + 2 * RM);
                const float vx = __ldcg(r + 3 * RM), vy = __ldcg(r + 4 * RM), vz = __ldcg(r + 5 * RM);
                I.x = f2_pack(x, x);
                I.y = f2_pack(y, y);
                I.z = f2_pack(z, z);
                I.vx = f2_pack(vx, vx);
                I.vy = f2_pack(vy, vy);
                I.vz = f2_pack(vz, vz);
                if (DSW) {
                    const float lx = __ldcg(r + 6 * RM), ly = __ldcg(r + 7 * RM), lz = __ldcg(r + 8 * RM);
                    I.lx = f2_pack(lx, lx);
                    I.ly = f2_pack(ly, ly);
                    I.lz = f2_pack(lz, lz);
                }
                return live ? __ldcg(A.act_out + p) : -1;
            };
            auto no_ds = [](const int, const bool, dsa::ds (&)[3], dsa::ds (&)[3]) { return -1; };
            auto store = [&](const int rr, const float *tot, const float *lw) {
                float *d = A.part + (static_cast<size_t>(rr) * G + g) * PW;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    d[c] = tot[c];
                    if (DSW) d[6 + c] = lw[c];
                }
            };
            rows_force<MODE, kGrThreads, SJ>(jsm, SJ, lo, L, na, T, A.eps2, 0.0f, load_i, no_ds, store, wred);
        }
        if (!barrier()) break;

        // 4. this CTA's rows: their G partials added in CTA order, then corrected
        for (int q0 = 0; q0 < mine; q0 += kGrThreads) {
            const int cq = min(kGrThreads, mine - q0);
            for (int k = warp; k < cq; k += kGrWarps) {  // one warp per row
                const float *src = A.part + static_cast<size_t>(off + q0 + k) * G * PW;
                float h[6], l[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) h[c] = l[c] = 0.0f;
                for (int r0 = 0; r0 < G; r0 += 96) {  // lane takes CTAs lane, lane + 32, ...: three loaded at once
                    float x[3][PW];
#pragma unroll
                    for (int u = 0; u < 3; ++u) {
                        const int r = r0 + 32 * u + lane;
#pragma unroll
                        for (int c = 0; c < PW; ++c) x[u][c] = r < G ? __ldcg(src + r * PW + c) : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 3; ++u)
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            if (DSW)
                                ds2_add(h[c], l[c], x[u][c], x[u][6 + c]);
                            else
                                h[c] = __fadd_rn(h[c], x[u][c]);
                        }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, h[c], o);
                        if (DSW) {
                            const float l2 = __shfl_xor_sync(0xffffffffu, l[c], o);
                            ds2_add(h[c], l[c], h2, l2);
                        } else {
                            h[c] = __fadd_rn(h[c], h2);
                        }
                    }
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        f_hi[k][c] = h[c];
                        f_lo[k][c] = l[c];
                    }
            }
            __syncthreads();
            auto due = [&](const int, const int r, const unsigned long long dd) {
                if (NB_CHECK(r >= lo && r - lo < nown, A.st, 10)) due_c[r - lo] = dd;
            };
            rows_correct<DSW>(S, own + q0, f_hi, f_lo, cq, tb, A.tick, A.eta, A.lmin, A.lmax, A.st, due);
            __syncthreads();
        }
        ++done;
        rows += na;
        last_t = static_cast<long long>(tb);
    }
    if (g == 0 && tid == 0) {
        A.sched_out->t_blk = static_cast<long long>(tb);
        A.sched_out->n_act = na;
        A.L->blocks = done;
        A.L->rows = rows;
        A.L->last_t = last_t;
        A.L->predicted = predicted;
    }
}


// CTAs of the mode's launch on this device (one per SM), or 0 when it cannot
// launch cooperatively with the largest shared memory; found once per mode.
template <int MODE>
int grid_size_for()
{
    static const int size = [] {
        int dev = 0, coop = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || !coop) {
            cudaGetLastError();
            return 0;
        }
        auto kern = grid_step_kernel<MODE, kGrMaxChunk>;
        const size_t smem = gr_smem<MODE, kGrMaxChunk>();
        int per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGrThreads, smem) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            return 0;
        }
        return sms;
    }();
    return size;
}

// Launches the instance of stride SJ (its shared-memory limit raised once).
template <int MODE, int SJ>
cudaError_t launch_sj(cudaLaunchConfig_t cfg, const GrArgs &A)
{
    static const cudaError_t set = cudaFuncSetAttribute(grid_step_kernel<MODE, SJ>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        static_cast<int>(gr_smem<MODE, SJ>()));
    if (set != cudaSuccess) return set;
    cfg.dynamicSmemBytes = gr_smem<MODE, SJ>();
    return cudaLaunchKernelEx(&cfg, grid_step_kernel<MODE, SJ>, A);
}
template <int MODE>
cudaError_t launch_mode(const cudaLaunchConfig_t &cfg, const GrArgs &A)
{
    if (A.chunk <= kGrStrides[0]) return launch_sj<MODE, kGrStrides[0]>(cfg, A);
    if (A.chunk <= kGrStrides[1]) return launch_sj<MODE, kGrStrides[1]>(cfg, A);
    if (A.chunk <= kGrStrides[2]) return launch_sj<MODE, kGrStrides[2]>(cfg, A);
    return launch_sj<MODE, kGrStrides[3]>(cfg, A);
}

// The scratch: barrier counter, published records, row buffer, partials, each
// starting on a 256-byte boundary; returns the bytes and fills the offsets.
size_t grid_layout(const int mode, const int rows_max, const int ctas, size_t off[4])
{
    const size_t na = mode == kModeComp ? SoaTile<kModeComp>::NA : SoaTile<kModePlain>::NA;
    const size_t pw = mode == kModeComp ? 12 : 6;
    const size_t rm = static_cast<size_t>(rows_max);
    const size_t sizes[4] = {sizeof(unsigned long long), sizeof(GrPub) * static_cast<size_t>(ctas),
                             sizeof(float) * (na - 1) * rm, sizeof(float) * pw * rm * static_cast<size_t>(ctas)};
    size_t at = 0;
    for (int q = 0; q < 4; ++q) {
        off[q] = at;
        at += (sizes[q] + 255) & ~size_t(255);
    }
    return at;
}

}  // namespace

int grid_step_size(int mode)
{
    if (mode == kModePlain) return grid_size_for<kModePlain>();
    if (mode == kModeComp) return grid_size_for<kModeComp>();
    return 0;
}

int grid_step_chunk(int64_t n, int ctas)
{
    if (ctas <= 0) return 0;
    const int64_t ch = ((n + ctas - 1) / ctas + 3) & ~int64_t(3);
    return ch <= kGrMaxChunk ? static_cast<int>(ch) : 0;
}

size_t grid_step_bytes(int mode, int rows_max, int ctas)
{
    size_t off[4];
    return grid_layout(mode, rows_max, ctas, off);
}

cudaError_t grid_step_launch(int mode, const State &S, const JStream &J, double eps2, double eta, int lmin, int lmax,
                             long long t_end, long long budget, int rows_max, long long last_t, unsigned stop_flags,
                             DevStatus *st, SchedOut *sched_out, StepLoop *L, int32_t *act_out, void *buf,
                             cudaStream_t s, int64_t *launches)
{
    const int G = grid_step_size(mode);
    const int CH = grid_step_chunk(S.n, G);
    if (G == 0 || CH == 0 || rows_max < 1 || !J.soa || !buf) return cudaErrorInvalidValue;
    GrArgs A;
    A.S = S;
    A.soa = J.soa;
    A.n_pad = J.n_pad;
    A.mass_j = J.soa + 3 * J.n_pad;
    A.chunk = CH;
    A.rows_max = rows_max;
    A.eps2 = static_cast<float>(eps2);
    A.tick = ldexp(1.0, -lmax);
    A.eta = eta;
    A.lmin = lmin;
    A.lmax = lmax;
    A.t_end = t_end;
    A.budget = budget;
    A.last_t = last_t;
    A.stop_flags = stop_flags;
    A.skip_arrival = g_skip_first_copy;
    A.st = st;
    A.sched_out = sched_out;
    A.L = L;
    A.act_out = act_out;
    size_t off[4];
    grid_layout(mode, rows_max, G, off);
    unsigned char *p = static_cast<unsigned char *>(buf);
    A.bar = reinterpret_cast<unsigned long long *>(p + off[0]);
    A.pub = reinterpret_cast<GrPub *>(p + off[1]);
    A.ri = reinterpret_cast<float *>(p + off[2]);
    A.part = reinterpret_cast<float *>(p + off[3]);
    cudaError_t e = cudaMemsetAsync(A.bar, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kGrThreads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = mode == kModeComp ? launch_mode<kModeComp>(cfg, A) : launch_mode<kModePlain>(cfg, A);
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace nb

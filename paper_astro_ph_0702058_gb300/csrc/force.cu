// Launch-shape choice and launch of the force evaluation (kernels in force_impl.cuh).
#include <atomic>
#include <algorithm>
#include <cmath>

#include "force_slice.cuh"
#include "force_x2.cuh"

// Block sizes the automatic shape gives the slice shape (packed plain and
// compensated modes, streams of kJSubMinTiles tiles or more).
#ifndef NB_SLICE_MIN_ROWS
#define NB_SLICE_MIN_ROWS 512
#endif
#ifndef NB_SLICE_MAX_ROWS
#define NB_SLICE_MAX_ROWS 8191
#endif

namespace nb {

cudaError_t force_dispatch_plain(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s);
cudaError_t force_dispatch_comp(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s);
int force_occupancy_plain(int threads, int ipt);
int force_occupancy_comp(int threads, int ipt);
cudaError_t reduce_plain(const float *part, int split, int n_act, double *acc, double *jerk, double *pot,
                         cudaStream_t s, const long long *n_act_dev);
cudaError_t reduce_comp(const float *part, int split, int n_act, double *acc, double *jerk, double *pot,
                        cudaStream_t s, const long long *n_act_dev);
cudaError_t force_dispatch_check(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s);
int force_occupancy_check(int threads, int ipt);
cudaError_t reduce_check(const float *part, int split, int n_act, double *acc, double *jerk, double *pot,
                         cudaStream_t s, const long long *n_act_dev);

int g_skip_first_copy = 0;  // test hook (nbody_debug_skip_tile_copy)

bool force_needs_aos(int mode)
{
    return !NB_PACKED || mode == kModeDS || mode == kModeSorted;
}

bool force_reads_device_rows(int mode)
{
    return NB_PACKED && (mode == kModePlain || mode == kModeComp);
}

namespace {

int shape_index(int threads, int ipt)
{
    if (ipt < 0) return threads == kJSubThreads ? 10 : -1;  // the j-subgroup shape
    if (threads == 512) return ipt == 1 ? 9 : -1;  // one i per thread only
    const int ti = threads == 64 ? 0 : threads == 128 ? 1 : threads == 256 ? 2 : -1;
    const int ii = ipt == 1 ? 0 : ipt == 2 ? 1 : ipt == 4 ? 2 : -1;
    return (ti < 0 || ii < 0) ? -1 : ti * 3 + ii;
}

// Resident blocks per SM of each compiled kernel (queried once per process;
// every device this library runs on is the same sm_103 part).
int occupancy(int mode, int threads, int ipt)
{
    static std::atomic<int> cache[5][11];  // resident blocks + 1; 0 until queried (host threads may race: same value)
    const int si = shape_index(threads, ipt);
    if (si < 0 || mode < 0 || mode > 4) return 0;
    int v = cache[mode][si].load(std::memory_order_acquire);
    if (v == 0) {
        v = 1 + (mode == kModeComp    ? force_occupancy_comp(threads, ipt)
                 : mode == kModeCheck ? force_occupancy_check(threads, ipt)
                 : mode == kModeDS    ? force_occupancy_ds()
                 : mode == kModeSorted ? 1
                                      : force_occupancy_plain(threads, ipt));
        cache[mode][si].store(v, std::memory_order_release);
    }
    return v - 1;
}

}  // namespace

int force_choose(int mode, int64_t n_act, int64_t n_pad, int sm_count, int req_threads, int req_ipt,
                 int req_split, ForceConfig *cfg, int req_jsub)
{
    const int n_tiles = static_cast<int>(n_pad / kJTile);
    // the slice shape: one CTA per SM over its slice of the stream, for mid-size blocks when the
    // caller fixes no parameter and the slice fits shared memory
    if (NB_PACKED && (mode == kModePlain || mode == kModeComp) && req_threads == 0 && req_ipt == 0 &&
        req_split <= 0 && req_jsub == 0 && n_act >= NB_SLICE_MIN_ROWS && n_act <= NB_SLICE_MAX_ROWS &&
        n_tiles >= kJSubMinTiles && slice_chunk(n_pad, sm_count) > 0) {
        cfg->threads = kSliceThreads;
        cfg->ipt = 1;
        cfg->jsub = 1;
        cfg->split = sm_count;
        cfg->tiles_per_split = 0;
        cfg->n_iblk = 1;
        cfg->slice = 1;
        return NBODY_OK;
    }
    int threads = req_threads;
    int ipt = req_ipt;
    // j-subgroups: blocks of kJSubMinRows to 8191 rows in the packed plain and compensated
    // modes take 256 threads as 64 rows x 4 subgroups, unless the caller fixes a shape
    // (for streams of kJSubMinTiles tiles or more: at small n a block is all latency).
    // Smaller blocks keep 64 threads, one per row: their time is one range's latency, and
    // one shape for all of them lets the block-step graph take them all.
    const bool jsub_ok = NB_PACKED && (mode == kModePlain || mode == kModeComp);
    const bool jsub = jsub_ok && (req_jsub == kJSub || (req_jsub == 0 && req_threads == 0 && req_ipt == 0 &&
                                                        n_act >= kJSubMinRows && n_act < 8192 &&
                                                        n_tiles >= kJSubMinTiles));
    if (req_jsub > 1 && (!jsub_ok || req_jsub != kJSub)) return NBODY_EINVAL;
    if (jsub) {
        threads = kJSubThreads;
        ipt = -1;  // the occupancy / shape key of the j-subgroup instance
    }
    // Packed loop: one i per thread keeps registers low (74 plain, 94
    // compensated) and resident warps high, which beats amortising the shared
    // loads over 2 or 4 i (134-252 registers).  At N = 2^20, in Tpairs/s:
    // plain 1.26 (256 x 1), 1.24 (128 x 1), 1.23 (128 x 2), 1.22 (128 x 4);
    // compensated 1.05, 1.03, 0.98, 0.97.  Small blocks take 64 threads so
    // that more blocks of fewer rows fill the GPU.
    if (mode == kModeDS) {  // one shape: 128 threads, one i each
        threads = 128;
        ipt = 1;
    }
    if (threads == 0) threads = n_act >= 8192 ? 256 : 64;
    if (ipt == 0) ipt = 1;
    if (shape_index(threads, ipt) < 0) return NBODY_EINVAL;
    const int per = jsub ? kJSubThreads / kJSub : threads * ipt;  // rows of a block
    const int n_iblk = static_cast<int>(std::max<int64_t>(1, (n_act + per - 1) / per));
    int split = req_split;
    if (split <= 0) {
        // At least one full wave of blocks; among a few larger splits take the
        // one whose last wave is fullest (fewer idle SMs at the end).
        const int slots = sm_count * std::max(1, occupancy(mode, threads, ipt));
        const int smin = std::max(1, (slots + n_iblk - 1) / n_iblk);
        auto eff = [&](int s) {
            const double waves = static_cast<double>(n_iblk) * s / slots;
            return waves / std::ceil(waves);
        };
        split = smin;
        double best = eff(smin);
        for (int s = smin + 1; s <= smin + 15; ++s) {
            const double e = eff(s);
            if (e > best + 0.02) {
                best = e;
                split = s;
            }
        }
    }
    split = std::max(1, std::min(split, n_tiles));
    if (req_split <= 0) {
        // More, shorter blocks balance the SMs better at the end of a launch:
        // +0.5-2 % for full forces, 10-20 % for blocks of 1k-2k rows at
        // N = 65536, up to about 12 waves.  The partial sums cost 28-56 bytes
        // per row and range, at most 12 x slots x threads x 56 bytes (~80 MB).
        const int slots = sm_count * std::max(1, occupancy(mode, threads, ipt));
        const int64_t want = (12LL * slots + n_iblk - 1) / n_iblk;
        if (want > split) split = static_cast<int>(std::min<int64_t>(want, n_tiles));
        // ...but at least two tiles per range when that still fills a wave of
        // blocks, so that each block's double buffer overlaps a copy with
        // compute (at N = 65536, compensated: +1.4 % at 1024 rows, +2.3 % at
        // 1594, +6 % at 4096 over one tile); blocks too small to fill the GPU
        // keep one tile per range, since their time is the latency of one range
        if (n_tiles >= 2 && static_cast<int64_t>(n_iblk) * (n_tiles / 2) >= slots)
            split = std::min(split, n_tiles / 2);
    }
    if (req_split <= 0 && jsub) {
        // j-subgroup blocks are short: give each range 8, 4 or 2 tiles while the grid
        // still fills the GPU (8 only with six waves or more).  At N = 65536: 1024 and
        // 1594 rows fastest with 4 tiles (compensated 117 and 164 us, against 125 and 184
        // with 2), 4096 rows with 8.  One wave of longer ranges (the balanced ranges allow
        // any split) measured slower: 1024 rows compensated in 19 ranges of 13-14 tiles,
        // one wave of 304 blocks, took 131 us against 114 with 4-tile ranges in 3.4
        // waves; the block scheduler evening out SMs of unequal speed with many short
        // blocks gains more than a full last wave.
        const int64_t slots = static_cast<int64_t>(sm_count) * std::max(1, occupancy(mode, threads, ipt));
        int t = 1;
        if (n_tiles >= 8 && static_cast<int64_t>(n_iblk) * (n_tiles / 8) >= 6 * slots) t = 8;
        else if (n_tiles >= 4 && static_cast<int64_t>(n_iblk) * (n_tiles / 4) >= slots) t = 4;
        else if (n_tiles >= 2 && static_cast<int64_t>(n_iblk) * (n_tiles / 2) >= slots) t = 2;
        split = (n_tiles + t - 1) / t;
    }
    const int tps = (n_tiles + split - 1) / split;
    split = (n_tiles + tps - 1) / tps;  // the fewest ranges of that length
    cfg->threads = threads;
    cfg->ipt = jsub ? 1 : ipt;
    cfg->jsub = jsub ? kJSub : 1;
    cfg->slice = 0;
    cfg->split = split;
    cfg->tiles_per_split = tps;
    cfg->n_iblk = n_iblk;
    return NBODY_OK;
}

size_t force_partial_bytes(int mode, const ForceConfig &cfg, int64_t n_act)
{
    if (cfg.split <= 1 || mode == kModeSorted) return 0;
    const size_t nc = two_word_sums(mode) ? 14 : 7;
    return static_cast<size_t>(cfg.split) * nc * static_cast<size_t>(n_act) * sizeof(float);
}

bool force_partials_fused(int mode, const ForceConfig &cfg)
{
    return force_reads_device_rows(mode) && cfg.split > 1 && cfg.split < kFusedSplitMax;
}

cudaError_t force_launch(int mode, const JStream &js, int64_t n, const int32_t *active, int64_t n_act, double eps2_d,
                         const ForceConfig &cfg, double *acc, double *jerk, double *pot, void *partials,
                         DevStatus *st, cudaStream_t s, int64_t *launches, const long long *n_act_dev, bool reduce)
{
    if (n_act <= 0) return cudaSuccess;
    const float eps2 = static_cast<float>(eps2_d);
    if (mode == kModeDS) {
        cudaError_t e = force_ds_launch(js, n, active, n_act, eps2_d, cfg, acc, jerk, pot, partials, st, s);
        if (e != cudaSuccess) return e;
        ++*launches;
        if (cfg.split > 1) {
            e = reduce_comp(static_cast<float *>(partials), cfg.split, static_cast<int>(n_act), acc, jerk, pot, s,
                            nullptr);
            if (e != cudaSuccess) return e;
            ++*launches;
        }
        return cudaSuccess;
    }
    if (mode == kModeSorted) {
        const cudaError_t e = force_sorted_launch(js, n, active, n_act, eps2, acc, jerk, pot, st, s);
        if (e == cudaSuccess) ++*launches;
        return e;
    }
    const ForceConfig &c = cfg;
    ForceParams P;
    P.posm = js.posm;
    P.vel = js.vel;
    P.poslo = js.poslo;
    P.soa = js.soa;
    P.active = active;
    P.n_act = static_cast<int>(n_act);
    P.n_act_dev = n_act_dev;
    P.n = static_cast<int>(n);
    P.n_tiles = static_cast<int>(js.n_pad / kJTile);
    P.eps2 = eps2;
    P.acc = acc;
    P.jerk = jerk;
    P.pot = pot;
    P.part = static_cast<float *>(partials);
    P.st = st;
    P.skip_first_copy = g_skip_first_copy;
    P.opaque_zero = 0;
    cudaError_t e = mode == kModeComp    ? force_dispatch_comp(P, c, s)
                    : mode == kModeCheck ? force_dispatch_check(P, c, s)
                                         : force_dispatch_plain(P, c, s);
    if (e != cudaSuccess) return e;
    ++*launches;
    if (c.split > 1 && reduce) {
        e = mode == kModeComp    ? reduce_comp(P.part, c.split, P.n_act, acc, jerk, pot, s, n_act_dev)
            : mode == kModeCheck ? reduce_check(P.part, c.split, P.n_act, acc, jerk, pot, s, n_act_dev)
                                 : reduce_plain(P.part, c.split, P.n_act, acc, jerk, pot, s, n_act_dev);
        if (e != cudaSuccess) return e;
        ++*launches;
    }
    return cudaSuccess;
}

}  // namespace nb

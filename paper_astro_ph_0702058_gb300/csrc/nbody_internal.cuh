// Internal declarations shared by the translation units of libnbody.so.
// Not part of the public ABI (that is include/nbody.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "nbody.h"

namespace nb {

// Records the message that nbody_last_error() returns in this thread; returns code.
int report_error(int code, const char *msg);

// j-particles per shared-memory tile; the j-stream is padded with massless
// particles at the origin to a multiple of this, and j-ranges of the split
// force kernel start on tile boundaries.
constexpr int kJTile = 256;
constexpr float kPadPosition = 1e15f;  // coordinate of the massless padding particles
constexpr int kModePlain = NBODY_MODE_PLAIN;
constexpr int kModeComp = NBODY_MODE_COMP;
constexpr int kModeCheck = NBODY_MODE_SUMCHECK;
constexpr int kModeSorted = NBODY_MODE_SORTED;
constexpr int kModeDS = NBODY_MODE_DS;
constexpr int64_t kSortedMaxN = 32768;  // sorted mode: all j terms of a row fit in shared memory
// Modes of force_kernel that read the hi/lo position split and keep double-single sums.
__host__ __device__ constexpr bool is_ds(int mode) { return mode == kModeComp || mode == kModeCheck; }
// Modes whose j-range partial sums are (hi, lo) pairs (14 floats per row).
constexpr bool two_word_sums(int mode) { return is_ds(mode) || mode == kModeDS; }
// What the predictor writes besides (x_hi, m_hi) and v_hi: 1 = position lo parts, 2 = also the
// mass lo part (in poslo.w) and the velocity lo parts.
constexpr int predict_lo_parts(int mode) { return mode == kModeDS ? 2 : is_ds(mode) ? 1 : 0; }

// Device-side status word of a context (written by kernels, read by the host).
enum : unsigned {
    kFlagNonfinite = 1u,
    kFlagDtMin = 2u,
    kFlagTimeout = 4u,
    kFlagBadIndex = 8u,
    kFlagDebugBounds = 16u,  // -DNB_DEBUG builds: an internal index check failed (the access was skipped)
};

struct DevStatus {
    unsigned int flags;
    int bad_index;
    unsigned long long below_min;
    unsigned long long nonfinite;
    int debug_site;  // -DNB_DEBUG builds: which check failed (sites listed at NB_CHECK's uses)
};

// Device-side index checks of the debug build (-DNB_DEBUG): a failed check
// records kFlagDebugBounds and its site in the status word and skips the
// access; it never traps.  In other builds NB_CHECK is true and costs nothing.
#ifdef NB_DEBUG
__device__ __forceinline__ bool nb_debug_check(const bool ok, DevStatus *st, const int site)
{
    if (!ok) {
        atomicOr(&st->flags, static_cast<unsigned>(kFlagDebugBounds));
        st->debug_site = site;
    }
    return ok;
}
#define NB_CHECK(cond, st, site) nb_debug_check((cond), (st), (site))
#else
#define NB_CHECK(cond, st, site) true
#endif

// Tiles [b, e) of j-range r when n_tiles tiles are cut into `split` ranges whose lengths
// differ by at most one tile (every force kernel: range r = blockIdx.y of split = gridDim.y).
__host__ __device__ __forceinline__ void jrange_tiles(const int r, const int split, const int n_tiles, int &b, int &e)
{
    b = static_cast<int>(static_cast<long long>(r) * n_tiles / split);
    e = static_cast<int>(static_cast<long long>(r + 1) * n_tiles / split);
}

// FP64 master state, structure of arrays: component c of particle i is x[c][i].
struct State {
    int64_t n;
    const double *m;
    double *x[3];
    double *v[3];
    double *a[3];
    double *k[3];
    int64_t *t;     // ticks of dt_min = 2^-lmax
    int8_t *level;  // dt = 2^-level
};

// Predicted j-stream read by the force kernel (n_pad entries each).
// Entries n .. n_pad-1 are massless padding far from every particle.
struct JStream {
    float4 *posm;   // (x_hi, y_hi, z_hi, m)
    float4 *vel;    // (vx, vy, vz, 0)
    float4 *poslo;  // (x - x_hi, y - y_hi, z - z_hi, m - m_hi) rounded to float; compensated (m part 0) and DS modes
    float4 *vello;  // (vx - vx_hi, vy - vy_hi, vz - vz_hi, 0) rounded to float; DS mode
    // The same stream as structure of arrays, kSoaArrays x n_pad floats: x_hi, y_hi, z_hi, m_hi,
    // vx_hi, vy_hi, vz_hi, x_lo, y_lo, z_lo (lo parts in the compensated modes).  The packed
    // force kernel copies its tiles straight from here; NULL (no-alloc callers) means AoS only.
    float *soa;
    int64_t n_pad;
    bool aos;  // the predictor also writes posm, vel, poslo (vello): a kernel of the context reads them
};
constexpr int kSoaArrays = 10;

struct ForceConfig {
    int threads;          // threads per block
    int ipt;              // i-particles per thread
    int split;            // j-ranges (gridDim.y)
    int tiles_per_split;  // tiles of kJTile j in the longest range (lengths differ by at most one)
    int n_iblk;           // i-blocks (gridDim.x)
    int jsub = 1;         // threads per row, each taking 1/jsub of every tile (1 or 4)
    int slice = 0;        // 1: the slice shape (one CTA per SM, split = CTAs; force_slice.cuh)
};
// The j-subgroup shape: 256 threads, 64 rows of 4 subgroups (packed plain and compensated modes).
constexpr int kJSubThreads = 256;
constexpr int kJSub = 4;
constexpr int kJSubMinRows = 512;   // automatic shape: j-subgroups from this many rows on,
constexpr int kJSubMinTiles = 64;   // for streams of at least this many tiles (n >= 16384)

// ---- force.cu ----
extern int g_skip_first_copy;  // test hook: force kernels leave out their first tile copy

// Picks the launch shape for n_act active particles against n_pad j.
// req_* > 0 override the automatic choice.
// req_jsub: 0 automatic, 1 one thread per row, 4 four (256 threads, one i each).
int force_choose(int mode, int64_t n_act, int64_t n_pad, int sm_count, int req_threads,
                 int req_ipt, int req_split, ForceConfig *cfg, int req_jsub = 0);
// Whether this mode's force kernels honour ForceParams::n_act_dev (the packed kernels).
bool force_reads_device_rows(int mode);
// Scratch bytes needed for partial sums when cfg.split > 1 (0 otherwise).
size_t force_partial_bytes(int mode, const ForceConfig &cfg, int64_t n_act);
// Launches the force evaluation (and the fixed-order partial reduction when
// split > 1).  acc/jerk: n_act*3, pot: n_act, device doubles.  With n_act_dev
// (packed plain/compensated kernels only) the launch is sized for n_act rows
// and the kernels read the actual block size from *n_act_dev on the device.
// With reduce = false and force_partials_fused(mode, cfg) the j-range partial
// sums are left in `partials` for the corrector to add (correct_launch).
cudaError_t force_launch(int mode, const JStream &js, int64_t n, const int32_t *active,
                         int64_t n_act, double eps2, const ForceConfig &cfg, double *acc,
                         double *jerk, double *pot, void *partials, DevStatus *st,
                         cudaStream_t s, int64_t *launches, const long long *n_act_dev = nullptr,
                         bool reduce = true);
// Splits below this are added by the block-step corrector itself (in the order of
// the one-thread-per-row reduction), which saves a dependent kernel per block.
constexpr int kFusedSplitMax = 8;
// Whether a block step of this mode and shape hands its partials to the corrector.
bool force_partials_fused(int mode, const ForceConfig &cfg);

// ---- force_ds.cu ----
int force_occupancy_ds();
cudaError_t force_ds_launch(const JStream &js, int64_t n, const int32_t *active, int64_t n_act, double eps2,
                            const ForceConfig &cfg, double *acc, double *jerk, double *pot, void *partials,
                            DevStatus *st, cudaStream_t s);

// ---- force_sorted.cu ----
// One block per active row; terms sorted by size and added in FP32 (n <= kSortedMaxN).
cudaError_t force_sorted_launch(const JStream &js, int64_t n, const int32_t *active, int64_t n_act, float eps2,
                                double *acc, double *jerk, double *pot, DevStatus *st, cudaStream_t s);

// ---- integrator.cu ----
struct SchedOut;
// t_dev / sched_dev (graph replays): the time and block size are read on the device.
cudaError_t predict_launch(const State &S, const JStream &J, int64_t t_new, int lmax, int lo_parts,
                           cudaStream_t s, int64_t *launches, const long long *t_dev = nullptr);
// With `part` (split > 1), row q's forces are the sum of its j-range partials
// (part[split][7 or 14][n_act], two_word: hi and lo words), added in ascending
// range order in FP64 as the one-thread-per-row reduction does; acc, jerk unused.
cudaError_t correct_launch(const State &S, const int32_t *active, int64_t n_act,
                           const double *acc, const double *jerk, int64_t t_new, double eta,
                           int lmin, int lmax, DevStatus *st, cudaStream_t s, int64_t *launches,
                           const SchedOut *sched_dev = nullptr, const float *part = nullptr, int split = 0,
                           bool two_word = false);
// a, k <- the full force at t = 0 (acc, jerk: n*3), t <- 0, level from Eq. (initTimestep).
cudaError_t init_levels_launch(const State &S, const double *acc, const double *jerk,
                               double eta_init, int lmin, int lmax, DevStatus *st,
                               cudaStream_t s, int64_t *launches);

struct SchedOut {
    long long t_blk;
    long long n_act;
};
// Scratch for the scheduler: sched_scratch_bytes(n) bytes of device memory.
size_t sched_scratch_bytes(int64_t n);
cudaError_t schedule_launch(const State &S, int lmax, int32_t *active, SchedOut *out,
                            void *scratch, cudaStream_t s, int64_t *launches);

// Control block of a device-side loop over block steps (a while-node of a CUDA
// graph whose body is one block step): the host sets t_end, budget and last_t
// before a launch and reads blocks, rows and last_t after it.
struct StepLoop {
    long long t_end;   // ticks: a block due later does not run
    long long budget;  // blocks the loop may still add in this launch
    long long blocks;  // blocks it added
    long long rows;    // their active rows
    long long last_t;  // block time of the last block that ran
    long long predicted;  // whole-GPU block-step kernel: the tick it left the j-stream predicted to, or -1
};
// What the loop's decision reads: the next block (scheduled in the same body)
// runs when no flag of stop_flags is raised in st, it is due by L->t_end, its
// size na has 0 < na < n_fits and fits[na] != 0, and L->budget is left.
struct LoopArgs {
    cudaGraphConditionalHandle h;
    const unsigned char *fits;
    long long n_fits;
    const DevStatus *st;
    unsigned stop_flags;
    StepLoop *L;
};
// Last nodes of the loop body: the next block's schedule (as schedule_launch)
// and the loop's decision, which sets the condition of la.h (fused into the
// scheduler's kernel when it is one block, n <= 2048).
cudaError_t schedule_loop_launch(const State &S, int lmax, int32_t *active, SchedOut *out, void *scratch,
                                 const LoopArgs &la, cudaStream_t s, int64_t *launches);

// ---- cluster_step.cu ----
// Block steps of systems of n_pad <= kClMaxPad inside one thread-block cluster
// (16 CTAs where the device allows it, else 8): packed plain and compensated
// modes, and the double-single mode for n_pad <= kClMaxPadDS.  One launch runs blocks while the next one is due by t_end, budget is
// left, no flag of stop_flags is raised and its size is 1 .. rows_max; it writes
// L->blocks, rows, last_t, the next block's time and size to sched_out and its
// list to act_out (n ints).
constexpr int kClMaxPad = 4096;
constexpr int kClMaxPadDS = 2048;  // the double-single mode's copy of the j-stream takes 64 B per particle
constexpr int kClMaxChunk = 512;   // particles per CTA (n_pad / cluster size)
// The cluster size the mode's kernel launches with on this device, or 0 (no cluster launch).
int cluster_step_size(int mode);
cudaError_t cluster_step_launch(int mode, const State &S, const JStream &J, double eps2, double eta, int lmin,
                                int lmax, long long t_end, long long budget, long long rows_max, long long last_t,
                                unsigned stop_flags, DevStatus *st, SchedOut *sched_out, StepLoop *L,
                                int32_t *act_out, cudaStream_t s, int64_t *launches);

// ---- grid_step.cu ----
// Block steps of larger systems (n <= CTAs x kGrMaxChunk) as one cooperative
// launch of one CTA per SM, packed plain and compensated modes, with the same
// contract as cluster_step_launch; `buf` is grid_step_bytes(mode, rows_max,
// grid_step_size(mode)) bytes of device scratch.  When it stops at a block
// larger than rows_max (with budget left, due by t_end, no stop flag) it also
// leaves the j-stream (J.soa) predicted to that block's time and sets
// L->predicted to it (else -1), so the separate kernels can run the block
// without the predictor.
constexpr int kGrMaxChunk = 3584;  // particles per CTA (their prediction is held in shared memory)
// CTAs of the mode's launch on this device (one per SM), or 0 (no cooperative launch).
int grid_step_size(int mode);
// Particles per CTA for n (ceil(n / ctas) rounded up to 4), or 0 when above kGrMaxChunk.
int grid_step_chunk(int64_t n, int ctas);
size_t grid_step_bytes(int mode, int rows_max, int ctas);
cudaError_t grid_step_launch(int mode, const State &S, const JStream &J, double eps2, double eta, int lmin, int lmax,
                             long long t_end, long long budget, int rows_max, long long last_t, unsigned stop_flags,
                             DevStatus *st, SchedOut *sched_out, StepLoop *L, int32_t *act_out, void *buf,
                             cudaStream_t s, int64_t *launches);

// E_kin and E_pot (phi scratch: n doubles; out: 2 doubles); the potential in
// FP64 or, with ds_potential, in double-single arithmetic (energy_ds.cu).
cudaError_t energy_launch(const State &S, double eps2, double *phi_scratch, double *out,
                          cudaStream_t s, int64_t *launches, bool ds_potential = false);
// ---- energy_ds.cu ----
// phi_i = -sum_{j != i} m_j / sqrt(eps2 + |x_j - x_i|^2) in double-single arithmetic (n doubles).
cudaError_t phi_ds_launch(const State &S, double eps2, double *phi, cudaStream_t s, int64_t *launches);
// min and max of t over all particles (out: 2 unsigned long long).
cudaError_t time_range_launch(const State &S, unsigned long long *out, cudaStream_t s,
                              int64_t *launches);

// Writes the masses of the j-stream (SoA and float4 forms) once, at set-up.
cudaError_t mass_jstream_launch(const State &S, const JStream &J, cudaStream_t s, int64_t *launches);
// posm, vel, poslo from the SoA stream (for readers of the float4 form when J.aos is off).
cudaError_t aos_from_soa_launch(const JStream &J, int64_t n, cudaStream_t s, int64_t *launches);
// Whether this mode's kernels read the float4 j-stream (the predictor must write it).
bool force_needs_aos(int mode);

// Fills j-stream entries n .. n_pad-1 with massless particles at kPadPosition.
cudaError_t pad_jstream_launch(const JStream &J, int64_t n, cudaStream_t s, int64_t *launches);
// a[i] = i for 0 <= i < n.
cudaError_t iota_launch(int32_t *a, int64_t n, cudaStream_t s, int64_t *launches);

// ---- adjoint.cu: reverse mode of a shared-step rollout ----
struct DiffGrads {
    double *gx[3], *gv[3], *ga[3], *gk[3];  // gradients of the state (x, v, a, k), SoA
    double *gxp[3], *gvp[3];                // gradients of the predicted x, v
    double *gm;                             // gradient of the masses
    float4 *gA, *gK;                        // upstream of the force (n_pad, zero padded)
};
// Doubles of scratch the force VJP needs for its j-range partial sums (0: none).
size_t vjp_scratch_doubles(int64_t n, int64_t n_pad, int sm_count);
cudaError_t force_vjp_launch(const JStream &J, const DiffGrads &G, int64_t n, float eps2, int sm_count,
                             double *scratch, cudaStream_t s, int64_t *launches);
cudaError_t adj_correct_launch(const DiffGrads &G, int64_t n, double dt, cudaStream_t s, int64_t *launches);
cudaError_t adj_predict_launch(const DiffGrads &G, int64_t n, double dt, cudaStream_t s, int64_t *launches);
cudaError_t adj_init_launch(const DiffGrads &G, int64_t n, cudaStream_t s, int64_t *launches);
cudaError_t loss_launch(const State &S, double eps2, const DiffGrads &G, double *lval, double *loss,
                        cudaStream_t s, int64_t *launches);
cudaError_t set_time_launch(const State &S, int64_t tick, int level, cudaStream_t s, int64_t *launches);

// Row-major n x 3 <-> three component arrays.
cudaError_t aos_to_soa_launch(const double *aos, double *c0, double *c1, double *c2, int64_t n,
                              cudaStream_t s, int64_t *launches);
cudaError_t soa_to_aos_launch(const double *c0, const double *c1, const double *c2, double *aos,
                              int64_t n, cudaStream_t s, int64_t *launches);

}  // namespace nb

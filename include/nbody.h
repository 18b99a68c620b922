/*
 * nbody.h -- C ABI of libnbody.so, a GB300 (sm_103a) implementation of the
 * direct-summation force evaluation inside the 4th-order Hermite
 * predictor-corrector with power-of-two block time steps of Portegies Zwart,
 * Belleman & Geldof (2007), "High Performance Direct Gravitational N-body
 * Simulations on Graphics Processing Units".
 *
 * The calls follow the paper's statement of one integration step (Sect. 2,
 * the bulleted step list): choose the block of particles with the smallest
 * t_i + dt_i (nbody_next_block), predict every particle to the block time
 * (nbody_predict), recompute acceleration, jerk and potential of the block
 * (nbody_force), and correct the block to fourth order with new time steps
 * (nbody_correct).
 *
 * Conventions used by every call:
 *   - Units: G = 1.  eps2 is the square of the Plummer softening length
 *     (Appendix A: r^2 = eps^2 + |x_j - x_i|^2).
 *   - Vectors exchanged with the caller are n x 3 row-major arrays of double
 *     (x0 y0 z0 x1 y1 z1 ...).  Index lists are int32, 0 <= i < n.
 *   - Time steps are powers of two, dt = 2^-level with
 *     lmin <= level <= lmax (dt_max = 2^-lmin, dt_min = 2^-lmax; the paper
 *     uses dt_min = 2^-26).  Time is counted internally in int64 ticks of
 *     dt_min; a time passed in as a double must be a whole number of ticks.
 *   - Pointers: every pointer argument may point to host memory or to device
 *     memory of the context's device (detected with cudaPointerGetAttributes),
 *     unless stated otherwise.  The caller keeps ownership of all its
 *     buffers; the library copies inputs, writes outputs, and holds no caller
 *     pointer after a call returns.
 *   - Streams: all device work of a context runs on the stream given in
 *     nbody_params.stream (NULL: the legacy default stream).  A call that
 *     returns data in host memory synchronises that stream before it returns;
 *     a call whose outputs are device memory or NULL returns without waiting.
 *   - Errors: every int-returning call returns NBODY_OK (0) or a negative
 *     NBODY_E* code and never aborts the process.  nbody_strerror() gives a
 *     static description of a code; nbody_last_error() the detailed message
 *     of the most recent failure in the calling thread.
 *   - A context is not thread-safe: serialise calls on one context.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NBODY_ABI_VERSION 1

enum {
    NBODY_OK = 0,
    NBODY_EINVAL = -1,     /* bad argument (null where required, out of range, bad time) */
    NBODY_ENOMEM = -2,     /* device or pinned-host allocation failed                       */
    NBODY_ECUDA = -3,      /* a CUDA runtime call failed (message in nbody_last_error)       */
    NBODY_EDTMIN = -4,     /* strict mode: a criterion asked for dt < dt_min                  */
    NBODY_ENONFINITE = -5, /* a corrected state or force was NaN or infinite                  */
    NBODY_ENOTSYNC = -6,   /* energy requested while particles sit at different times         */
    NBODY_ETIMEOUT = -7,   /* a bounded device-side wait gave up (error flag, no hang)       */
    NBODY_ESTATE = -8      /* call out of order (e.g. correct without a matching force)      */
};

/* Force-evaluation precision (the pair loop; FP64 everywhere else). */
enum {
    NBODY_MODE_PLAIN = 0,  /* FP32 pair math on FP32 positions, FP32 accumulation           */
    NBODY_MODE_COMP = 1,   /* FP32 pair math on x_j - x_i formed from hi/lo splits of the
                              FP64 positions; double-single (compensated) accumulation      */
    NBODY_MODE_SUMCHECK = 2, /* test mode for the compensated summation: the production
                              kernel's tiles, j-ranges and packed pair loop with the pair term
                              of NBODY_MODE_COMP formed with the correctly rounded reciprocal
                              square root and no contracted operations, so that every FP32 term
                              is reproducible on a CPU, and every term folded into the
                              double-single sums on its own (the production mode sums 128
                              terms in FP32 first).  Slower; nbody_force / nbody_step only
                              (not the ensemble or the no-alloc entry point).              */
    NBODY_MODE_SORTED = 3, /* ablation of the accumulation order (Sect. 6 of the paper): the
                              plain-mode FP32 pair terms, formed with correctly rounded
                              operations in a fixed order, sorted by magnitude per row and
                              component and added in FP32 from the smallest.  One block per
                              active particle; n <= 32768 (NBODY_EINVAL above).  nbody_force /
                              nbody_step only.                                              */
    NBODY_MODE_DS = 4      /* double-single pair arithmetic (~46 significant bits) on the
                              FP32 pipe: positions, velocities and masses as hi/lo splits of
                              the FP64 values, rsqrt seed plus one Newton step, every product
                              and sum double-single.  About 1e-12 from the FP64 definition;
                              roughly 10x the FP32 work of the compensated mode.  nbody_force /
                              nbody_step / nbody_diff_rollout only.                        */
};

typedef struct nbody_ctx nbody_ctx; /* opaque; owns all of its device memory */

typedef struct {
    double eta;       /* accuracy parameter nu of Eq. (timestep); the paper uses 0.01     */
    double eta_init;  /* nu of Eq. (initTimestep); <= 0 means "same as eta"               */
    int lmin;         /* dt_max = 2^-lmin (paper: 0.125, lmin = 3)                          */
    int lmax;         /* dt_min = 2^-lmax (paper: 2^-26, lmax = 26); 0 <= lmin <= lmax <= 40 */
    int mode;         /* NBODY_MODE_PLAIN, _COMP, _SUMCHECK, _SORTED or _DS                  */
    int strict;       /* nonzero: a step clamped at dt_min makes nbody_correct fail with
                         NBODY_EDTMIN (the step is still taken); zero: it is only counted */
    int i_block;      /* force tuning, 0 = automatic (1): i-particles per thread (1, 2, 4)  */
    int j_tile;       /* force tuning, 0 = automatic (256 for blocks of >= 8192 rows, else
                         64): threads per block (64, 128, 256, or 512 with i_block 1)     */
    int j_split;      /* force tuning, 0 = automatic (about 12 waves of blocks): number of
                         j-ranges (>= 1); the double-single mode always takes 128 x 1     */
    int j_sub;        /* force tuning, plain and compensated modes: 0 = automatic (4 for
                         blocks of 512 to 8191 rows when j_tile and i_block are 0, else 1);
                         1 = one thread per row; 4 = 256 threads as 64 rows x 4 threads,
                         each taking a quarter of every j-tile (j_tile, i_block ignored).
                         With all four force-tuning fields 0, blocks of 512 to 8191 rows of
                         streams of 16384 to 3584 x SMs particles take the slice shape
                         instead: one block of 512 threads per SM over its contiguous
                         slice of the j-stream held in shared memory, j_split = SMs       */
    void *stream;     /* cudaStream_t for all work of the context, or NULL                  */
} nbody_params;

/* Fills *p with the defaults: eta 0.01, eta_init = eta, lmin 6, lmax 26, plain
 * mode, not strict, automatic tuning, NULL stream. */
void nbody_default_params(nbody_params *p);

/* Start of a run (Sect. 2; initial time step Eq. initTimestep).
 * Creates a context on the current CUDA device for n >= 1 particles:
 * m[n] masses, x[n*3] positions, v[n*3] velocities (copied; host or device),
 * softening eps2 >= 0.  Computes the full force on all particles at t = 0
 * and each particle's first level from dt = eta_init |a| / |k|.
 * On success *out receives the context (free with nbody_free).
 * Errors: EINVAL (null pointer, n < 1 or n > 2^31 - 1, eps2 < 0, bad levels or
 * mode), ENOMEM, ECUDA, ENONFINITE (non-finite input or initial force). */
int nbody_init(nbody_ctx **out, int64_t n, const double *m, const double *x,
               const double *v, double eps2, const nbody_params *p);

/* Block scheduler (Sect. 2, first bullet): t_blk = min_i (t_i + dt_i); the
 * block is every i with t_i + dt_i == t_blk exactly, in ascending index.
 * Writes the block time (double) to *t_blk, its size to *n_act, and the list
 * to active[0 .. n_act) when active is not NULL (room for n entries needed).
 * Synchronises the context stream.  Errors: EINVAL (null t_blk / n_act). */
int nbody_next_block(nbody_ctx *ctx, double *t_blk, int64_t *n_act, int32_t *active);

/* Predictor (Sect. 2): x_p = x + v dt + a dt^2/2 + k dt^3/6 and
 * v_p = v + a dt + k dt^2/2 for ALL particles, dt = t - t_i, in FP64; stores
 * the predicted positions/velocities as the FP32 j-stream that nbody_force
 * reads.  t must be a whole number of ticks and >= every t_i.
 * Errors: EINVAL (t not on the tick grid or before some t_i). */
int nbody_predict(nbody_ctx *ctx, double t);

/* Force on the listed particles from all n predicted particles (Eq. Force with
 * the softened pair term of Appendix A; j = i excluded):
 *   a_i   = sum_j m_j dx / r^3
 *   k_i   = sum_j m_j (dv / r^3 - 3 (dx.dv) dx / r^5)
 *   phi_i = -sum_j m_j / r,    dx = x_j - x_i, dv = v_j - v_i, r^2 = eps2 + dx.dx
 * evaluated at the state of the last nbody_predict.  active[n_act] (host or
 * device) lists distinct or repeated indices; 0 <= n_act <= n.  Results for
 * row q (particle active[q]) go to acc[q*3..], jerk[q*3..], pot[q] when those
 * pointers are not NULL (host or device, double); they are always kept in the
 * context for nbody_correct.  Errors: EINVAL (index out of range is checked on
 * the device and reported here when outputs are host memory, else at the next
 * synchronising call), ESTATE (no prediction yet), ETIMEOUT. */
int nbody_force(nbody_ctx *ctx, const int32_t *active, int64_t n_act,
                double *acc, double *jerk, double *pot);

/* Corrector of Sect. 2 and the new time step of Eq. (timestep) for the listed
 * particles, which must be distinct.  Row q of the forces belongs to
 * active[q].  acc/jerk (n_act x 3, host or device) supply the forces at the
 * predicted state; both NULL means "the results of the last nbody_force",
 * which must then have had the same n_act.  The corrected step ends at the
 * time of the last nbody_predict.  New level: largest power of two <= the
 * criterion, clamped to [dt_min, dt_max]; it shrinks at once and grows by
 * one level at most, only when the new time is a multiple of twice the old
 * step.  Errors: EINVAL, ESTATE, ENONFINITE (state updated; flagged rows are
 * set to dt_min), EDTMIN (strict mode only). */
int nbody_correct(nbody_ctx *ctx, const int32_t *active, int64_t n_act,
                  const double *acc, const double *jerk);

/* Block steps (schedule -> predict -> force -> correct) until every particle
 * has reached t_end (a multiple of dt_max, >= the current time), or until
 * max_steps blocks have been taken (max_steps <= 0: no limit).  *n_steps
 * (may be NULL) receives the number of blocks taken.  Errors: as the calls
 * it makes; EINVAL when t_end is not a multiple of dt_max. */
int nbody_step(nbody_ctx *ctx, double t_end, int64_t max_steps, int64_t *n_steps);

/* Energy diagnostic at a synchronised time (every t_i equal):
 * E_kin = sum m v^2 / 2, E_pot = sum_i m_i phi_i / 2 with the softened phi_i
 * (j = i excluded), in FP64 on the device.  Synchronises the stream.
 * Errors: ENOTSYNC when the particles are not at one time. */
int nbody_energy(nbody_ctx *ctx, double *ekin, double *epot);

/* The same diagnostic with the potential in double-single arithmetic on the
 * FP32 pipe: positions, masses and eps2 split into (hi, lo) float pairs,
 * 1/r from the MUFU seed and one Newton step with a double-single residual,
 * each 256-particle tile's terms summed in double-single and the tile sums
 * in FP64.  Agrees with nbody_energy to ~1e-13 relative and avoids an FP64
 * square root and division per pair, which make nbody_energy take about a
 * minute at n = 2^20 on GB300.  E_kin is FP64 as in nbody_energy.
 * Synchronises the stream.  Errors: ENOTSYNC as nbody_energy. */
int nbody_energy_ds(nbody_ctx *ctx, double *ekin, double *epot);

/* Waits for all work of the context and reports device-side errors raised
 * since the last report: ETIMEOUT (a bounded wait gave up), EINVAL (an index
 * out of range in an active list), ENONFINITE (a non-finite corrected row),
 * EDTMIN (strict mode: a step clamped at dt_min).  Calls that synchronise
 * (nbody_next_block, nbody_energy, nbody_get_state, nbody_step, and
 * nbody_force with host outputs) report the same errors. */
int nbody_sync(nbody_ctx *ctx);

/* Checkpoint: copies the FP64 state into caller buffers (host or device;
 * any may be NULL): x, v, a, k (n x 3), t_tick (n, ticks of dt_min) and
 * level (n).  Synchronises the stream. */
int nbody_get_state(nbody_ctx *ctx, double *x, double *v, double *a, double *k,
                    int64_t *t_tick, int8_t *level);

/* Resume: overwrites the whole state from caller buffers (none may be NULL;
 * masses and eps2 stay those of nbody_init).  Requires every t_tick to be a
 * multiple of its step 2^(lmax - level) and lmin <= level <= lmax.
 * Invalidates the last prediction and force.  Errors: EINVAL. */
int nbody_set_state(nbody_ctx *ctx, const double *x, const double *v, const double *a,
                    const double *k, const int64_t *t_tick, const int8_t *level);

/* Copies the predicted j-stream of the last nbody_predict into caller
 * buffers (host or device; any may be NULL), n x 4 floats each:
 * posm = (x_hi, y_hi, z_hi, m_hi), vel = (vx_hi, vy_hi, vz_hi, 0) and, in the
 * compensated, summation-check and double-single modes, poslo = (x - x_hi,
 * y - y_hi, z - z_hi, m - m_hi) rounded to float (the mass part only in the
 * double-single mode; zeros in the plain and sorted modes).  Synchronises the
 * stream.  Errors: ESTATE (no prediction). */
int nbody_get_predicted(nbody_ctx *ctx, float *posm, float *vel, float *poslo);

/* Counters of the context since nbody_init. */
typedef struct {
    int64_t n;             /* particles                                            */
    int64_t n_pad;         /* j-stream length (n rounded up to the tile length)    */
    int64_t blocks;        /* block steps corrected                                */
    int64_t below_dt_min;  /* steps clamped at dt_min                              */
    int64_t nonfinite;     /* corrected rows found non-finite                      */
    int64_t force_calls;   /* nbody_force calls                                    */
    int64_t pairs;         /* pair interactions evaluated: sum of n_act * (n - 1)  */
    int64_t kernel_launches; /* device kernels launched by the library            */
    int last_threads;      /* launch shape of the last force kernel               */
    int last_i_per_thread;
    int last_j_split;
    int mode;
    int64_t graph_blocks;  /* block steps nbody_step ran inside a replayed CUDA graph */
    int64_t loop_blocks;   /* of those, the ones the device-side loop added (no host round trip) */
    int last_j_sub;        /* threads per row of the last force kernel (1 or 4)    */
    int64_t cluster_blocks; /* block steps nbody_step ran in the one-cluster kernel */
    int64_t grid_blocks;   /* block steps nbody_step ran in the whole-GPU cooperative kernel */
} nbody_stats;

int nbody_get_stats(nbody_ctx *ctx, nbody_stats *s);

/* Releases every resource of the context (NULL is allowed). */
void nbody_free(nbody_ctx *ctx);

/* Static description of an NBODY_* code. */
const char *nbody_strerror(int code);

/* Detailed message of the last failure in this thread ("" if none). */
const char *nbody_last_error(void);

/* Test hook: the k-th device allocation from now fails with ENOMEM
 * (k >= 1; 0 disables).  Lets the out-of-memory paths be exercised. */
void nbody_debug_fail_alloc(int k);

/* Test hook: while on (nonzero), force kernels launched from this process do
 * not issue the copy of their first j-tile, so each block's bounded wait for
 * that tile gives up after about 2 s; the kernel records the timeout and
 * returns, and the call reports NBODY_ETIMEOUT.  Likewise the last CTA of the
 * whole-GPU block-step kernel (level 3 of nbody_debug_step_graphs) leaves
 * before its first grid barrier, whose bounded wait in the other CTAs gives up
 * after about 1 s.  Nothing faults or hangs and the context stays usable.
 * Exercises the failure path of the device waits. */
void nbody_debug_skip_tile_copy(int on);

/* Test switch for how nbody_step runs blocks small enough for one captured
 * CUDA graph (predictor, force, corrector, the next block's schedule, reading
 * the block time and size on the device):
 *   0  separate launches from the host for every block;
 *   1  one graph replay per block, then the host reads the next block back;
 *   2  the block step is the body of a device-side loop (a while-node
 *      of the graph): after each block's schedule one thread lets the next
 *      block run in the same replay while it is due by t_end, takes the
 *      graph's launch shape, no error flag is raised and the loop has added
 *      fewer than 1024 blocks to the replay's first; the host then reads back
 *      the next block.  Without while-nodes
 *      it acts as 1.
 *   3  (default) as 2, except that in the plain and compensated modes with
 *      n_pad <= 4096, and in the double-single mode with n_pad <= 2048, with
 *      automatic force shapes (j_tile, i_block, j_split, j_sub all 0), every
 *      block runs in one launch of a kernel of one
 *      thread-block cluster (16 or 8 CTAs) that repeats schedule, predictor,
 *      force and corrector on the device while the next block is due by
 *      t_end, no error flag is raised and max_steps allows (at most 4096
 *      blocks per launch).  Larger plain and compensated systems (n up to
 *      3584 per SM, automatic shapes) run their blocks of up to 4095 rows in
 *      one cooperative launch of one CTA per SM that repeats the same steps,
 *      its CTAs meeting at three grid barriers per block (each gives up after
 *      about 1 s and raises NBODY_ETIMEOUT); a larger block ends the launch
 *      and runs as at level 2.  Both kernels' forces are the same pair terms
 *      summed in another order, so their results differ from levels 0-2 in
 *      the last bits.
 * A context captures its graph in the form of the level in force when it
 * builds it (once, and again only if its scratch buffer moves); a loop graph
 * run at level 1 stops after each block.
 * The graph is used only when its launch shape is the one the separate
 * launches would take, so levels 0-2 give the same results bit for bit.
 * Values outside 0..3 are clamped. */
void nbody_debug_step_graphs(int level);

/* ------------------------------------------------------------ differentiation
 * Reverse mode of a shared-step rollout: the force of Eq. (Force) at t = 0,
 * then `steps` Hermite steps (Sect. 2 predictor and corrector) of one shared
 * step dt = 2^-level, in the precision `mode` (FP32 pair math, FP64 state).
 * Loss L = sum_i |x_i|^2 + E_pot at the end, E_pot the softened potential
 * energy (FP64).  Writes L to *loss and its gradients with respect to the
 * initial positions, velocities (n x 3) and masses (n) to g_x0, g_v0, g_m
 * (host or device).  The adjoint transposes the predictor and corrector and
 * applies a hand-written vector-Jacobian product of the pair force (FP32
 * pair math, FP64 totals); states are checkpointed every checkpoint_every
 * steps (<= 0: 16) and each segment is recomputed forward during the
 * backward sweep.  eps2 must be > 0.  Allocates its own scratch; waits.
 * Errors: EINVAL, ENOMEM, ECUDA, ENONFINITE. */
int nbody_diff_rollout(int64_t n, const double *m, const double *x0, const double *v0, double eps2,
                       int level, int64_t steps, int64_t checkpoint_every, int mode, double *loss,
                       double *g_x0, double *g_v0, double *g_m, void *stream);

/* The rollout above as a function (x0, v0, m) -> (x_T, v_T): the final
 * positions and velocities (n x 3, host or device; either may be NULL, not
 * both).  Allocates its own context; waits.  Errors: as nbody_diff_rollout. */
int nbody_rollout(int64_t n, const double *m, const double *x0, const double *v0, double eps2,
                  int level, int64_t steps, int mode, double *x_T, double *v_T, void *stream);

/* Vector-Jacobian product of nbody_rollout: given cotangents g_xT, g_vT of
 * the final positions and velocities (n x 3, host or device; NULL means
 * zero), writes g_x0 = (dx_T/dx0)^T g_xT + (dv_T/dx0)^T g_vT, and likewise
 * g_v0 (n x 3) and g_m (n) (host or device; NULL outputs are skipped, not all
 * three).  The same checkpointed reverse sweep as nbody_diff_rollout (the
 * transposed corrector and predictor of Sect. 2 and the hand-written
 * vector-Jacobian product of Eq. Force), seeded with the cotangents instead of
 * the loss gradient; the forward run is recomputed inside.  Errors: as
 * nbody_diff_rollout. */
int nbody_rollout_vjp(int64_t n, const double *m, const double *x0, const double *v0, double eps2,
                      int level, int64_t steps, int64_t checkpoint_every, int mode, const double *g_xT,
                      const double *g_vT, double *g_x0, double *g_v0, double *g_m, void *stream);

/* ---------------------------------------------------------------- ensembles
 * Many independent clusters integrated together: each cluster runs the block-
 * step scheme of Sect. 2 with its own schedule (its own t_blk and block), and
 * one batched step advances every unfinished cluster by one of its block
 * steps.  The batched step is five kernels sized from device-side counts (a
 * scheduler per cluster, a planner, the predictor, a persistent force kernel
 * working through a list of (cluster, i-block, j-range) items, the corrector),
 * so nbody_ens_run captures it once in a CUDA graph and replays it without a
 * host synchronisation per step. */
typedef struct nbody_ens nbody_ens; /* opaque; owns all of its device memory */

/* Creates an ensemble of n_clusters clusters on the current device.  sizes
 * [n_clusters] (host or device) gives each cluster's particle count (>= 1);
 * m, x, v hold all clusters' particles one after the other (cluster 0 first),
 * in the layout of nbody_init.  Every cluster starts at t = 0 with its full
 * force and first levels (Eq. initTimestep).  p as for nbody_init, except that
 * j_tile, i_block and j_split give the ensemble's force shape (threads per
 * block, i per thread, tiles per j-range; 0 = 64, 1, 4; see
 * nbody_ens_set_shape).  The ensemble runs on p->stream (which must allow
 * stream capture: not the legacy default stream) or, if that is NULL, on a
 * stream of its own.
 * Errors: EINVAL, ENOMEM, ECUDA, ENONFINITE. */
int nbody_ens_init(nbody_ens **out, int64_t n_clusters, const int64_t *sizes, const double *m,
                   const double *x, const double *v, double eps2, const nbody_params *p);

/* Force launch shape: threads per block (32, 64 or 128), i-particles per thread
 * (1 or 2), and j-tiles of 256 particles per work item (>= 1; each cluster is
 * cut into at most 8 j-ranges).  Errors: EINVAL for unsupported shapes. */
int nbody_ens_set_shape(nbody_ens *e, int threads, int i_block, int tiles_per_range);

/* Autotuner: times `steps` batched steps towards t_end for every supported
 * shape from the current state (restored after each trial), keeps the fastest
 * and returns it (any output may be NULL); best_ms is its time per batched
 * step.  The ensemble's state is unchanged. */
int nbody_ens_tune(nbody_ens *e, double t_end, int steps, int *threads, int *i_block,
                   int *tiles_per_range, double *best_ms);

/* One batched step towards t_end (a multiple of dt_max), without a graph;
 * *n_live receives the number of clusters that took a block step.  Waits. */
int nbody_ens_step(nbody_ens *e, double t_end, int64_t *n_live);

/* Batched steps through a CUDA graph until every cluster has reached t_end
 * (a multiple of dt_max); the host checks completion every check_every graph
 * launches (<= 0: 16).  *n_steps (may be NULL) receives the batched steps
 * that did work.  Waits.  The first call, and every call after a change of
 * t_end or shape, captures the graph on the ensemble's stream. */
int nbody_ens_run(nbody_ens *e, double t_end, int64_t check_every, int64_t *n_steps);

/* Per-cluster E_kin, E_pot (n_clusters each, host) at a time when every
 * particle of each cluster is at that cluster's common time; else ENOTSYNC. */
int nbody_ens_energy(nbody_ens *e, double *ekin, double *epot);

/* State of all particles in the layout of nbody_get_state (any may be NULL). */
int nbody_ens_get_state(nbody_ens *e, double *x, double *v, double *a, double *k,
                        int64_t *t_tick, int8_t *level);

/* Block steps taken and pair interactions (sum of n_act (N_c - 1) over its
 * blocks) evaluated per cluster since nbody_ens_init (n_clusters each, host;
 * may be NULL), and the number of kernels the ensemble has launched. */
int nbody_ens_get_stats(nbody_ens *e, int64_t *blocks_per_cluster, int64_t *pairs_per_cluster,
                        int64_t *kernel_launches);

void nbody_ens_free(nbody_ens *e);

/* Force on a list without any device allocation.  The paper has no
 * counterpart: this call serves callers that cannot allocate device memory
 * while they run (a host application that owns all GPU memory through its
 * own pool, code under a latency budget that cannot afford an allocation or
 * the synchronisation of a free, deployments whose footprint must be fixed
 * at load time).  It evaluates the same sums as nbody_force, with j = i
 * excluded, always with the j-range split and its partial sums held in a
 * fixed scratch array inside the library: 16 MiB of device memory that
 * every GPU loading the library holds until the process exits.
 *   posm, vel (and poslo in NBODY_MODE_COMP): the caller's predicted j-stream,
 *     16-byte aligned device memory of the current device, n_pad =
 *     256 * ceil(n / 256) entries of 4 floats each, in the layout
 *     nbody_get_predicted returns: (x, y, z, m), (vx, vy, vz, 0),
 *     (x_lo, y_lo, z_lo, 0).  Entries n .. n_pad-1 must have zero mass and lie
 *     away from every particle (the library pads with (1e15, 1e15, 1e15, 0)).
 *   active[n_act]: int32 indices in device memory of the current device,
 *     0 <= n_act <= 131072 (the scratch limit; larger blocks return
 *     NBODY_EINVAL).
 *   acc, jerk (n_act x 3), pot (n_act): 8-byte aligned device doubles of the
 *     current device, written.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls share the
 * scratch array: calls that
 * overlap on the GPU race, so serialise them.  The call waits for its work
 * on `stream` and returns NBODY_EINVAL (bad argument; a host, misaligned or
 * other-device pointer; index out of range), NBODY_ETIMEOUT or NBODY_ECUDA;
 * it never calls cudaMalloc, cudaFree or any allocating routine. */
int nbody_force_noalloc(const float *posm, const float *vel, const float *poslo, int64_t n,
                        const int32_t *active, int64_t n_act, double eps2, int mode,
                        double *acc, double *jerk, double *pot, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_H */

// Host side of the C ABI declared in include/nbody.h: context ownership,
// argument checks, host/device pointer handling, the block-step call
// sequence of Sect. 2 of Portegies Zwart, Belleman & Geldof (2007), and
// reporting of device-side status flags.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "nbody_internal.cuh"

using namespace nb;

namespace {

thread_local char g_err[512] = "";
int g_fail_alloc = 0;    // allocation-failure injection countdown (test hook)
// nbody_step's small blocks (test switch): 0 separate launches, 1 one graph
// replay per block, 2 a device-side loop of blocks in each replay
int g_step_graphs = 3;
constexpr int64_t kLoopCap = 1024;  // blocks one replay of the loop may run
constexpr int64_t kClusterCap = 4096;  // blocks one launch of the cluster or the grid kernel may run
#ifndef NB_GRID_ROWS
#define NB_GRID_ROWS 4095
#endif
constexpr int kGridRows = NB_GRID_ROWS;  // largest block the whole-GPU block-step kernel runs

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a sticky launch error of this thread
    return fail(e == cudaErrorMemoryAllocation ? NBODY_ENOMEM : NBODY_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define NB_CUDA(call, what)                         \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

cudaError_t dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (g_fail_alloc > 0 && --g_fail_alloc == 0) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes ? bytes : 16);
}

cudaError_t host_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (g_fail_alloc > 0 && --g_fail_alloc == 0) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, bytes ? bytes : 16);
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

int nb::report_error(int code, const char *msg)
{
    std::snprintf(g_err, sizeof g_err, "%s", msg);
    return code;
}

struct nbody_ctx {
    int64_t n = 0, n_pad = 0;
    double eps2 = 0.0;
    nbody_params p{};
    cudaStream_t s = nullptr;
    int sm_count = 0;

    double *state = nullptr;  // 13 n doubles: m, x[3], v[3], a[3], k[3]
    int64_t *t = nullptr;
    int8_t *level = nullptr;
    float4 *jbuf = nullptr;   // 4 n_pad float4 (posm, vel, poslo, vello), then kSoaArrays n_pad floats (SoA)
    int32_t *act_force = nullptr, *act_corr = nullptr, *act_sched = nullptr;
    double *f_acc = nullptr, *f_jerk = nullptr, *f_pot = nullptr;
    double *stage = nullptr;  // 6 n doubles: external forces / AoS staging
    void *partials = nullptr;
    size_t partials_cap = 0;
    void *sched_scratch = nullptr;
    SchedOut *sched_out = nullptr;
    DevStatus *st = nullptr;
    double *phi = nullptr;
    double *e_out = nullptr;
    unsigned long long *trange = nullptr;
    // pinned host mirrors
    SchedOut *sched_host = nullptr;
    DevStatus *st_host = nullptr;
    double *e_host = nullptr;
    unsigned long long *trange_host = nullptr;

    State S{};
    JStream J{};
    int64_t t_max = 0;      // largest t_i (ticks)
    int64_t t_pred = 0;     // time of the last prediction (ticks)
    // nbody_step's small-block graph: predict, force, correct, schedule the next block and read
    // it back, all sized for graph_rows rows and reading the block time and size on the device;
    // with graph_loop the block step is the body of a while-node that repeats it on the device
    // while the next block fits (graph_fits) and the loop control (loop_dev) allows
    cudaGraphExec_t step_graph = nullptr;
    int64_t graph_rows = 0;
    ForceConfig graph_cfg{};
    void *graph_partials = nullptr;
    int64_t graph_launches = 0;  // kernel nodes per block step of a replay
    bool graph_loop = false;
    unsigned char *graph_fits = nullptr;  // graph_rows + 1 flags: block size na takes the graph's shape
    StepLoop *loop_dev = nullptr;
    StepLoop *loop_host = nullptr;
    void *grid_buf = nullptr;  // scratch of the whole-GPU block-step kernel (grid_step_bytes)
    int grid_rows = 0;         // largest block it runs
    bool pred_valid = false;
    int64_t force_n_act = -1;
    int fused_split = 0;  // > 1: the last force left its j-range partials for the corrector
    nbody_stats stats{};
};

namespace {

void release(nbody_ctx *c)
{
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    void *dev[] = {c->state, c->t, c->level, c->jbuf, c->act_force, c->act_corr, c->act_sched,
                   c->f_acc, c->f_jerk, c->f_pot, c->stage, c->partials, c->sched_scratch,
                   c->sched_out, c->st, c->phi, c->e_out, c->trange, c->graph_fits, c->loop_dev, c->grid_buf};
    for (void *d : dev)
        if (d) cudaFree(d);
    void *host[] = {c->sched_host, c->st_host, c->e_host, c->trange_host, c->loop_host};
    for (void *h : host)
        if (h) cudaFreeHost(h);
    delete c;
}

int to_ticks(const nbody_ctx *c, double t, int64_t *out)
{
    const double tt = std::ldexp(t, c->p.lmax);
    if (!std::isfinite(tt) || tt < 0.0 || tt > 4.0e18 || tt != std::floor(tt))
        return fail(NBODY_EINVAL, "time %.17g is not a non-negative multiple of dt_min = 2^-%d", t, c->p.lmax);
    *out = static_cast<int64_t>(tt);
    return NBODY_OK;
}

// Copies n bytes from a host or device pointer into device memory.
cudaError_t to_device(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
}

// Reads the device status after the stream has drained and turns raised flags
// into an error code (the flags are then cleared; the counters keep counting).
int absorb_status(nbody_ctx *c)
{
    const DevStatus h = *c->st_host;
    c->stats.below_dt_min = static_cast<int64_t>(h.below_min);
    c->stats.nonfinite = static_cast<int64_t>(h.nonfinite);
    const unsigned f = h.flags;
    if (!f) return NBODY_OK;
    cudaMemsetAsync(&c->st->flags, 0, sizeof(unsigned), c->s);
    c->st_host->flags = 0;
    if (f & kFlagDebugBounds)
        return fail(NBODY_ECUDA, "debug build: a device-side index check failed at site %d (access skipped)",
                    h.debug_site);
    if (f & kFlagTimeout)
        return fail(NBODY_ETIMEOUT, "a bounded device-side wait (for a j-tile or at a grid barrier) gave up");
    if (f & kFlagBadIndex)
        return fail(NBODY_EINVAL, "active list row %d holds an index outside [0, %lld)", h.bad_index,
                    static_cast<long long>(c->n));
    if (f & kFlagNonfinite)
        return fail(NBODY_ENONFINITE, "non-finite force or corrected state (%llu rows so far)", h.nonfinite);
    if ((f & kFlagDtMin) && c->p.strict)
        return fail(NBODY_EDTMIN, "a time-step criterion fell below dt_min = 2^-%d (%llu clamps so far)",
                    c->p.lmax, h.below_min);
    return NBODY_OK;
}

// Enqueues the status read-back, drains the stream and reports new flags.
int sync_and_check(nbody_ctx *c)
{
    NB_CUDA(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->s),
            "status read-back");
    NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
    return absorb_status(c);
}

int ensure_partials(nbody_ctx *c, size_t bytes)
{
    if (bytes <= c->partials_cap) return NBODY_OK;
    if (c->partials) {
        NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
        cudaFree(c->partials);
        c->partials = nullptr;
        c->partials_cap = 0;
    }
    const size_t cap = std::max(bytes, static_cast<size_t>(1) << 20);
    NB_CUDA(dev_alloc(&c->partials, cap), "partial-sum scratch allocation");
    c->partials_cap = cap;
    return NBODY_OK;
}

// Force on a device list already in act_force.  With for_step, a shape whose
// partials the corrector adds (force_partials_fused) skips the reduction;
// fused_split then tells correct_internal to read them.
int force_internal(nbody_ctx *c, int64_t n_act, bool for_step = false)
{
    ForceConfig cfg{};
    const int r = force_choose(c->p.mode, n_act, c->n_pad, c->sm_count, c->p.j_tile, c->p.i_block, c->p.j_split,
                               &cfg, c->p.j_sub);
    if (r != NBODY_OK) return fail(r, "unsupported force shape: %d threads x %d i per thread", c->p.j_tile, c->p.i_block);
    const int rp = ensure_partials(c, force_partial_bytes(c->p.mode, cfg, n_act));
    if (rp != NBODY_OK) return rp;
    int64_t launches = 0;
    const bool fused = for_step && force_partials_fused(c->p.mode, cfg);
    NB_CUDA(force_launch(c->p.mode, c->J, c->n, c->act_force, n_act, c->eps2, cfg,
                         c->f_acc, c->f_jerk, c->f_pot, c->partials, c->st, c->s, &launches, nullptr, !fused),
            "force kernel launch");
    c->fused_split = fused ? cfg.split : 0;
    c->stats.kernel_launches += launches;
    c->stats.force_calls += 1;
    c->stats.pairs += n_act * (c->n - 1);
    c->stats.last_threads = cfg.threads;
    c->stats.last_i_per_thread = cfg.ipt;
    c->stats.last_j_split = cfg.split;
    c->stats.last_j_sub = cfg.jsub;
    c->force_n_act = fused ? -1 : n_act;  // a fused force left no rows for nbody_correct to reuse
    return NBODY_OK;
}

int predict_internal(nbody_ctx *c, int64_t tick)
{
    if (tick < c->t_max)
        return fail(NBODY_EINVAL, "prediction time %lld ticks is before a particle time %lld",
                    static_cast<long long>(tick), static_cast<long long>(c->t_max));
    NB_CUDA(predict_launch(c->S, c->J, tick, c->p.lmax, predict_lo_parts(c->p.mode), c->s, &c->stats.kernel_launches),
            "predictor launch");
    c->t_pred = tick;
    c->pred_valid = true;
    c->force_n_act = -1;
    return NBODY_OK;
}

int correct_internal(nbody_ctx *c, const int32_t *act_dev, int64_t n_act, const double *acc_dev,
                     const double *jerk_dev, bool fused_partials = false)
{
    const int split = fused_partials ? c->fused_split : 0;
    NB_CUDA(correct_launch(c->S, act_dev, n_act, acc_dev, jerk_dev, c->t_pred, c->p.eta, c->p.lmin, c->p.lmax,
                           c->st, c->s, &c->stats.kernel_launches, nullptr,
                           split > 1 ? static_cast<const float *>(c->partials) : nullptr, split,
                           two_word_sums(c->p.mode)),
            "corrector launch");
    if (n_act > 0) {
        c->t_max = std::max(c->t_max, c->t_pred);
        c->stats.blocks += 1;
    }
    c->pred_valid = false;  // the corrected particles moved: predict again before the next force
    c->force_n_act = -1;
    return NBODY_OK;
}

int schedule_internal(nbody_ctx *c, int64_t *t_blk, int64_t *n_act)
{
    NB_CUDA(schedule_launch(c->S, c->p.lmax, c->act_sched, c->sched_out, c->sched_scratch, c->s,
                            &c->stats.kernel_launches),
            "scheduler launch");
    NB_CUDA(cudaMemcpyAsync(c->sched_host, c->sched_out, sizeof(SchedOut), cudaMemcpyDeviceToHost, c->s),
            "schedule read-back");
    const int r = sync_and_check(c);
    if (r != NBODY_OK) return r;
    *t_blk = c->sched_host->t_blk;
    *n_act = c->sched_host->n_act;
    return NBODY_OK;
}

int check_params(const nbody_params *p)
{
    if (!(p->eta > 0.0) || !std::isfinite(p->eta)) return fail(NBODY_EINVAL, "eta must be positive");
    if (p->lmin < 0 || p->lmax > 40 || p->lmin > p->lmax)
        return fail(NBODY_EINVAL, "need 0 <= lmin <= lmax <= 40 (got %d, %d)", p->lmin, p->lmax);
    if (p->mode != NBODY_MODE_PLAIN && p->mode != NBODY_MODE_COMP && p->mode != NBODY_MODE_SUMCHECK &&
        p->mode != NBODY_MODE_SORTED && p->mode != NBODY_MODE_DS)
        return fail(NBODY_EINVAL, "unknown mode %d", p->mode);
    if (p->j_tile != 0 && p->j_tile != 64 && p->j_tile != 128 && p->j_tile != 256 && p->j_tile != 512)
        return fail(NBODY_EINVAL, "j_tile must be 0, 64, 128, 256 or 512");
    if (p->j_tile == 512 && p->i_block > 1) return fail(NBODY_EINVAL, "512 threads take i_block 0 or 1");
    if (p->i_block != 0 && p->i_block != 1 && p->i_block != 2 && p->i_block != 4)
        return fail(NBODY_EINVAL, "i_block must be 0, 1, 2 or 4");
    if (p->j_split < 0) return fail(NBODY_EINVAL, "j_split must be >= 0");
    if (p->j_sub != 0 && p->j_sub != 1 && p->j_sub != 4) return fail(NBODY_EINVAL, "j_sub must be 0, 1 or 4");
    return NBODY_OK;
}

int energy_common(nbody_ctx *c, double *ekin, double *epot, bool ds_potential)
{
    NB_CUDA(time_range_launch(c->S, c->trange, c->s, &c->stats.kernel_launches), "time-range kernel");
    NB_CUDA(cudaMemcpyAsync(c->trange_host, c->trange, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s),
            "time-range read-back");
    int r = sync_and_check(c);
    if (r != NBODY_OK) return r;
    if (c->trange_host[0] != c->trange_host[1])
        return fail(NBODY_ENOTSYNC, "particles are at different times (%llu .. %llu ticks)", c->trange_host[0],
                    c->trange_host[1]);
    NB_CUDA(energy_launch(c->S, c->eps2, c->phi, c->e_out, c->s, &c->stats.kernel_launches, ds_potential),
            "energy kernels");
    NB_CUDA(cudaMemcpyAsync(c->e_host, c->e_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s), "energy read-back");
    r = sync_and_check(c);
    if (r != NBODY_OK) return r;
    *ekin = c->e_host[0];
    *epot = c->e_host[1];
    return NBODY_OK;
}

// A shared-step rollout (the force at t = 0, then `steps` Hermite steps of dt = 2^-level) and, with
// `backward`, the reverse sweep: seeded with the loss L = sum |x|^2 + E_pot (seed_loss) or with the
// cotangents g_xT, g_vT of the final positions and velocities (either may be NULL: zero).  Outputs
// that are NULL are not written.
int rollout_impl(const char *who, int64_t n, const double *m, const double *x0, const double *v0, double eps2,
                 int level, int64_t steps, int64_t checkpoint_every, int mode, bool backward, bool seed_loss,
                 const double *g_xT, const double *g_vT, double *loss, double *x_T, double *v_T, double *g_x0,
                 double *g_v0, double *g_m, void *stream)
{
    g_err[0] = '\0';
    if (!m || !x0 || !v0) return fail(NBODY_EINVAL, "%s: null argument", who);
    if (!(eps2 > 0.0)) return fail(NBODY_EINVAL, "%s: eps2 must be > 0", who);
    if (level < 0 || level > 40 || steps < 0) return fail(NBODY_EINVAL, "%s: bad level or steps", who);
    if (checkpoint_every <= 0) checkpoint_every = 16;
    nbody_params p;
    nbody_default_params(&p);
    p.lmin = p.lmax = level;  // one shared power-of-two step: every block is all particles
    p.mode = mode;
    p.stream = stream;
    nbody_ctx *c = nullptr;
    int r = nbody_init(&c, n, m, x0, v0, eps2, &p);
    if (r != NBODY_OK) return r;
    c->J.aos = true;  // the force's vector-Jacobian product reads the float4 j-stream
    const size_t nd = static_cast<size_t>(n);
    const size_t npad = static_cast<size_t>(c->n_pad);
    const int64_t n_ck = steps / checkpoint_every + 1;
    const size_t state_doubles = 12 * nd;  // x, v, a, k (contiguous after m)
    double *ck = nullptr, *seg = nullptr, *gbuf = nullptr, *lval = nullptr, *dloss = nullptr, *vjp = nullptr;
    float4 *g4 = nullptr;
    DiffGrads G{};
    const double dt = std::ldexp(1.0, -level);
    const float e2 = static_cast<float>(eps2);
    cudaStream_t s = c->s;
    int64_t *L = &c->stats.kernel_launches;
    auto done = [&](int code) {
        cudaStreamSynchronize(s);
        void *bufs[] = {ck, seg, gbuf, lval, dloss, g4, vjp};
        for (void *b : bufs)
            if (b) cudaFree(b);
        nbody_free(c);
        return code;
    };
#define NB_DR(call, what)                                     \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return done(cuda_fail(e_, what)); \
    } while (0)
    // the state after the last step, copied out row-major
    auto copy_final = [&]() -> int {
        if (x_T) {
            NB_CUDA(soa_to_aos_launch(c->S.x[0], c->S.x[1], c->S.x[2], c->stage, n, s, L), "layout");
            NB_CUDA(cudaMemcpyAsync(x_T, c->stage, 3 * nd * sizeof(double), cudaMemcpyDefault, s), "state copy");
        }
        if (v_T) {
            NB_CUDA(soa_to_aos_launch(c->S.v[0], c->S.v[1], c->S.v[2], c->stage + 3 * nd, n, s, L), "layout");
            NB_CUDA(cudaMemcpyAsync(v_T, c->stage + 3 * nd, 3 * nd * sizeof(double), cudaMemcpyDefault, s),
                    "state copy");
        }
        return NBODY_OK;
    };
    if (!backward) {
        NB_DR(iota_launch(c->act_force, n, s, L), "index kernel");
        for (int64_t k = 0; k < steps; ++k) {
            r = predict_internal(c, k + 1);
            if (r == NBODY_OK) r = force_internal(c, n);
            if (r == NBODY_OK) r = correct_internal(c, c->act_force, n, c->f_acc, c->f_jerk);
            if (r != NBODY_OK) return done(r);
        }
        r = copy_final();
        if (r == NBODY_OK) r = sync_and_check(c);
        return done(r);
    }
    NB_DR(dev_alloc(reinterpret_cast<void **>(&ck), n_ck * state_doubles * sizeof(double)), "checkpoints");
    NB_DR(dev_alloc(reinterpret_cast<void **>(&seg), checkpoint_every * state_doubles * sizeof(double)), "segment");
    NB_DR(dev_alloc(reinterpret_cast<void **>(&gbuf), 19 * nd * sizeof(double)), "gradients");
    NB_DR(dev_alloc(reinterpret_cast<void **>(&lval), nd * sizeof(double)), "loss terms");
    NB_DR(dev_alloc(reinterpret_cast<void **>(&dloss), sizeof(double)), "loss");
    NB_DR(dev_alloc(reinterpret_cast<void **>(&g4), 2 * npad * sizeof(float4)), "force upstream");
    const size_t vjp_doubles = vjp_scratch_doubles(n, c->n_pad, c->sm_count);
    if (vjp_doubles) NB_DR(dev_alloc(reinterpret_cast<void **>(&vjp), vjp_doubles * sizeof(double)), "adjoint scratch");
    NB_DR(cudaMemsetAsync(gbuf, 0, 19 * nd * sizeof(double), s), "memset");
    NB_DR(cudaMemsetAsync(g4, 0, 2 * npad * sizeof(float4), s), "memset");
    for (int q = 0; q < 3; ++q) {
        G.gx[q] = gbuf + (0 + q) * nd;
        G.gv[q] = gbuf + (3 + q) * nd;
        G.ga[q] = gbuf + (6 + q) * nd;
        G.gk[q] = gbuf + (9 + q) * nd;
        G.gxp[q] = gbuf + (12 + q) * nd;
        G.gvp[q] = gbuf + (15 + q) * nd;
    }
    G.gm = gbuf + 18 * nd;
    G.gA = g4;
    G.gK = g4 + npad;
    double *xvak = c->state + nd;  // x[3], v[3], a[3], k[3]
    NB_DR(iota_launch(c->act_force, n, s, L), "index kernel");
    // one shared Hermite step from tick s0 to s0 + 1 (all particles in the block)
    auto step = [&](int64_t s0) -> int {
        int rr = predict_internal(c, s0 + 1);
        if (rr != NBODY_OK) return rr;
        rr = force_internal(c, n);
        if (rr != NBODY_OK) return rr;
        return correct_internal(c, c->act_force, n, c->f_acc, c->f_jerk);
    };
    auto restore = [&](const double *src, int64_t tick) -> int {
        NB_CUDA(cudaMemcpyAsync(xvak, src, state_doubles * sizeof(double), cudaMemcpyDeviceToDevice, s), "restore");
        NB_CUDA(set_time_launch(c->S, tick, level, s, L), "time kernel");
        c->t_max = tick;
        return NBODY_OK;
    };
    // forward with checkpoints
    NB_DR(cudaMemcpyAsync(ck, xvak, state_doubles * sizeof(double), cudaMemcpyDeviceToDevice, s), "checkpoint");
    for (int64_t k = 0; k < steps; ++k) {
        r = step(k);
        if (r != NBODY_OK) return done(r);
        if ((k + 1) % checkpoint_every == 0)
            NB_DR(cudaMemcpyAsync(ck + ((k + 1) / checkpoint_every) * state_doubles, xvak,
                                  state_doubles * sizeof(double), cudaMemcpyDeviceToDevice, s),
                  "checkpoint");
    }
    r = copy_final();  // before the backward sweep overwrites the state
    if (r != NBODY_OK) return done(r);
    if (seed_loss) {
        NB_DR(loss_launch(c->S, eps2, G, lval, dloss, s, L), "loss kernels");
    } else {  // the cotangents of the final x, v seed the sweep (row-major n x 3 -> components)
        if (g_xT) {
            NB_DR(to_device(c->stage, g_xT, 3 * nd * sizeof(double), s), "cotangent upload");
            NB_DR(aos_to_soa_launch(c->stage, G.gx[0], G.gx[1], G.gx[2], n, s, L), "layout kernel");
        }
        if (g_vT) {
            NB_DR(to_device(c->stage + 3 * nd, g_vT, 3 * nd * sizeof(double), s), "cotangent upload");
            NB_DR(aos_to_soa_launch(c->stage + 3 * nd, G.gv[0], G.gv[1], G.gv[2], n, s, L), "layout kernel");
        }
    }
    // backward, one checkpoint segment at a time
    for (int64_t seg0 = (steps - 1) / checkpoint_every * checkpoint_every; steps > 0 && seg0 >= 0;
         seg0 -= checkpoint_every) {
        const int64_t seg1 = std::min(seg0 + checkpoint_every, steps);
        r = restore(ck + (seg0 / checkpoint_every) * state_doubles, seg0);
        if (r != NBODY_OK) return done(r);
        for (int64_t k = seg0; k < seg1; ++k) {
            NB_DR(cudaMemcpyAsync(seg + (k - seg0) * state_doubles, xvak, state_doubles * sizeof(double),
                                  cudaMemcpyDeviceToDevice, s),
                  "segment");
            if (k + 1 < seg1) {
                r = step(k);
                if (r != NBODY_OK) return done(r);
            }
        }
        for (int64_t k = seg1 - 1; k >= seg0; --k) {
            r = restore(seg + (k - seg0) * state_doubles, k);
            if (r != NBODY_OK) return done(r);
            r = predict_internal(c, k + 1);  // j-stream at the predicted state of step k
            if (r != NBODY_OK) return done(r);
            NB_DR(adj_correct_launch(G, n, dt, s, L), "adjoint corrector");
            NB_DR(force_vjp_launch(c->J, G, n, e2, c->sm_count, vjp, s, L), "force adjoint");
            NB_DR(adj_predict_launch(G, n, dt, s, L), "adjoint predictor");
        }
    }
    // the t = 0 force
    r = restore(ck, 0);
    if (r != NBODY_OK) return done(r);
    r = predict_internal(c, 0);
    if (r != NBODY_OK) return done(r);
    NB_DR(adj_init_launch(G, n, s, L), "adjoint init");
    NB_DR(force_vjp_launch(c->J, G, n, e2, c->sm_count, vjp, s, L), "force adjoint");
    if (seed_loss && loss) NB_DR(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDefault, s), "loss copy");
    if (g_x0) {
        NB_DR(soa_to_aos_launch(G.gxp[0], G.gxp[1], G.gxp[2], c->stage, n, s, L), "layout");
        NB_DR(cudaMemcpyAsync(g_x0, c->stage, 3 * nd * sizeof(double), cudaMemcpyDefault, s), "gradient copy");
    }
    if (g_v0) {
        NB_DR(soa_to_aos_launch(G.gvp[0], G.gvp[1], G.gvp[2], c->stage + 3 * nd, n, s, L), "layout");
        NB_DR(cudaMemcpyAsync(g_v0, c->stage + 3 * nd, 3 * nd * sizeof(double), cudaMemcpyDefault, s),
              "gradient copy");
    }
    if (g_m) NB_DR(cudaMemcpyAsync(g_m, G.gm, nd * sizeof(double), cudaMemcpyDefault, s), "gradient copy");
    r = sync_and_check(c);
#undef NB_DR
    return done(r);
}

}  // namespace

extern "C" {

void nbody_default_params(nbody_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->eta = 0.01;
    p->eta_init = 0.0;
    p->lmin = 6;
    p->lmax = 26;
    p->mode = NBODY_MODE_PLAIN;
}

int nbody_init(nbody_ctx **out, int64_t n, const double *m, const double *x, const double *v, double eps2,
               const nbody_params *p)
{
    g_err[0] = '\0';
    if (!out || !m || !x || !v) return fail(NBODY_EINVAL, "nbody_init: null pointer argument");
    *out = nullptr;
    if (n < 1 || n > 2147483647LL) return fail(NBODY_EINVAL, "nbody_init: n = %lld out of range", static_cast<long long>(n));
    if (p && p->mode == NBODY_MODE_SORTED && n > kSortedMaxN)
        return fail(NBODY_EINVAL, "nbody_init: the sorted mode takes n <= %lld", static_cast<long long>(kSortedMaxN));
    if (!(eps2 >= 0.0) || !std::isfinite(eps2)) return fail(NBODY_EINVAL, "nbody_init: eps2 must be finite and >= 0");
    nbody_params prm;
    if (p) prm = *p;
    else nbody_default_params(&prm);
    int r = check_params(&prm);
    if (r != NBODY_OK) return r;
    if (prm.eta_init <= 0.0) prm.eta_init = prm.eta;

    nbody_ctx *c = new (std::nothrow) nbody_ctx;
    if (!c) return fail(NBODY_ENOMEM, "nbody_init: host allocation failed");
    c->n = n;
    c->n_pad = (n + kJTile - 1) / kJTile * kJTile;
    c->eps2 = eps2;
    c->p = prm;
    c->s = static_cast<cudaStream_t>(prm.stream);

    auto bail = [&](int code) {
        release(c);
        return code;
    };
#define NB_INIT(call, what)                        \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, what)); \
    } while (0)

    int dev = 0;
    NB_INIT(cudaGetDevice(&dev), "cudaGetDevice");
    NB_INIT(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const size_t nd = static_cast<size_t>(n);
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->state), 13 * nd * sizeof(double)), "state allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->t), nd * sizeof(int64_t)), "time allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->level), nd), "level allocation");
    const size_t jbytes = static_cast<size_t>(c->n_pad) * (4 * sizeof(float4) + kSoaArrays * sizeof(float));
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->jbuf), jbytes), "j-stream allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->act_force), nd * sizeof(int32_t)), "list allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->act_corr), nd * sizeof(int32_t)), "list allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->act_sched), nd * sizeof(int32_t)), "list allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->f_acc), 3 * nd * sizeof(double)), "force allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->f_jerk), 3 * nd * sizeof(double)), "force allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->f_pot), nd * sizeof(double)), "force allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->stage), 6 * nd * sizeof(double)), "staging allocation");
    NB_INIT(dev_alloc(&c->sched_scratch, sched_scratch_bytes(n)), "scheduler scratch allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->sched_out), sizeof(SchedOut)), "scheduler allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->st), sizeof(DevStatus)), "status allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->phi), nd * sizeof(double)), "energy scratch allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->e_out), 2 * sizeof(double)), "energy allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->trange), 2 * sizeof(unsigned long long)), "time-range allocation");
    NB_INIT(host_alloc(reinterpret_cast<void **>(&c->sched_host), sizeof(SchedOut)), "pinned allocation");
    NB_INIT(host_alloc(reinterpret_cast<void **>(&c->st_host), sizeof(DevStatus)), "pinned allocation");
    NB_INIT(host_alloc(reinterpret_cast<void **>(&c->e_host), 2 * sizeof(double)), "pinned allocation");
    NB_INIT(host_alloc(reinterpret_cast<void **>(&c->trange_host), 2 * sizeof(unsigned long long)),
            "pinned allocation");
    NB_INIT(dev_alloc(reinterpret_cast<void **>(&c->loop_dev), sizeof(StepLoop)), "loop control allocation");
    NB_INIT(host_alloc(reinterpret_cast<void **>(&c->loop_host), sizeof(StepLoop)), "pinned allocation");
    std::memset(c->st_host, 0, sizeof(DevStatus));

    State &S = c->S;
    S.n = n;
    S.m = c->state;
    for (int q = 0; q < 3; ++q) {
        S.x[q] = c->state + (1 + q) * nd;
        S.v[q] = c->state + (4 + q) * nd;
        S.a[q] = c->state + (7 + q) * nd;
        S.k[q] = c->state + (10 + q) * nd;
    }
    S.t = c->t;
    S.level = c->level;
    c->J.posm = c->jbuf;
    c->J.vel = c->jbuf + c->n_pad;
    c->J.poslo = c->jbuf + 2 * c->n_pad;
    c->J.vello = c->jbuf + 3 * c->n_pad;
    c->J.soa = reinterpret_cast<float *>(c->jbuf + 4 * c->n_pad);
    c->J.n_pad = c->n_pad;
    c->J.aos = force_needs_aos(prm.mode);

    cudaStream_t s = c->s;
    int64_t *L = &c->stats.kernel_launches;
    NB_INIT(cudaMemsetAsync(c->jbuf, 0, jbytes, s), "memset");
    NB_INIT(pad_jstream_launch(c->J, n, s, &c->stats.kernel_launches), "padding kernel");
    NB_INIT(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s), "memset");
    NB_INIT(cudaMemsetAsync(c->state + 7 * nd, 0, 6 * nd * sizeof(double), s), "memset");
    NB_INIT(cudaMemsetAsync(c->t, 0, nd * sizeof(int64_t), s), "memset");
    NB_INIT(to_device(c->state, m, nd * sizeof(double), s), "mass upload");
    NB_INIT(to_device(c->stage, x, 3 * nd * sizeof(double), s), "position upload");
    NB_INIT(aos_to_soa_launch(c->stage, S.x[0], S.x[1], S.x[2], n, s, L), "layout kernel");
    NB_INIT(to_device(c->stage + 3 * nd, v, 3 * nd * sizeof(double), s), "velocity upload");
    NB_INIT(aos_to_soa_launch(c->stage + 3 * nd, S.v[0], S.v[1], S.v[2], n, s, L), "layout kernel");
    NB_INIT(mass_jstream_launch(S, c->J, s, L), "mass kernel");

    // t = 0: predicted state = state; full force; first levels.
    r = predict_internal(c, 0);
    if (r != NBODY_OK) return bail(r);
    NB_INIT(iota_launch(c->act_force, n, s, L), "index kernel");
    r = force_internal(c, n);
    if (r != NBODY_OK) return bail(r);
    NB_INIT(init_levels_launch(S, c->f_acc, c->f_jerk, c->p.eta_init, c->p.lmin, c->p.lmax, c->st, s, L),
            "initial level kernel");
    c->force_n_act = -1;
    c->pred_valid = false;
    c->t_max = 0;
    r = sync_and_check(c);
    if (r == NBODY_EDTMIN) r = NBODY_OK;  // the first steps may be clamped; counted, not fatal here
    if (r != NBODY_OK) return bail(r);
    c->stats.n = n;
    c->stats.n_pad = c->n_pad;
    c->stats.mode = c->p.mode;
#undef NB_INIT
    *out = c;
    return NBODY_OK;
}

int nbody_next_block(nbody_ctx *c, double *t_blk, int64_t *n_act, int32_t *active)
{
    if (!c || !t_blk || !n_act) return fail(NBODY_EINVAL, "nbody_next_block: null argument");
    int64_t tb = 0, na = 0;
    int r = schedule_internal(c, &tb, &na);
    if (r != NBODY_OK) return r;
    *t_blk = std::ldexp(static_cast<double>(tb), -c->p.lmax);
    *n_act = na;
    if (active && na > 0) {
        NB_CUDA(cudaMemcpyAsync(active, c->act_sched, static_cast<size_t>(na) * sizeof(int32_t), cudaMemcpyDefault,
                                c->s),
                "active list copy");
        if (!is_device_ptr(active)) NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
    }
    return NBODY_OK;
}

int nbody_predict(nbody_ctx *c, double t)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_predict: null context");
    int64_t tick;
    const int r = to_ticks(c, t, &tick);
    if (r != NBODY_OK) return r;
    return predict_internal(c, tick);
}

int nbody_force(nbody_ctx *c, const int32_t *active, int64_t n_act, double *acc, double *jerk, double *pot)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_force: null context");
    if (n_act < 0 || n_act > c->n) return fail(NBODY_EINVAL, "nbody_force: n_act = %lld outside [0, n]", static_cast<long long>(n_act));
    if (n_act > 0 && !active) return fail(NBODY_EINVAL, "nbody_force: null active list");
    if (!c->pred_valid) return fail(NBODY_ESTATE, "nbody_force: no prediction since the last correction");
    const size_t na = static_cast<size_t>(n_act);
    NB_CUDA(to_device(c->act_force, active, na * sizeof(int32_t), c->s), "active list upload");
    int r = force_internal(c, n_act);
    if (r != NBODY_OK) return r;
    bool host_out = false;
    if (acc) {
        NB_CUDA(cudaMemcpyAsync(acc, c->f_acc, 3 * na * sizeof(double), cudaMemcpyDefault, c->s), "acc copy");
        host_out |= !is_device_ptr(acc);
    }
    if (jerk) {
        NB_CUDA(cudaMemcpyAsync(jerk, c->f_jerk, 3 * na * sizeof(double), cudaMemcpyDefault, c->s), "jerk copy");
        host_out |= !is_device_ptr(jerk);
    }
    if (pot) {
        NB_CUDA(cudaMemcpyAsync(pot, c->f_pot, na * sizeof(double), cudaMemcpyDefault, c->s), "pot copy");
        host_out |= !is_device_ptr(pot);
    }
    if (host_out) {
        r = sync_and_check(c);
        if (r != NBODY_OK) return r;
    }
    return NBODY_OK;
}

int nbody_correct(nbody_ctx *c, const int32_t *active, int64_t n_act, const double *acc, const double *jerk)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_correct: null context");
    if (n_act < 0 || n_act > c->n) return fail(NBODY_EINVAL, "nbody_correct: n_act = %lld outside [0, n]", static_cast<long long>(n_act));
    if (n_act > 0 && !active) return fail(NBODY_EINVAL, "nbody_correct: null active list");
    if ((acc == nullptr) != (jerk == nullptr)) return fail(NBODY_EINVAL, "nbody_correct: give both acc and jerk, or neither");
    if (!c->pred_valid) return fail(NBODY_ESTATE, "nbody_correct: no prediction to correct from");
    const size_t na = static_cast<size_t>(n_act);
    const double *fa = c->f_acc, *fj = c->f_jerk;
    if (!acc) {
        if (c->force_n_act != n_act)
            return fail(NBODY_ESTATE, "nbody_correct: the last nbody_force had %lld rows, not %lld",
                        static_cast<long long>(c->force_n_act), static_cast<long long>(n_act));
    } else {
        NB_CUDA(to_device(c->stage, acc, 3 * na * sizeof(double), c->s), "acc upload");
        NB_CUDA(to_device(c->stage + 3 * c->n, jerk, 3 * na * sizeof(double), c->s), "jerk upload");
        fa = c->stage;
        fj = c->stage + 3 * c->n;
    }
    NB_CUDA(to_device(c->act_corr, active, na * sizeof(int32_t), c->s), "active list upload");
    return correct_internal(c, c->act_corr, n_act, fa, fj);
}

namespace {

// Rows the small-block graph is sized for: its force grid (rows / 64 x j-ranges)
// stays near 2048 blocks, so blocks beyond the actual size exit at little cost,
// and below the rows where the automatic shape turns to j-subgroups, so that all
// the small blocks share the graph's shape.
int64_t graph_rows_for(const nbody_ctx *c)
{
    const int64_t n_tiles = c->n_pad / kJTile;
    const int64_t by_grid = 64 * std::max<int64_t>(1, 2048 / n_tiles);
    const int64_t cap = n_tiles >= kJSubMinTiles ? kJSubMinRows - 1 : 8191;
    return std::min<int64_t>({c->n, by_grid, cap});
}

bool same_shape(const ForceConfig &a, const ForceConfig &b)
{
    return a.threads == b.threads && a.ipt == b.ipt && a.jsub == b.jsub && a.split == b.split &&
           a.tiles_per_split == b.tiles_per_split && a.slice == b.slice;
}

// One block step sized for graph_rows rows, captured on cs: predictor, force,
// corrector and the next block's schedule, all reading the block time and size
// on the device; with la, the loop's decision after the schedule.
cudaError_t capture_block_step(nbody_ctx *c, cudaStream_t cs, int64_t *launches, const LoopArgs *la)
{
    const int64_t rows = c->graph_rows;
    cudaError_t e = predict_launch(c->S, c->J, 0, c->p.lmax, predict_lo_parts(c->p.mode), cs, launches,
                                   &c->sched_out->t_blk);
    const bool fused = force_partials_fused(c->p.mode, c->graph_cfg);
    if (e == cudaSuccess)
        e = force_launch(c->p.mode, c->J, c->n, c->act_sched, rows, c->eps2, c->graph_cfg, c->f_acc, c->f_jerk,
                         c->f_pot, c->partials, c->st, cs, launches, &c->sched_out->n_act, !fused);
    if (e == cudaSuccess)
        e = correct_launch(c->S, c->act_sched, rows, c->f_acc, c->f_jerk, 0, c->p.eta, c->p.lmin, c->p.lmax, c->st,
                           cs, launches, c->sched_out, fused ? static_cast<const float *>(c->partials) : nullptr,
                           fused ? c->graph_cfg.split : 0, two_word_sums(c->p.mode));
    if (e == cudaSuccess)
        e = la ? schedule_loop_launch(c->S, c->p.lmax, c->act_sched, c->sched_out, c->sched_scratch, *la, cs, launches)
               : schedule_launch(c->S, c->p.lmax, c->act_sched, c->sched_out, c->sched_scratch, cs, launches);
    return e;
}

// Status flags that end the device-side loop: every error flag, and the dt_min
// clamp in strict mode (the flags the host would report after that block).
unsigned loop_stop_flags(const nbody_ctx *c)
{
    return kFlagTimeout | kFlagBadIndex | kFlagNonfinite | kFlagDebugBounds | (c->p.strict ? kFlagDtMin : 0u);
}

// Blocks of this context may run in the one-cluster kernel (level 3).
bool cluster_steps(const nbody_ctx *c)
{
    const int mode = c->p.mode;
    if (g_step_graphs < 3 || (mode != NBODY_MODE_PLAIN && mode != NBODY_MODE_COMP && mode != NBODY_MODE_DS))
        return false;
    if (c->p.j_tile != 0 || c->p.i_block != 0 || c->p.j_split != 0 || c->p.j_sub != 0) return false;
    if (!c->J.soa || c->n_pad > (mode == NBODY_MODE_DS ? kClMaxPadDS : kClMaxPad)) return false;
    const int C = cluster_step_size(c->p.mode);
    return C > 0 && c->n_pad / C <= kClMaxChunk;
}

// Blocks of up to kGridRows rows of this context may run in the whole-GPU
// cooperative kernel (level 3, plain and compensated systems past the cluster
// kernel's sizes, n <= CTAs x kGrMaxChunk).
bool grid_steps(const nbody_ctx *c)
{
    const int mode = c->p.mode;
    if (g_step_graphs < 3 || (mode != NBODY_MODE_PLAIN && mode != NBODY_MODE_COMP)) return false;
    if (c->p.j_tile != 0 || c->p.i_block != 0 || c->p.j_split != 0 || c->p.j_sub != 0) return false;
    if (!c->J.soa || cluster_steps(c)) return false;
    return grid_step_chunk(c->n, grid_step_size(mode)) > 0;
}

// Builds the replayed graph: the block step as the body of a while-node, whose
// last kernel decides whether the next block runs in the same replay, then the
// read-back of the next block, the status and the loop control.  Without
// while-nodes (loop = false) the graph holds one block step.
cudaError_t capture_step_graph(nbody_ctx *c, bool loop, cudaGraph_t *out, int64_t *launches)
{
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    cudaGraphNode_t loop_node = nullptr;
    cudaGraph_t body = nullptr;
    cudaGraphConditionalHandle h{};
    e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess && loop) {
        e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        if (e == cudaSuccess) e = cudaGraphAddNode(&loop_node, g, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    cudaGraph_t captured = nullptr;
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(cs, loop ? body : g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const LoopArgs la{h, c->graph_fits, c->graph_rows + 1, c->st, loop_stop_flags(c), c->loop_dev};
        cudaError_t e2 = capture_block_step(c, cs, launches, loop ? &la : nullptr);
        if (e2 == cudaSuccess && !loop) e2 = cudaMemcpyAsync(c->sched_host, c->sched_out, sizeof(SchedOut),
                                                              cudaMemcpyDeviceToHost, cs);
        if (e2 == cudaSuccess && !loop)
            e2 = cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, cs);
        e = cudaStreamEndCapture(cs, &captured);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && loop) {
        e = cudaStreamBeginCaptureToGraph(cs, g, &loop_node, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = cudaMemcpyAsync(c->sched_host, c->sched_out, sizeof(SchedOut), cudaMemcpyDeviceToHost, cs);
            if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, cs);
            if (e2 == cudaSuccess)
                e2 = cudaMemcpyAsync(c->loop_host, c->loop_dev, sizeof(StepLoop), cudaMemcpyDeviceToHost, cs);
            e = cudaStreamEndCapture(cs, &captured);
            if (e == cudaSuccess) e = e2;
        }
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    *out = g;
    return cudaSuccess;
}

// Fills graph_fits: flag na is set when a block of na rows takes the graph's
// launch shape, the test the host applies before a replay.
int set_graph_fits(nbody_ctx *c)
{
    const int64_t len = c->graph_rows + 1;
    std::vector<unsigned char> fits(static_cast<size_t>(len), 0);
    for (int64_t na = 1; na < len; ++na) {
        ForceConfig cfg{};
        fits[na] = force_choose(c->p.mode, na, c->n_pad, c->sm_count, c->p.j_tile, c->p.i_block, c->p.j_split,
                                &cfg, c->p.j_sub) == NBODY_OK && same_shape(cfg, c->graph_cfg);
    }
    NB_CUDA(dev_alloc(reinterpret_cast<void **>(&c->graph_fits), static_cast<size_t>(len)), "graph table allocation");
    NB_CUDA(cudaMemcpy(c->graph_fits, fits.data(), static_cast<size_t>(len), cudaMemcpyHostToDevice),
            "graph table upload");
    return NBODY_OK;
}

// Captures the graph once (and again when the partial-sum scratch moved).
int build_step_graph(nbody_ctx *c)
{
    if (c->step_graph && c->graph_partials == c->partials) return NBODY_OK;
    if (c->step_graph) {
        cudaGraphExecDestroy(c->step_graph);
        c->step_graph = nullptr;
    }
    const int rp = ensure_partials(c, force_partial_bytes(c->p.mode, c->graph_cfg, c->graph_rows));
    if (rp != NBODY_OK) return rp;
    if (!c->graph_fits) {
        const int rf = set_graph_fits(c);
        if (rf != NBODY_OK) return rf;
    }
    int64_t launches = 0;
    cudaGraph_t g = nullptr;
    bool loop = g_step_graphs >= 2;  // the form is fixed when a context first builds its graph
    cudaError_t e = capture_step_graph(c, loop, &g, &launches);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_graph, g, 0);
    if (e != cudaSuccess && loop) {  // no while-nodes: one block step per replay
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        g = nullptr;
        c->step_graph = nullptr;
        loop = false;
        launches = 0;
        e = capture_step_graph(c, false, &g, &launches);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_graph, g, 0);
    }
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->step_graph = nullptr;
        return cuda_fail(e, "step graph capture");
    }
    c->graph_partials = c->partials;
    c->graph_launches = launches;
    c->graph_loop = loop;
    return NBODY_OK;
}

}  // namespace

int nbody_step(nbody_ctx *c, double t_end, int64_t max_steps, int64_t *n_steps)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_step: null context");
    int64_t tend;
    int r = to_ticks(c, t_end, &tend);
    if (r != NBODY_OK) return r;
    const int64_t dtmax = int64_t(1) << (c->p.lmax - c->p.lmin);
    if (tend % dtmax != 0) return fail(NBODY_EINVAL, "nbody_step: t_end must be a multiple of dt_max = 2^-%d", c->p.lmin);
    if (tend < c->t_max) return fail(NBODY_EINVAL, "nbody_step: t_end is before the current time");
    int64_t done = 0;
    // Small blocks replay one graph (predict, force, correct, next schedule and its read-back) when its
    // launch shape is the one the separate launches would take, so both give the same bits; inside a
    // replay a device-side loop runs the following blocks while they fit too.
    const bool packed = force_reads_device_rows(c->p.mode);
    if (g_step_graphs > 0 && packed && c->graph_rows == 0) {
        c->graph_rows = graph_rows_for(c);
        if (force_choose(c->p.mode, c->graph_rows, c->n_pad, c->sm_count, c->p.j_tile, c->p.i_block, c->p.j_split,
                         &c->graph_cfg, c->p.j_sub) != NBODY_OK)
            c->graph_rows = -1;
    }
    int64_t tb = 0, na = 0;
    r = schedule_internal(c, &tb, &na);
    const bool cluster = cluster_steps(c);
    bool cluster_declined = false;  // the cluster kernel ran none of the blocks it was offered
    const bool grid = !cluster && grid_steps(c);
    bool grid_declined = false;  // likewise the whole-GPU kernel
    bool grid_pending = false;   // the next block is not scheduled on the host: the grid kernel schedules it
    if (grid && !c->grid_buf) {
        c->grid_rows = static_cast<int>(std::min<int64_t>(kGridRows, c->n));
        NB_CUDA(dev_alloc(&c->grid_buf, grid_step_bytes(c->p.mode, c->grid_rows, grid_step_size(c->p.mode))),
                "grid block-step scratch allocation");
    }
    while (r == NBODY_OK && tb <= tend && !(max_steps > 0 && done >= max_steps)) {
        if (cluster && !cluster_declined) {
            StepLoop *L = c->loop_host;
            const int64_t left = max_steps > 0 ? max_steps - done : kClusterCap;
            NB_CUDA(cluster_step_launch(c->p.mode, c->S, c->J, c->eps2, c->p.eta, c->p.lmin, c->p.lmax, tend,
                                        std::min(left, kClusterCap), c->n, c->t_pred, loop_stop_flags(c), c->st,
                                        c->sched_out, c->loop_dev, c->act_sched, c->s, &c->stats.kernel_launches),
                    "cluster block-step launch");
            NB_CUDA(cudaMemcpyAsync(L, c->loop_dev, sizeof(StepLoop), cudaMemcpyDeviceToHost, c->s), "loop read-back");
            NB_CUDA(cudaMemcpyAsync(c->sched_host, c->sched_out, sizeof(SchedOut), cudaMemcpyDeviceToHost, c->s),
                    "schedule read-back");
            NB_CUDA(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->s),
                    "status read-back");
            NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
            const int64_t blocks = L->blocks;
            c->stats.force_calls += blocks;
            c->stats.pairs += L->rows * (c->n - 1);
            c->stats.blocks += blocks;
            c->stats.cluster_blocks += blocks;
            if (blocks > 0) {
                c->t_max = std::max(c->t_max, static_cast<int64_t>(L->last_t));
                c->t_pred = L->last_t;
                c->pred_valid = false;
                c->force_n_act = -1;
            }
            done += blocks;
            r = absorb_status(c);
            if (r != NBODY_OK) break;
            tb = c->sched_host->t_blk;
            na = c->sched_host->n_act;
            cluster_declined = blocks == 0;  // that block takes the path below once
            continue;
        }
        if (grid && !grid_declined && (grid_pending || na <= c->grid_rows)) {
            grid_pending = false;
            StepLoop *L = c->loop_host;
            const int64_t left = max_steps > 0 ? max_steps - done : kClusterCap;
            NB_CUDA(grid_step_launch(c->p.mode, c->S, c->J, c->eps2, c->p.eta, c->p.lmin, c->p.lmax, tend,
                                     std::min(left, kClusterCap), c->grid_rows, c->t_pred, loop_stop_flags(c), c->st,
                                     c->sched_out, c->loop_dev, c->act_sched, c->grid_buf, c->s,
                                     &c->stats.kernel_launches),
                    "grid block-step launch");
            NB_CUDA(cudaMemcpyAsync(L, c->loop_dev, sizeof(StepLoop), cudaMemcpyDeviceToHost, c->s), "loop read-back");
            NB_CUDA(cudaMemcpyAsync(c->sched_host, c->sched_out, sizeof(SchedOut), cudaMemcpyDeviceToHost, c->s),
                    "schedule read-back");
            NB_CUDA(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->s),
                    "status read-back");
            NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
            const int64_t blocks = L->blocks;
            c->stats.force_calls += blocks;
            c->stats.pairs += L->rows * (c->n - 1);
            c->stats.blocks += blocks;
            c->stats.grid_blocks += blocks;
            if (blocks > 0) {
                c->t_max = std::max(c->t_max, static_cast<int64_t>(L->last_t));
                c->t_pred = L->last_t;
                c->pred_valid = false;
                c->force_n_act = -1;
            }
            if (L->predicted >= 0) {  // it stopped at a larger block and left the j-stream predicted to its time
                c->t_pred = L->predicted;
                c->pred_valid = true;
                c->force_n_act = -1;
            }
            done += blocks;
            r = absorb_status(c);
            if (r != NBODY_OK) break;
            tb = c->sched_host->t_blk;
            na = c->sched_host->n_act;
            grid_declined = blocks == 0;  // that block takes the path below once
            continue;
        }
        cluster_declined = false;
        grid_declined = false;
        ForceConfig cfg{};
        // (not beside the grid kernel: the graph's device loop would go on with the small blocks that follow)
        bool use_graph = !grid && g_step_graphs > 0 && packed && c->graph_rows > 0 && na <= c->graph_rows &&
                         force_choose(c->p.mode, na, c->n_pad, c->sm_count, c->p.j_tile, c->p.i_block,
                                      c->p.j_split, &cfg, c->p.j_sub) == NBODY_OK &&
                         same_shape(cfg, c->graph_cfg);
        if (use_graph) {
            r = build_step_graph(c);
            if (r != NBODY_OK) break;
            StepLoop *L = c->loop_host;
            if (c->graph_loop) {  // the first block is this one; the loop may add up to `budget` more
                const int64_t left = max_steps > 0 ? max_steps - done - 1 : kLoopCap;
                L->t_end = tend;
                L->budget = g_step_graphs >= 2 ? std::min(left, kLoopCap) : 0;
                L->blocks = 0;
                L->rows = 0;
                L->last_t = tb;
                NB_CUDA(cudaMemcpyAsync(c->loop_dev, L, sizeof(StepLoop), cudaMemcpyHostToDevice, c->s),
                        "loop control upload");
            }
            NB_CUDA(cudaGraphLaunch(c->step_graph, c->s), "step graph launch");
            NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
            const int64_t more = c->graph_loop ? L->blocks : 0;
            const int64_t last_t = c->graph_loop ? L->last_t : tb;
            const int64_t rows = na + (c->graph_loop ? L->rows : 0);
            c->stats.kernel_launches += (1 + more) * c->graph_launches;
            c->stats.force_calls += 1 + more;
            c->stats.pairs += rows * (c->n - 1);
            c->stats.blocks += 1 + more;
            c->stats.graph_blocks += 1 + more;
            c->stats.loop_blocks += more;
            c->stats.last_threads = cfg.threads;
            c->stats.last_i_per_thread = cfg.ipt;
            c->stats.last_j_split = cfg.split;
            c->stats.last_j_sub = cfg.jsub;
            c->t_max = std::max(c->t_max, last_t);
            c->t_pred = last_t;
            c->pred_valid = false;
            c->force_n_act = -1;
            done += 1 + more;
            r = absorb_status(c);
            if (r != NBODY_OK) break;
            tb = c->sched_host->t_blk;
            na = c->sched_host->n_act;
            continue;
        }
        if (!(grid && c->pred_valid && c->t_pred == tb)) {
            r = predict_internal(c, tb);
            if (r != NBODY_OK) break;
        }
        NB_CUDA(cudaMemcpyAsync(c->act_force, c->act_sched, static_cast<size_t>(na) * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, c->s),
                "list copy");
        r = force_internal(c, na, true);
        if (r != NBODY_OK) break;
        r = correct_internal(c, c->act_sched, na, c->f_acc, c->f_jerk, true);
        if (r != NBODY_OK) break;
        ++done;
        if (grid) {  // the grid kernel schedules the next block (and runs it, when it is small)
            grid_pending = true;
            continue;
        }
        r = schedule_internal(c, &tb, &na);
    }
    if (n_steps) *n_steps = done;
    if (r != NBODY_OK) return r;
    return sync_and_check(c);
}

int nbody_sync(nbody_ctx *c)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_sync: null context");
    return sync_and_check(c);
}

int nbody_energy(nbody_ctx *c, double *ekin, double *epot)
{
    if (!c || !ekin || !epot) return fail(NBODY_EINVAL, "nbody_energy: null argument");
    return energy_common(c, ekin, epot, false);
}

int nbody_energy_ds(nbody_ctx *c, double *ekin, double *epot)
{
    if (!c || !ekin || !epot) return fail(NBODY_EINVAL, "nbody_energy_ds: null argument");
    return energy_common(c, ekin, epot, true);
}

int nbody_get_state(nbody_ctx *c, double *x, double *v, double *a, double *k, int64_t *t_tick, int8_t *level)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_get_state: null context");
    const size_t nd = static_cast<size_t>(c->n);
    double *const *src[4] = {c->S.x, c->S.v, c->S.a, c->S.k};
    double *dst[4] = {x, v, a, k};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        double *tmp = c->stage + (q & 1) * 3 * nd;
        NB_CUDA(soa_to_aos_launch(src[q][0], src[q][1], src[q][2], tmp, c->n, c->s, &c->stats.kernel_launches),
                "layout kernel");
        NB_CUDA(cudaMemcpyAsync(dst[q], tmp, 3 * nd * sizeof(double), cudaMemcpyDefault, c->s), "state copy");
    }
    if (t_tick) NB_CUDA(cudaMemcpyAsync(t_tick, c->t, nd * sizeof(int64_t), cudaMemcpyDefault, c->s), "time copy");
    if (level) NB_CUDA(cudaMemcpyAsync(level, c->level, nd, cudaMemcpyDefault, c->s), "level copy");
    return sync_and_check(c);
}

int nbody_set_state(nbody_ctx *c, const double *x, const double *v, const double *a, const double *k,
                    const int64_t *t_tick, const int8_t *level)
{
    if (!c || !x || !v || !a || !k || !t_tick || !level) return fail(NBODY_EINVAL, "nbody_set_state: null argument");
    const size_t nd = static_cast<size_t>(c->n);
    std::vector<int64_t> th(nd);
    std::vector<int8_t> lh(nd);
    NB_CUDA(cudaMemcpy(th.data(), t_tick, nd * sizeof(int64_t), cudaMemcpyDefault), "time read");
    NB_CUDA(cudaMemcpy(lh.data(), level, nd, cudaMemcpyDefault), "level read");
    int64_t tmax = 0;
    for (size_t i = 0; i < nd; ++i) {
        const int L = lh[i];
        if (L < c->p.lmin || L > c->p.lmax) return fail(NBODY_EINVAL, "nbody_set_state: level[%zu] = %d out of range", i, L);
        const int64_t step = int64_t(1) << (c->p.lmax - L);
        if (th[i] < 0 || th[i] % step != 0)
            return fail(NBODY_EINVAL, "nbody_set_state: t_tick[%zu] is not a multiple of its step", i);
        tmax = std::max(tmax, th[i]);
    }
    NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
    const double *srcs[4] = {x, v, a, k};
    double **dsts[4] = {c->S.x, c->S.v, c->S.a, c->S.k};
    for (int q = 0; q < 4; ++q) {
        double *tmp = c->stage + (q & 1) * 3 * nd;
        NB_CUDA(to_device(tmp, srcs[q], 3 * nd * sizeof(double), c->s), "state upload");
        NB_CUDA(aos_to_soa_launch(tmp, dsts[q][0], dsts[q][1], dsts[q][2], c->n, c->s, &c->stats.kernel_launches),
                "layout kernel");
    }
    NB_CUDA(cudaMemcpyAsync(c->t, th.data(), nd * sizeof(int64_t), cudaMemcpyHostToDevice, c->s), "time upload");
    NB_CUDA(cudaMemcpyAsync(c->level, lh.data(), nd, cudaMemcpyHostToDevice, c->s), "level upload");
    c->t_max = tmax;
    c->pred_valid = false;
    c->force_n_act = -1;
    return sync_and_check(c);
}

int nbody_get_predicted(nbody_ctx *c, float *posm, float *vel, float *poslo)
{
    if (!c) return fail(NBODY_EINVAL, "nbody_get_predicted: null context");
    if (!c->pred_valid) return fail(NBODY_ESTATE, "nbody_get_predicted: no current prediction");
    const size_t bytes = static_cast<size_t>(c->n) * sizeof(float4);
    if (!c->J.aos && (posm || vel || poslo))  // this context's predictor writes the SoA stream only
        NB_CUDA(aos_from_soa_launch(c->J, c->n, c->s, &c->stats.kernel_launches), "layout kernel");
    if (posm) NB_CUDA(cudaMemcpyAsync(posm, c->J.posm, bytes, cudaMemcpyDefault, c->s), "j-stream copy");
    if (vel) NB_CUDA(cudaMemcpyAsync(vel, c->J.vel, bytes, cudaMemcpyDefault, c->s), "j-stream copy");
    if (poslo) NB_CUDA(cudaMemcpyAsync(poslo, c->J.poslo, bytes, cudaMemcpyDefault, c->s), "j-stream copy");
    return sync_and_check(c);
}

int nbody_get_stats(nbody_ctx *c, nbody_stats *s)
{
    if (!c || !s) return fail(NBODY_EINVAL, "nbody_get_stats: null argument");
    NB_CUDA(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->s), "status read-back");
    NB_CUDA(cudaStreamSynchronize(c->s), "stream synchronise");
    c->stats.below_dt_min = static_cast<int64_t>(c->st_host->below_min);
    c->stats.nonfinite = static_cast<int64_t>(c->st_host->nonfinite);
    *s = c->stats;
    return NBODY_OK;
}


int nbody_diff_rollout(int64_t n, const double *m, const double *x0, const double *v0, double eps2, int level,
                       int64_t steps, int64_t checkpoint_every, int mode, double *loss, double *g_x0,
                       double *g_v0, double *g_m, void *stream)
{
    if (!loss || !g_x0 || !g_v0 || !g_m) return fail(NBODY_EINVAL, "nbody_diff_rollout: null argument");
    return rollout_impl("nbody_diff_rollout", n, m, x0, v0, eps2, level, steps, checkpoint_every, mode, true, true,
                        nullptr, nullptr, loss, nullptr, nullptr, g_x0, g_v0, g_m, stream);
}

int nbody_rollout(int64_t n, const double *m, const double *x0, const double *v0, double eps2, int level,
                  int64_t steps, int mode, double *x_T, double *v_T, void *stream)
{
    if (!x_T && !v_T) return fail(NBODY_EINVAL, "nbody_rollout: no output");
    return rollout_impl("nbody_rollout", n, m, x0, v0, eps2, level, steps, 0, mode, false, false, nullptr, nullptr,
                        nullptr, x_T, v_T, nullptr, nullptr, nullptr, stream);
}

int nbody_rollout_vjp(int64_t n, const double *m, const double *x0, const double *v0, double eps2, int level,
                      int64_t steps, int64_t checkpoint_every, int mode, const double *g_xT, const double *g_vT,
                      double *g_x0, double *g_v0, double *g_m, void *stream)
{
    if (!g_x0 && !g_v0 && !g_m) return fail(NBODY_EINVAL, "nbody_rollout_vjp: no output");
    return rollout_impl("nbody_rollout_vjp", n, m, x0, v0, eps2, level, steps, checkpoint_every, mode, true, false,
                        g_xT, g_vT, nullptr, nullptr, nullptr, g_x0, g_v0, g_m, stream);
}

void nbody_free(nbody_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->s);
    release(c);
}

const char *nbody_strerror(int code)
{
    switch (code) {
    case NBODY_OK: return "success";
    case NBODY_EINVAL: return "invalid argument";
    case NBODY_ENOMEM: return "out of memory";
    case NBODY_ECUDA: return "CUDA runtime error";
    case NBODY_EDTMIN: return "time step below dt_min";
    case NBODY_ENONFINITE: return "non-finite force or state";
    case NBODY_ENOTSYNC: return "particles not at a common time";
    case NBODY_ETIMEOUT: return "device-side wait timed out";
    case NBODY_ESTATE: return "call out of order";
    default: return "unknown error code";
    }
}

const char *nbody_last_error(void) { return g_err; }

void nbody_debug_fail_alloc(int k) { g_fail_alloc = k > 0 ? k : 0; }

void nbody_debug_skip_tile_copy(int on) { nb::g_skip_first_copy = on ? 1 : 0; }

void nbody_debug_step_graphs(int level) { g_step_graphs = level < 0 ? 0 : (level > 3 ? 3 : level); }

}  // extern "C"

/*
 * FP64 CPU oracle of the 4th-order Hermite block-time-step N-body method of
 * Portegies Zwart, Belleman & Geldof (2007), "High Performance Direct
 * Gravitational N-body Simulations on Graphics Processing Units".
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the library itself never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Everything is plain, sequential-in-j FP64 arithmetic, written in the
 * order and notation of Sect. 2 of the paper; OpenMP only spreads
 * independent particles i over threads (each i is summed alone, in
 * ascending j, so results do not depend on the thread count).
 *
 * Conventions (shared with the library's public API, nothing else):
 *   - G = 1; positions, velocities, accelerations, jerks are n x 3 row-major
 *     (x0 y0 z0 x1 y1 z1 ...) arrays of double.
 *   - Time is kept as an int64 count of ticks of dt_min = 2^-lmax.
 *   - A time step is a power of two dt = 2^-level with lmin <= level <= lmax
 *     (dt_max = 2^-lmin, dt_min = 2^-lmax).
 */
#ifndef NBODY_ORACLE_H
#define NBODY_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

void orc_set_threads(int n);
int orc_get_threads(void);

/* Acceleration, jerk and potential on each listed particle i from all j != i.
 * Pair term of Appendix A (dx = x_j - x_i, Plummer softening eps2) which fixes
 * the sign of Eq. (Force); the sum excludes j = i as Eq. (Force) states.
 * acc, jerk: n_act x 3; pot: n_act.  Any output may be NULL. */
void orc_force(int64_t n, const double *m, const double *x, const double *v,
               double eps2, int64_t n_act, const int32_t *active,
               double *acc, double *jerk, double *pot);

/* Correctly rounded (to nearest, ties to even) single-precision 1/sqrt(r2)
 * for a positive normal float r2, by exact integer comparison of squared
 * rounding midpoints against 1/r2.  Returns NaN for r2 <= 0 or non-finite. */
float orc_rsqrt_rn_f32(float r2);

/* The summation check of the compensated force (reading of the 1e-10
 * summation bound): the same listed sums as orc_force, but every pair term is
 * first formed in single precision exactly as the compensated pair term
 * computes it with correctly rounded operations in a fixed order:
 *   hi = fl32(x), lo = fl32(x - hi), u = fl32(v), mu = fl32(m), e2 = fl32(eps2);
 *   dx = (hi_j - hi_i) + (lo_j - lo_i);  dv = u_j - u_i;
 *   r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, e2)));  rinv = rsqrt_rn(r2);
 *   xv = fma(dz, dvz, fma(dy, dvy, dx * dvx));
 *   mr = mu_j * rinv;  mr3 = mr * (rinv * rinv);  w = 3 * (xv * (rinv * rinv));
 *   terms: mr3 * dx_c,  mr3 * fma(-w, dx_c, dv_c),  -mr.
 * Each term is then summed over j in ascending order in FP64 with Neumaier's
 * compensation, so the result is the sum of those FP32 terms to ~1e-16. */
void orc_force_fp32_terms(int64_t n, const double *m, const double *x, const double *v,
                          double eps2, int64_t n_act, const int32_t *active,
                          double *acc, double *jerk, double *pot);

/* Sorted-summation ablation (Sect. 6 of the paper: add the forces by size,
 * smallest first).  The plain pair terms in single precision, from
 * hi = fl32(x), u = fl32(v), mu = fl32(m), e2 = fl32(eps2):
 *   dx = hi_j - hi_i;  dv = u_j - u_i;  then as orc_force_fp32_terms;
 * for each listed i and each of the 7 components, the terms over j != i are
 * sorted by magnitude (ties: by the raw bits as unsigned integers, so -x after
 * x) and added in FP32 from the smallest.  Exact in the sense that every step
 * is one correctly rounded single-precision operation. */
void orc_force_sorted_fp32(int64_t n, const double *m, const double *x, const double *v,
                           double eps2, int64_t n_act, const int32_t *active,
                           double *acc, double *jerk, double *pot);

/* Predictor of Sect. 2: every particle from its own time t_tick[i] to t_new. */
void orc_predict(int64_t n, const double *x, const double *v, const double *a,
                 const double *k, const int64_t *t_tick, int64_t t_new, int lmax,
                 double *xp, double *vp);

/* Eq. (initTimestep): dt = eta |a| / |k| (INFINITY when |k| = 0). */
double orc_dt_initial(const double *a, const double *k, double eta);

/* Eq. (timestep) with end-of-step quantities: a1 = a_p, k1 = k_p,
 * a2e = a^(2) + a^(3) dt, a3 = a^(3).  INFINITY when the denominator is 0. */
double orc_dt_aarseth(const double *a1, const double *k1, const double *a2e,
                      const double *a3, double eta);

/* Smallest level L with 2^-L <= dt, clamped to [lmin, lmax].  *below_min is
 * set to 1 when dt < 2^-lmax (the clamp raised the step), else 0.
 * dt <= 0 gives lmax with *below_min = 1; NaN gives -1. */
int orc_level_floor(double dt, int lmin, int lmax, int *below_min);

/* Power-of-two block rule for the level after a step ending at tick t_new:
 * shrink to l_crit at once; grow by one level at most, and only when t_new
 * is a multiple of twice the old step. */
int orc_next_level(int l_old, int l_crit, int64_t t_new, int lmin, int lmax);

/* Block scheduler (Sect. 2, integration-step list): t_blk = min_i (t_i + dt_i),
 * active = every i with t_i + dt_i == t_blk, ascending.  Returns n_act. */
int64_t orc_schedule(int64_t n, const int64_t *t_tick, const int8_t *level,
                     int lmax, int64_t *t_blk, int32_t *active);

/* Corrector of Sect. 2 on the listed particles, followed by the new time step.
 * xp, vp: predicted state of all n particles (orc_predict to t_new);
 * acc_new, jerk_new: n_act x 3 forces at the predicted state.
 * Updates x, v, a, k, t_tick, level of the listed particles in place.
 * dt_crit (n_act, may be NULL) receives the unquantised criterion.
 * Returns the number of listed particles with a non-finite result;
 * *n_below_min (may be NULL) is incremented per clamp at dt_min. */
int64_t orc_correct(int64_t n_act, const int32_t *active,
                    double *x, double *v, double *a, double *k,
                    int64_t *t_tick, int8_t *level,
                    const double *xp, const double *vp,
                    const double *acc_new, const double *jerk_new,
                    int64_t t_new, double eta, int lmin, int lmax,
                    double *dt_crit, int64_t *n_below_min);

/* Start of a run (Sect. 2): full force on all particles at t = 0, then the
 * initial level from Eq. (initTimestep).  Sets a, k, t_tick = 0, level. */
void orc_init(int64_t n, const double *m, const double *x, const double *v,
              double eps2, double eta_init, int lmin, int lmax,
              double *a, double *k, int64_t *t_tick, int8_t *level,
              int64_t *n_below_min);

/* Kinetic and potential energy: sum m v^2 / 2 and sum_i m_i phi_i / 2 with
 * the softened phi_i of Appendix A, excluding j = i. */
void orc_energy(int64_t n, const double *m, const double *x, const double *v,
                double eps2, double *ekin, double *epot);

/* Block steps (Sect. 2 step list) until the next block would pass t_end_tick
 * or max_blocks blocks are done.  Records per block t_blk (blk_t) and n_act
 * (blk_n), and appends the active lists to blk_lists while list_cap allows
 * (any of the three may be NULL).  Returns the number of blocks done, or
 * -(blocks done) - 1 when a non-finite state stopped the run. */
int64_t orc_evolve(int64_t n, const double *m, double *x, double *v,
                   double *a, double *k, int64_t *t_tick, int8_t *level,
                   double eps2, double eta, int lmin, int lmax,
                   int64_t t_end_tick, int64_t max_blocks,
                   int64_t *blk_t, int64_t *blk_n,
                   int32_t *blk_lists, int64_t list_cap,
                   int64_t *n_below_min);

#ifdef __cplusplus
}
#endif
#endif

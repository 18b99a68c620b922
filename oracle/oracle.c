/*
 * FP64 CPU oracle of the Hermite-4 block-time-step method (Portegies Zwart,
 * Belleman & Geldof 2007, Sect. 2 and Appendix A).  TEST INFRASTRUCTURE
 * ONLY: see oracle.h.  Built with -ffp-contract=off so that x86 and Arm
 * hosts give identical bits.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double norm3(const double *u) { return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

/* Appendix A pair term, summed over j != i (Eq. Force).  For particle i:
 *   dx = x_j - x_i, dv = v_j - v_i, r^2 = eps^2 + dx.dx
 *   a   += m_j dx / r^3
 *   k   += m_j (dv / r^3 - 3 (dx.dv) dx / r^5)
 *   phi -= m_j / r                                                       */
void orc_force(int64_t n, const double *m, const double *x, const double *v,
               double eps2, int64_t n_act, const int32_t *active,
               double *acc, double *jerk, double *pot)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n_act; q++) {
        const int64_t i = active[q];
        double ai[3] = {0, 0, 0}, ki[3] = {0, 0, 0}, phi = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx[3], dv[3];
            for (int c = 0; c < 3; c++) {
                dx[c] = x[3 * j + c] - x[3 * i + c];
                dv[c] = v[3 * j + c] - v[3 * i + c];
            }
            const double r2 = eps2 + dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
            const double xv = dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2];
            const double rinv = 1.0 / sqrt(r2);
            const double r3inv = rinv * rinv * rinv;
            const double r5inv = r3inv * rinv * rinv;
            for (int c = 0; c < 3; c++) {
                ai[c] += m[j] * dx[c] * r3inv;
                ki[c] += m[j] * (dv[c] * r3inv - 3.0 * xv * dx[c] * r5inv);
            }
            phi -= m[j] * rinv;
        }
        for (int c = 0; c < 3; c++) {
            if (acc) acc[3 * q + c] = ai[c];
            if (jerk) jerk[3 * q + c] = ki[c];
        }
        if (pot) pot[q] = phi;
    }
}

/* Decomposes a positive finite float g as G * 2^e with G a 24-bit integer. */
static void f32_parts(float g, uint64_t *G, int *e)
{
    int k;
    const float fr = frexpf(g, &k); /* g = fr * 2^k, 0.5 <= fr < 1 */
    *G = (uint64_t)ldexpf(fr, 24);
    *e = k - 24;
}

/* Sign of mid^2 * r2 - 1, mid the midpoint of the positive floats a < b,
 * computed exactly in 128-bit integers. */
static int mid_sq_times_cmp1(float a, float b, float r2)
{
    uint64_t A, B, R;
    int ea, eb, er;
    f32_parts(a, &A, &ea);
    f32_parts(b, &B, &eb);
    f32_parts(r2, &R, &er);
    const int e0 = ea < eb ? ea : eb;
    /* a + b = S * 2^e0, mid = S * 2^(e0 - 1), S < 2^26 */
    const uint64_t S = (A << (ea - e0)) + (B << (eb - e0));
    const unsigned __int128 P = (unsigned __int128)(S * S) * R; /* < 2^76 */
    const int K = 2 * (e0 - 1) + er;                            /* mid^2 r2 = P * 2^K */
    if (K >= 0) return 1;                                        /* P >= 1 */
    if (-K >= 127) return -1;
    const unsigned __int128 one = (unsigned __int128)1 << (-K);
    return P < one ? -1 : (P > one ? 1 : 0);
}

float orc_rsqrt_rn_f32(float r2)
{
    if (!(r2 > 0.0f) || !isfinite(r2) || !isnormal(r2)) return NAN;
    float f = (float)(1.0 / sqrt((double)r2));
    for (int it = 0; it < 8; it++) {
        /* 1/sqrt(r2) > mid  <=>  mid^2 r2 < 1 (everything positive) */
        const float up = nextafterf(f, INFINITY);
        if (mid_sq_times_cmp1(f, up, r2) < 0) {
            f = up;
            continue;
        }
        const float dn = nextafterf(f, 0.0f);
        if (mid_sq_times_cmp1(dn, f, r2) > 0) {
            f = dn;
            continue;
        }
        break; /* a tie (mid^2 r2 == 1) would need S = 1; S is odd and > 1 */
    }
    return f;
}

/* Neumaier's compensated summation step (Neumaier 1974). */
static void neumaier_add(double *s, double *c, double t)
{
    const double u = *s + t;
    if (fabs(*s) >= fabs(t))
        *c += (*s - u) + t;
    else
        *c += (t - u) + *s;
    *s = u;
}

void orc_force_fp32_terms(int64_t n, const double *m, const double *x, const double *v,
                          double eps2, int64_t n_act, const int32_t *active,
                          double *acc, double *jerk, double *pot)
{
    const float e2 = (float)eps2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n_act; q++) {
        const int64_t i = active[q];
        float hi_i[3], lo_i[3], u_i[3];
        for (int c = 0; c < 3; c++) {
            hi_i[c] = (float)x[3 * i + c];
            lo_i[c] = (float)(x[3 * i + c] - (double)hi_i[c]);
            u_i[c] = (float)v[3 * i + c];
        }
        double s[7] = {0}, cmp[7] = {0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            float dx[3], dv[3];
            for (int c = 0; c < 3; c++) {
                const float hj = (float)x[3 * j + c];
                const float lj = (float)(x[3 * j + c] - (double)hj);
                dx[c] = (hj - hi_i[c]) + (lj - lo_i[c]);
                dv[c] = (float)v[3 * j + c] - u_i[c];
            }
            const float r2 = fmaf(dx[2], dx[2], fmaf(dx[1], dx[1], fmaf(dx[0], dx[0], e2)));
            const float rinv = orc_rsqrt_rn_f32(r2);
            const float xv = fmaf(dx[2], dv[2], fmaf(dx[1], dv[1], dx[0] * dv[0]));
            const float rinv2 = rinv * rinv;
            const float mr = (float)m[j] * rinv;
            const float mr3 = mr * rinv2;
            const float w = 3.0f * (xv * rinv2);
            for (int c = 0; c < 3; c++) {
                neumaier_add(&s[c], &cmp[c], (double)(mr3 * dx[c]));
                neumaier_add(&s[3 + c], &cmp[3 + c], (double)(mr3 * fmaf(-w, dx[c], dv[c])));
            }
            neumaier_add(&s[6], &cmp[6], (double)(-mr));
        }
        for (int c = 0; c < 3; c++) {
            if (acc) acc[3 * q + c] = s[c] + cmp[c];
            if (jerk) jerk[3 * q + c] = s[3 + c] + cmp[3 + c];
        }
        if (pot) pot[q] = s[6] + cmp[6];
    }
}

static uint32_t f32_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

/* Order by magnitude, then by the raw bits. */
static int cmp_size(const void *pa, const void *pb)
{
    const uint32_t a = f32_bits(*(const float *)pa), b = f32_bits(*(const float *)pb);
    const uint32_t ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;
    if (ma != mb) return ma < mb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

void orc_force_sorted_fp32(int64_t n, const double *m, const double *x, const double *v,
                           double eps2, int64_t n_act, const int32_t *active,
                           double *acc, double *jerk, double *pot)
{
    const float e2 = (float)eps2;
#pragma omp parallel
    {
        float *t[7];
        for (int c = 0; c < 7; c++) t[c] = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < n_act; q++) {
            const int64_t i = active[q];
            float hi_i[3], u_i[3];
            for (int c = 0; c < 3; c++) {
                hi_i[c] = (float)x[3 * i + c];
                u_i[c] = (float)v[3 * i + c];
            }
            int64_t cnt = 0;
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                float dx[3], dv[3];
                for (int c = 0; c < 3; c++) {
                    dx[c] = (float)x[3 * j + c] - hi_i[c];
                    dv[c] = (float)v[3 * j + c] - u_i[c];
                }
                const float r2 = fmaf(dx[2], dx[2], fmaf(dx[1], dx[1], fmaf(dx[0], dx[0], e2)));
                const float rinv = orc_rsqrt_rn_f32(r2);
                const float xv = fmaf(dx[2], dv[2], fmaf(dx[1], dv[1], dx[0] * dv[0]));
                const float rinv2 = rinv * rinv;
                const float mr = (float)m[j] * rinv;
                const float mr3 = mr * rinv2;
                const float w = 3.0f * (xv * rinv2);
                for (int c = 0; c < 3; c++) {
                    t[c][cnt] = mr3 * dx[c];
                    t[3 + c][cnt] = mr3 * fmaf(-w, dx[c], dv[c]);
                }
                t[6][cnt] = -mr;
                cnt++;
            }
            float sum[7];
            for (int c = 0; c < 7; c++) {
                qsort(t[c], (size_t)cnt, sizeof(float), cmp_size);
                float s = 0.0f;
                for (int64_t k = 0; k < cnt; k++) s = s + t[c][k];
                sum[c] = s;
            }
            for (int c = 0; c < 3; c++) {
                if (acc) acc[3 * q + c] = (double)sum[c];
                if (jerk) jerk[3 * q + c] = (double)sum[3 + c];
            }
            if (pot) pot[q] = (double)sum[6];
        }
        for (int c = 0; c < 7; c++) free(t[c]);
    }
}

/* Predictor, Sect. 2: x_p = x + v dt + a dt^2/2 + k dt^3/6,
 *                     v_p = v + a dt + k dt^2/2,  dt = t_new - t_i.      */
void orc_predict(int64_t n, const double *x, const double *v, const double *a,
                 const double *k, const int64_t *t_tick, int64_t t_new, int lmax,
                 double *xp, double *vp)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        const double dt = ldexp((double)(t_new - t_tick[i]), -lmax);
        const double dt2 = dt * dt, dt3 = dt2 * dt;
        for (int c = 0; c < 3; c++) {
            const int64_t e = 3 * i + c;
            xp[e] = x[e] + v[e] * dt + a[e] * dt2 / 2.0 + k[e] * dt3 / 6.0;
            vp[e] = v[e] + a[e] * dt + k[e] * dt2 / 2.0;
        }
    }
}

/* Eq. (initTimestep), read as dt = eta |a| / |k|. */
double orc_dt_initial(const double *a, const double *k, double eta)
{
    const double kn = norm3(k);
    if (kn == 0.0) return INFINITY;
    return eta * norm3(a) / kn;
}

/* Eq. (timestep): dt = [eta (|a||a2| + |k|^2) / (|k||a3| + |a2|^2)]^(1/2),
 * with "k^2" and "a2^2" read as squared norms. */
double orc_dt_aarseth(const double *a1, const double *k1, const double *a2e,
                      const double *a3, double eta)
{
    const double an = norm3(a1), kn = norm3(k1), a2n = norm3(a2e), a3n = norm3(a3);
    const double num = an * a2n + kn * kn;
    const double den = kn * a3n + a2n * a2n;
    if (den == 0.0) return INFINITY;
    return sqrt(eta * num / den);
}

/* Time steps are powers of two (Sect. 2, block list) between
 * dt_max = 2^-lmin and dt_min = 2^-lmax (Sect. 4 setup). */
int orc_level_floor(double dt, int lmin, int lmax, int *below_min)
{
    if (below_min) *below_min = 0;
    if (isnan(dt)) return -1;
    if (dt <= 0.0) {                      /* criterion collapsed: smallest step */
        if (below_min) *below_min = 1;
        return lmax;
    }
    if (isinf(dt)) return lmin;
    int e;
    (void)frexp(dt, &e);      /* dt = f 2^e, 0.5 <= f < 1: largest 2^-L <= dt is 2^(e-1) */
    int L = 1 - e;
    if (L < lmin) L = lmin;
    if (L > lmax) {
        L = lmax;
        if (below_min) *below_min = 1;
    }
    return L;
}

int orc_next_level(int l_old, int l_crit, int64_t t_new, int lmin, int lmax)
{
    (void)lmax;
    if (l_crit >= l_old) return l_crit;                 /* same or smaller step */
    const int64_t two_dt_old = (int64_t)2 << (lmax - l_old);
    if (l_old - 1 >= lmin && t_new % two_dt_old == 0) return l_old - 1;
    return l_old;
}

int64_t orc_schedule(int64_t n, const int64_t *t_tick, const int8_t *level,
                     int lmax, int64_t *t_blk, int32_t *active)
{
    int64_t tmin = INT64_MAX;
    for (int64_t i = 0; i < n; i++) {
        const int64_t tn = t_tick[i] + ((int64_t)1 << (lmax - level[i]));
        if (tn < tmin) tmin = tn;
    }
    int64_t na = 0;
    for (int64_t i = 0; i < n; i++) {
        const int64_t tn = t_tick[i] + ((int64_t)1 << (lmax - level[i]));
        if (tn == tmin) active[na++] = (int32_t)i;
    }
    *t_blk = tmin;
    return na;
}

/* Corrector of Sect. 2 (notation of the paper: "a-double-dot" is a^(2),
 * "k-double-dot" is a^(3); Delta a = a - a_p), then Eq. (timestep). */
int64_t orc_correct(int64_t n_act, const int32_t *active,
                    double *x, double *v, double *a, double *k,
                    int64_t *t_tick, int8_t *level,
                    const double *xp, const double *vp,
                    const double *acc_new, const double *jerk_new,
                    int64_t t_new, double eta, int lmin, int lmax,
                    double *dt_crit, int64_t *n_below_min)
{
    int64_t bad = 0, below = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad, below)
    for (int64_t q = 0; q < n_act; q++) {
        const int64_t i = active[q];
        const double dt = ldexp((double)(t_new - t_tick[i]), -lmax);
        const double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
        double a2[3], a3[3], a2e[3], xn[3], vn[3];
        const double *ap = acc_new + 3 * q, *kp = jerk_new + 3 * q;
        int finite = 1;
        for (int c = 0; c < 3; c++) {
            const int64_t e = 3 * i + c;
            const double da = a[e] - ap[c];
            a2[c] = -6.0 * da / dt2 - (4.0 * k[e] + 2.0 * kp[c]) / dt;
            a3[c] = 12.0 * da / dt3 + 6.0 * (k[e] + kp[c]) / dt2;
            xn[c] = xp[e] + a2[c] / 24.0 * dt4 + a3[c] / 120.0 * dt5;
            vn[c] = vp[e] + a2[c] / 6.0 * dt3 + a3[c] / 24.0 * dt4;
            a2e[c] = a2[c] + a3[c] * dt;
            if (!isfinite(xn[c]) || !isfinite(vn[c]) || !isfinite(ap[c]) || !isfinite(kp[c]))
                finite = 0;
        }
        const double dtc = orc_dt_aarseth(ap, kp, a2e, a3, eta);
        if (dt_crit) dt_crit[q] = dtc;
        int bm = 0;
        const int lc = orc_level_floor(dtc, lmin, lmax, &bm);
        below += bm;
        for (int c = 0; c < 3; c++) {
            const int64_t e = 3 * i + c;
            x[e] = xn[c];
            v[e] = vn[c];
            a[e] = ap[c];
            k[e] = kp[c];
        }
        t_tick[i] = t_new;
        if (!finite || lc < 0) {
            bad += 1;
            level[i] = (int8_t)lmax;
        } else {
            level[i] = (int8_t)orc_next_level(level[i], lc, t_new, lmin, lmax);
        }
    }
    if (n_below_min) *n_below_min += below;
    return bad;
}

void orc_init(int64_t n, const double *m, const double *x, const double *v,
              double eps2, double eta_init, int lmin, int lmax,
              double *a, double *k, int64_t *t_tick, int8_t *level,
              int64_t *n_below_min)
{
    int32_t *all = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) all[i] = (int32_t)i;
    orc_force(n, m, x, v, eps2, n, all, a, k, NULL);
    free(all);
    int64_t below = 0;
    for (int64_t i = 0; i < n; i++) {
        int bm = 0;
        int L = orc_level_floor(orc_dt_initial(a + 3 * i, k + 3 * i, eta_init), lmin, lmax, &bm);
        if (L < 0) L = lmax;
        below += bm;
        level[i] = (int8_t)L;
        t_tick[i] = 0;
    }
    if (n_below_min) *n_below_min += below;
}

void orc_energy(int64_t n, const double *m, const double *x, const double *v,
                double eps2, double *ekin, double *epot)
{
    double *phi = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double p = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double r2 = eps2;
            for (int c = 0; c < 3; c++) {
                const double d = x[3 * j + c] - x[3 * i + c];
                r2 += d * d;
            }
            p -= m[j] / sqrt(r2);
        }
        phi[i] = p;
    }
    double ek = 0.0, ep = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double *vi = v + 3 * i;
        ek += 0.5 * m[i] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
        ep += 0.5 * m[i] * phi[i];
    }
    free(phi);
    *ekin = ek;
    *epot = ep;
}

int64_t orc_evolve(int64_t n, const double *m, double *x, double *v,
                   double *a, double *k, int64_t *t_tick, int8_t *level,
                   double eps2, double eta, int lmin, int lmax,
                   int64_t t_end_tick, int64_t max_blocks,
                   int64_t *blk_t, int64_t *blk_n,
                   int32_t *blk_lists, int64_t list_cap,
                   int64_t *n_below_min)
{
    const size_t n3 = (size_t)3 * (size_t)(n > 0 ? n : 1);
    double *xp = (double *)malloc(sizeof(double) * n3);
    double *vp = (double *)malloc(sizeof(double) * n3);
    double *an = (double *)malloc(sizeof(double) * n3);
    double *kn = (double *)malloc(sizeof(double) * n3);
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t nb = 0, used = 0, result;
    int lists_full = 0;
    for (;;) {
        if (nb >= max_blocks) { result = nb; break; }
        int64_t t_blk;
        const int64_t na = orc_schedule(n, t_tick, level, lmax, &t_blk, act);
        if (t_blk > t_end_tick) { result = nb; break; }
        orc_predict(n, x, v, a, k, t_tick, t_blk, lmax, xp, vp);
        orc_force(n, m, xp, vp, eps2, na, act, an, kn, NULL);
        const int64_t bad = orc_correct(na, act, x, v, a, k, t_tick, level, xp, vp, an, kn,
                                        t_blk, eta, lmin, lmax, NULL, n_below_min);
        if (blk_t) blk_t[nb] = t_blk;
        if (blk_n) blk_n[nb] = na;
        if (blk_lists && !lists_full) {
            if (used + na <= list_cap) {
                memcpy(blk_lists + used, act, sizeof(int32_t) * (size_t)na);
                used += na;
            } else {
                lists_full = 1;
            }
        }
        nb++;
        if (bad) { result = -nb - 1; break; }
    }
    free(xp); free(vp); free(an); free(kn); free(act);
    return result;
}

/*
 * hg_oracle.c -- plain, slow, single-threaded FP64 oracle of the 6th-order
 * Hermite block-timestep direct-summation integrator described in
 * Capuzzo-Dolcetta, Spera & Punzo, "A fully parallel, high precision, N-body
 * code running on hybrid computing platforms" (HiGPUs), Sect. 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The CUDA library never
 * includes, links or calls it, and it shares no code with the CUDA library.
 *
 * Everything is IEEE double, evaluated term by term in the order the paper
 * writes it; build with -ffp-contract=off so that x86 and Arm give identical
 * bits.  Units: G = 1.  Vectors are [n][3] row-major doubles.
 *
 * Readings where the paper is silent or garbled (each is marked "Reading"):
 *  R1  softening enters every r_ij^2, including the ones in alpha and beta
 *      (Sect. 2, softened potential; the evaluation equations omit it);
 *  R2  the bare "6 alpha" in the snap equation is alpha_ij;
 *  R3  in the snap term a_ij is the difference of predicted total
 *      accelerations a_j,pred - a_i,pred, as defined under the equations;
 *  R4  the predictor's time argument is the elapsed time t_block - t_j;
 *  R5  crackle (needed by the predictor), pop and the 5th derivative (needed by
 *      the p = 6 criterion) come from the degree-5 Hermite interpolant through
 *      a, jerk, snap at both ends of the step; crackle starts at zero;
 *  R6  the first step uses the criterion with p = 4 and its own accuracy
 *      parameter eta_init (crackle = 0, so A^(2) = |snap|);
 *  R7  power-of-two blocks: shrink to the largest 2^k <= criterion; grow at
 *      most x2 per step and only when the new time is a multiple of the
 *      doubled step; clamp to [dt_min, dt_max];
 *  R8  the potential energy is -sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps^2).
 * Besides the paper's 6th-order scheme the integrator offers the 4th-order
 * Hermite scheme its criterion admits with p = 4 (or_correct4, or_interp4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double dot3(const double *p, const double *q) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; }
static double norm3(const double *p) { return sqrt(dot3(p, p)); }

/* Sect. 3 item 1 (prediction step): Taylor series of position to crackle*h^5/120,
 * velocity to crackle*h^4/24 and acceleration to crackle*h^3/6, with h the time
 * elapsed since each particle's own time (Reading R4). */
void or_predict(int64_t n, const double *x, const double *v, const double *a, const double *jk,
                const double *s, const double *c, const double *t, double t_to,
                double *xp, double *vp, double *ap)
{
    for (int64_t i = 0; i < n; ++i) {
        double h = t_to - t[i];
        double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
        for (int k = 0; k < 3; ++k) {
            int64_t q = 3 * i + k;
            xp[q] = x[q] + v[q] * h + a[q] * h2 / 2.0 + jk[q] * h3 / 6.0 + s[q] * h4 / 24.0 + c[q] * h5 / 120.0;
            vp[q] = v[q] + a[q] * h + jk[q] * h2 / 2.0 + s[q] * h3 / 6.0 + c[q] * h4 / 24.0;
            ap[q] = a[q] + jk[q] * h + s[q] * h2 / 2.0 + c[q] * h3 / 6.0;
        }
    }
}

/* Sect. 3 item 2 (evaluation step): for each listed i, the sums over j != i of
 *   a_ij = m_j r_ij / r^3,
 *   j_ij = m_j v_ij / r^3 - 3 alpha a_ij,
 *   s_ij = m_j a_ij / r^3 - 6 alpha j_ij - 3 beta a_ij,
 * with r_ij = r_j - r_i, v_ij, a_ij the differences of predicted data,
 * r^2 = |r_ij|^2 + eps^2 (R1), alpha r^2 = r.v, beta r^2 = v^2 + r.a + alpha^2 r^2
 * (R2, R3).  Sums run over j in index order. */
void or_eval(int64_t n, const double *mass, const double *xp, const double *vp, const double *ap,
             double eps, int64_t n_act, const int32_t *idx, double *acc, double *jerk, double *snap)
{
    for (int64_t q = 0; q < n_act; ++q) {
        int64_t i = idx[q];
        double A[3] = {0, 0, 0}, J[3] = {0, 0, 0}, S[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r[3], v[3], a[3];
            for (int k = 0; k < 3; ++k) {
                r[k] = xp[3 * j + k] - xp[3 * i + k];
                v[k] = vp[3 * j + k] - vp[3 * i + k];
                a[k] = ap[3 * j + k] - ap[3 * i + k];
            }
            double r2 = dot3(r, r) + eps * eps;
            double alpha = dot3(r, v) / r2;
            double beta = (dot3(v, v) + dot3(r, a)) / r2 + alpha * alpha;
            double r3 = r2 * sqrt(r2);
            for (int k = 0; k < 3; ++k) {
                double aij = mass[j] * r[k] / r3;
                double jij = mass[j] * v[k] / r3 - 3.0 * alpha * aij;
                double sij = mass[j] * a[k] / r3 - 6.0 * alpha * jij - 3.0 * beta * aij;
                A[k] += aij;
                J[k] += jij;
                S[k] += sij;
            }
        }
        for (int k = 0; k < 3; ++k) {
            acc[3 * q + k] = A[k];
            jerk[3 * q + k] = J[k];
            snap[3 * q + k] = S[k];
        }
    }
}

/* Condition scale of the evaluation sums: for each listed i, sum over j != i of
 * the norms |a_ij|, |j_ij|, |s_ij| of the pair terms defined above (out: [n_act][3]).
 * Any summation of the terms in working precision u has an error bounded by a
 * small multiple of u times these sums. */
void or_eval_absum(int64_t n, const double *mass, const double *xp, const double *vp, const double *ap,
                   double eps, int64_t n_act, const int32_t *idx, double *out)
{
    for (int64_t q = 0; q < n_act; ++q) {
        int64_t i = idx[q];
        double sa = 0.0, sj = 0.0, ss = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r[3], v[3], a[3], A[3], J[3], S[3];
            for (int k = 0; k < 3; ++k) {
                r[k] = xp[3 * j + k] - xp[3 * i + k];
                v[k] = vp[3 * j + k] - vp[3 * i + k];
                a[k] = ap[3 * j + k] - ap[3 * i + k];
            }
            double r2 = dot3(r, r) + eps * eps;
            double alpha = dot3(r, v) / r2;
            double beta = (dot3(v, v) + dot3(r, a)) / r2 + alpha * alpha;
            double r3 = r2 * sqrt(r2);
            for (int k = 0; k < 3; ++k) {
                A[k] = mass[j] * r[k] / r3;
                J[k] = mass[j] * v[k] / r3 - 3.0 * alpha * A[k];
                S[k] = mass[j] * a[k] / r3 - 6.0 * alpha * J[k] - 3.0 * beta * A[k];
            }
            sa += norm3(A);
            sj += norm3(J);
            ss += norm3(S);
        }
        out[3 * q] = sa;
        out[3 * q + 1] = sj;
        out[3 * q + 2] = ss;
    }
}

/* Sect. 3 item 3 (correction step), for one particle over a step of length h. */
void or_correct(double h, const double *x0, const double *v0, const double *a0, const double *j0,
                const double *s0, const double *a1, const double *j1, const double *s1,
                double *x1, double *v1)
{
    for (int k = 0; k < 3; ++k) {
        v1[k] = v0[k] + h / 2.0 * (a1[k] + a0[k]) - h * h / 10.0 * (j1[k] - j0[k])
              + h * h * h / 120.0 * (s1[k] + s0[k]);
        x1[k] = x0[k] + h / 2.0 * (v1[k] + v0[k]) - h * h / 10.0 * (a1[k] - a0[k])
              + h * h * h / 120.0 * (j1[k] + j0[k]);
    }
}

/* Reading R5: the degree-5 polynomial a(tau) on [0, h] matching a, jerk, snap at
 * both ends.  With
 *   A = a1 - a0 - j0 h - s0 h^2/2,  J = (j1 - j0 - s0 h) h,  S = (s1 - s0) h^2
 * its 3rd, 4th and 5th derivatives at tau = h are
 *   crackle = (60A - 36J + 9S)/h^3, pop = (360A - 192J + 36S)/h^4,
 *   a5 = (720A - 360J + 60S)/h^5. */
void or_interp(double h, const double *a0, const double *j0, const double *s0, const double *a1,
               const double *j1, const double *s1, double *c1, double *p1, double *q1)
{
    for (int k = 0; k < 3; ++k) {
        double A = a1[k] - a0[k] - j0[k] * h - s0[k] * h * h / 2.0;
        double J = (j1[k] - j0[k] - s0[k] * h) * h;
        double S = (s1[k] - s0[k]) * h * h;
        c1[k] = (60.0 * A - 36.0 * J + 9.0 * S) / (h * h * h);
        p1[k] = (360.0 * A - 192.0 * J + 36.0 * S) / (h * h * h * h);
        q1[k] = (720.0 * A - 360.0 * J + 60.0 * S) / (h * h * h * h * h);
    }
}

/* 4th-order variant (the paper's criterion with p = 4): the two-point Hermite
 * corrector of the standard 4th-order Hermite scheme (Makino & Aarseth 1992),
 * from a and jerk at both ends of the step:
 *   v1 = v0 + h/2 (a0 + a1) + h^2/12 (j0 - j1),
 *   x1 = x0 + h/2 (v0 + v1) + h^2/12 (a0 - a1). */
void or_correct4(double h, const double *x0, const double *v0, const double *a0, const double *j0,
                 const double *a1, const double *j1, double *x1, double *v1)
{
    for (int k = 0; k < 3; ++k) {
        v1[k] = v0[k] + h / 2.0 * (a0[k] + a1[k]) + h * h / 12.0 * (j0[k] - j1[k]);
        x1[k] = x0[k] + h / 2.0 * (v0[k] + v1[k]) + h * h / 12.0 * (a0[k] - a1[k]);
    }
}

/* The cubic a(tau) on [0, h] matching a and jerk at both ends: its 3rd
 * derivative (crackle, constant) is c = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3 and
 * its 2nd derivative (snap) at tau = 0 is (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2;
 * s1 = snap at tau = h = s0 + c h. */
void or_interp4(double h, const double *a0, const double *j0, const double *a1, const double *j1,
                double *s1, double *c1)
{
    for (int k = 0; k < 3; ++k) {
        double c = (12.0 * (a0[k] - a1[k]) + 6.0 * h * (j0[k] + j1[k])) / (h * h * h);
        double s0 = (-6.0 * (a0[k] - a1[k]) - h * (4.0 * j0[k] + 2.0 * j1[k])) / (h * h);
        s1[k] = s0 + c * h;
        c1[k] = c;
    }
}

/* Sect. 3, generalized Aarseth criterion: dt = eta (A^(1) / A^(p-2))^(1/(p-3)),
 * A^(s) = sqrt(|a^(s-1)| |a^(s+1)| + |a^(s)|^2).  deriv holds a^(0) .. a^(p-1)
 * as p consecutive 3-vectors.  A^(p-2) = 0 gives +inf (no limit). */
double or_criterion(double eta, int p, const double *deriv)
{
    double nrm[8];
    for (int s = 0; s < p && s < 8; ++s)
        nrm[s] = norm3(deriv + 3 * s);
    double A1 = sqrt(nrm[0] * nrm[2] + nrm[1] * nrm[1]);
    double Ap = sqrt(nrm[p - 3] * nrm[p - 1] + nrm[p - 2] * nrm[p - 2]);
    if (Ap == 0.0)
        return INFINITY;
    double ratio = A1 / Ap;
    if (p - 3 == 1)
        return eta * ratio;
    if (p - 3 == 3)
        return eta * cbrt(ratio);
    return eta * pow(ratio, 1.0 / (double)(p - 3));
}

/* Reading R7: power-of-two block step after a step of length dt_old that ends at t_new. */
double or_block_dt(double crit, double dt_old, double t_new, double dt_min, double dt_max)
{
    double dt = dt_old;
    if (crit < dt) {
        while (dt > crit && dt > dt_min)
            dt = dt / 2.0;
    } else if (crit >= 2.0 * dt && 2.0 * dt <= dt_max && fmod(t_new, 2.0 * dt) == 0.0) {
        dt = 2.0 * dt;
    }
    if (dt < dt_min)
        dt = dt_min;
    if (dt > dt_max)
        dt = dt_max;
    return dt;
}

/* Reading R6/R7: first step, the largest power of two <= crit within [dt_min, dt_max]. */
double or_block_dt_init(double crit, double dt_min, double dt_max)
{
    double dt = dt_max;
    while (dt > crit && dt > dt_min)
        dt = dt / 2.0;
    return dt;
}

/* Table 1, section 1: the next block time t_next = min_i (t_i + dt_i) and the
 * ascending list of particles with t_i + dt_i == t_next.  Returns m. */
int64_t or_next_block(int64_t n, const double *t, const double *dt, double *t_next, int32_t *idx)
{
    double tn = INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (t[i] + dt[i] < tn)
            tn = t[i] + dt[i];
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (t[i] + dt[i] == tn)
            idx[m++] = (int32_t)i;
    *t_next = tn;
    return m;
}

/* Sect. 2 softened pair potential (Reading R8) and kinetic energy. */
void or_energy(int64_t n, const double *mass, const double *x, const double *v, double eps,
               double *kinetic, double *potential)
{
    double K = 0.0, W = 0.0;
    for (int64_t i = 0; i < n; ++i)
        K += 0.5 * mass[i] * dot3(v + 3 * i, v + 3 * i);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double r[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            W -= mass[i] * mass[j] / sqrt(dot3(r, r) + eps * eps);
        }
    *kinetic = K;
    *potential = W;
}

/* Total angular momentum L = sum_i m_i r_i x v_i, the quantity whose magnitude
 * Sect. 5.1 checks for conservation (Delta L_k). */
void or_angular_momentum(int64_t n, const double *mass, const double *x, const double *v, double *L)
{
    double Lx = 0.0, Ly = 0.0, Lz = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double *r = x + 3 * i, *u = v + 3 * i;
        Lx += mass[i] * (r[1] * u[2] - r[2] * u[1]);
        Ly += mass[i] * (r[2] * u[0] - r[0] * u[2]);
        Lz += mass[i] * (r[0] * u[1] - r[1] * u[0]);
    }
    L[0] = Lx;
    L[1] = Ly;
    L[2] = Lz;
}

/* ------------------------------------------------------------------------- */
/* The whole integrator: Sect. 3 items 1-3 repeated block by block.           */
/* ------------------------------------------------------------------------- */
typedef struct or_sys {
    int64_t n;
    int order;                                     /* 6 (the paper's scheme) or 4 */
    double eps, eta, eta_init, dt_min, dt_max, t_sys;
    int64_t steps, interactions;
    double *m, *x, *v, *a, *j, *s, *c, *t, *dt;   /* state at each particle's own time */
    double *xp, *vp, *ap;                          /* predicted data */
    double *ra, *rj, *rs;                          /* evaluation results [n][3] */
    int32_t *idx;
} or_sys;

enum { OR_M, OR_X, OR_V, OR_A, OR_J, OR_S, OR_C, OR_T, OR_DT };

static double *or_field(or_sys *sy, int f, int64_t *len)
{
    int64_t n = sy->n;
    switch (f) {
    case OR_M: *len = n; return sy->m;
    case OR_X: *len = 3 * n; return sy->x;
    case OR_V: *len = 3 * n; return sy->v;
    case OR_A: *len = 3 * n; return sy->a;
    case OR_J: *len = 3 * n; return sy->j;
    case OR_S: *len = 3 * n; return sy->s;
    case OR_C: *len = 3 * n; return sy->c;
    case OR_T: *len = n; return sy->t;
    case OR_DT: *len = n; return sy->dt;
    default: *len = 0; return NULL;
    }
}

void or_sys_free(or_sys *sy)
{
    if (!sy)
        return;
    double *bufs[] = {sy->m, sy->x, sy->v, sy->a, sy->j, sy->s, sy->c, sy->t, sy->dt,
                      sy->xp, sy->vp, sy->ap, sy->ra, sy->rj, sy->rs};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k)
        free(bufs[k]);
    free(sy->idx);
    free(sy);
}

/* Allocate a system holding the given state; no evaluation is made. */
or_sys *or_sys_alloc(int64_t n, double eps, double eta, double eta_init, double dt_min, double dt_max)
{
    or_sys *sy = (or_sys *)calloc(1, sizeof(or_sys));
    if (!sy)
        return NULL;
    sy->n = n;
    sy->eps = eps;
    sy->eta = eta;
    sy->eta_init = eta_init;
    sy->dt_min = dt_min;
    sy->dt_max = dt_max;
    sy->order = 6;
    size_t s1 = (size_t)n * sizeof(double), s3 = 3 * s1;
    sy->m = malloc(s1); sy->t = malloc(s1); sy->dt = malloc(s1);
    sy->x = malloc(s3); sy->v = malloc(s3); sy->a = malloc(s3); sy->j = malloc(s3);
    sy->s = malloc(s3); sy->c = malloc(s3);
    sy->xp = malloc(s3); sy->vp = malloc(s3); sy->ap = malloc(s3);
    sy->ra = malloc(s3); sy->rj = malloc(s3); sy->rs = malloc(s3);
    sy->idx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!sy->m || !sy->t || !sy->dt || !sy->x || !sy->v || !sy->a || !sy->j || !sy->s || !sy->c ||
        !sy->xp || !sy->vp || !sy->ap || !sy->ra || !sy->rj || !sy->rs || !sy->idx) {
        or_sys_free(sy);
        return NULL;
    }
    return sy;
}

/* Start-up: all particles active at t = 0 (prediction is the identity), one full
 * evaluation, crackle = 0 and the first step from the p = 4 criterion with
 * eta_init (Reading R6). */
or_sys *or_sys_create_order(int64_t n, const double *mass, const double *pos, const double *vel, double eps,
                            double eta, double eta_init, double dt_min, double dt_max, int order)
{
    or_sys *sy = or_sys_alloc(n, eps, eta, eta_init, dt_min, dt_max);
    if (!sy)
        return NULL;
    sy->order = order;
    memcpy(sy->m, mass, (size_t)n * sizeof(double));
    memcpy(sy->x, pos, 3 * (size_t)n * sizeof(double));
    memcpy(sy->v, vel, 3 * (size_t)n * sizeof(double));
    memset(sy->a, 0, 3 * (size_t)n * sizeof(double));
    memset(sy->j, 0, 3 * (size_t)n * sizeof(double));
    memset(sy->s, 0, 3 * (size_t)n * sizeof(double));
    memset(sy->c, 0, 3 * (size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        sy->t[i] = 0.0;
        sy->idx[i] = (int32_t)i;
    }
    or_eval(n, sy->m, sy->x, sy->v, sy->a, eps, n, sy->idx, sy->ra, sy->rj, sy->rs);
    sy->interactions = n * n;
    for (int64_t i = 0; i < n; ++i) {
        double d[12];
        memcpy(d + 0, sy->ra + 3 * i, 3 * sizeof(double));
        memcpy(d + 3, sy->rj + 3 * i, 3 * sizeof(double));
        memcpy(d + 6, sy->rs + 3 * i, 3 * sizeof(double));
        memset(d + 9, 0, 3 * sizeof(double));
        memcpy(sy->a + 3 * i, d + 0, 3 * sizeof(double));
        memcpy(sy->j + 3 * i, d + 3, 3 * sizeof(double));
        if (order == 6)   /* the 4th-order scheme keeps a and jerk only */
            memcpy(sy->s + 3 * i, d + 6, 3 * sizeof(double));
        sy->dt[i] = or_block_dt_init(or_criterion(eta_init, 4, d), dt_min, dt_max);
    }
    sy->t_sys = 0.0;
    return sy;
}

or_sys *or_sys_create(int64_t n, const double *mass, const double *pos, const double *vel, double eps,
                      double eta, double eta_init, double dt_min, double dt_max)
{
    return or_sys_create_order(n, mass, pos, vel, eps, eta, eta_init, dt_min, dt_max, 6);
}

/* Corrector, interpolation and new step for the m listed particles whose step
 * ends at t_now, from the evaluation results held in ra/rj/rs[0..m). */
static void or_sys_finish(or_sys *sy, int64_t m, double t_now)
{
    for (int64_t q = 0; q < m; ++q) {
        int64_t i = sy->idx[q];
        double h = sy->dt[i];
        double *a1 = sy->ra + 3 * q, *j1 = sy->rj + 3 * q, *s1 = sy->rs + 3 * q;
        double x1[3], v1[3], d[18];
        if (sy->order == 4) {
            /* 4th-order scheme: corrector from a and jerk, snap and crackle at the
             * step's end from the cubic interpolant, the p = 4 criterion; the
             * stored snap and crackle stay zero (the predictor ends at jerk). */
            or_correct4(h, sy->x + 3 * i, sy->v + 3 * i, sy->a + 3 * i, sy->j + 3 * i, a1, j1, x1, v1);
            memcpy(d + 0, a1, 3 * sizeof(double));
            memcpy(d + 3, j1, 3 * sizeof(double));
            or_interp4(h, sy->a + 3 * i, sy->j + 3 * i, a1, j1, d + 6, d + 9);
            double crit4 = or_criterion(sy->eta, 4, d);
            memcpy(sy->x + 3 * i, x1, 3 * sizeof(double));
            memcpy(sy->v + 3 * i, v1, 3 * sizeof(double));
            memcpy(sy->a + 3 * i, a1, 3 * sizeof(double));
            memcpy(sy->j + 3 * i, j1, 3 * sizeof(double));
            sy->t[i] = t_now;
            sy->dt[i] = or_block_dt(crit4, h, t_now, sy->dt_min, sy->dt_max);
            continue;
        }
        or_correct(h, sy->x + 3 * i, sy->v + 3 * i, sy->a + 3 * i, sy->j + 3 * i, sy->s + 3 * i,
                   a1, j1, s1, x1, v1);
        or_interp(h, sy->a + 3 * i, sy->j + 3 * i, sy->s + 3 * i, a1, j1, s1, d + 9, d + 12, d + 15);
        memcpy(d + 0, a1, 3 * sizeof(double));
        memcpy(d + 3, j1, 3 * sizeof(double));
        memcpy(d + 6, s1, 3 * sizeof(double));
        double crit = or_criterion(sy->eta, 6, d);
        memcpy(sy->x + 3 * i, x1, 3 * sizeof(double));
        memcpy(sy->v + 3 * i, v1, 3 * sizeof(double));
        memcpy(sy->a + 3 * i, a1, 3 * sizeof(double));
        memcpy(sy->j + 3 * i, j1, 3 * sizeof(double));
        memcpy(sy->s + 3 * i, s1, 3 * sizeof(double));
        memcpy(sy->c + 3 * i, d + 9, 3 * sizeof(double));
        sy->t[i] = t_now;
        sy->dt[i] = or_block_dt(crit, h, t_now, sy->dt_min, sy->dt_max);
    }
}

/* One block time step (Table 1 sections 1, 2, 3, 8): select, predict, evaluate,
 * correct.  Returns m; *t_out receives the block time. */
int64_t or_sys_step(or_sys *sy, double *t_out)
{
    double tn;
    int64_t m = or_next_block(sy->n, sy->t, sy->dt, &tn, sy->idx);
    or_predict(sy->n, sy->x, sy->v, sy->a, sy->j, sy->s, sy->c, sy->t, tn, sy->xp, sy->vp, sy->ap);
    or_eval(sy->n, sy->m, sy->xp, sy->vp, sy->ap, sy->eps, m, sy->idx, sy->ra, sy->rj, sy->rs);
    or_sys_finish(sy, m, tn);
    sy->t_sys = tn;
    sy->steps += 1;
    sy->interactions += m * sy->n;
    if (t_out)
        *t_out = tn;
    return m;
}

/* Block steps until every particle has reached t_end (t_end must be a block
 * boundary such as a multiple of dt_max).  Returns the number of steps. */
int64_t or_sys_advance(or_sys *sy, double t_end)
{
    int64_t k = 0;
    for (;;) {
        double tn;
        int32_t *scratch = sy->idx;
        or_next_block(sy->n, sy->t, sy->dt, &tn, scratch);
        if (tn > t_end)
            break;
        or_sys_step(sy, NULL);
        ++k;
    }
    return k;
}

/* Energy of the system predicted to time t (identity for particles already at t). */
void or_sys_energy(or_sys *sy, double t, double *kinetic, double *potential)
{
    or_predict(sy->n, sy->x, sy->v, sy->a, sy->j, sy->s, sy->c, sy->t, t, sy->xp, sy->vp, sy->ap);
    or_energy(sy->n, sy->m, sy->xp, sy->vp, sy->eps, kinetic, potential);
}

/* Angular momentum of the system predicted to time t. */
void or_sys_angular_momentum(or_sys *sy, double t, double *L)
{
    or_predict(sy->n, sy->x, sy->v, sy->a, sy->j, sy->s, sy->c, sy->t, t, sy->xp, sy->vp, sy->ap);
    or_angular_momentum(sy->n, sy->m, sy->xp, sy->vp, L);
}

/* Predict every particle to t and evaluate the listed particles (state injection checks). */
void or_sys_predict_eval(or_sys *sy, double t, int64_t m, const int32_t *idx, double *acc, double *jerk,
                         double *snap)
{
    or_predict(sy->n, sy->x, sy->v, sy->a, sy->j, sy->s, sy->c, sy->t, t, sy->xp, sy->vp, sy->ap);
    or_eval(sy->n, sy->m, sy->xp, sy->vp, sy->ap, sy->eps, m, idx, acc, jerk, snap);
}

/* Predict every particle to t and return the condition scales of the listed particles. */
void or_sys_predict_absum(or_sys *sy, double t, int64_t m, const int32_t *idx, double *out)
{
    or_predict(sy->n, sy->x, sy->v, sy->a, sy->j, sy->s, sy->c, sy->t, t, sy->xp, sy->vp, sy->ap);
    or_eval_absum(sy->n, sy->m, sy->xp, sy->vp, sy->ap, sy->eps, m, idx, out);
}

int or_sys_get(or_sys *sy, int field, double *out)
{
    int64_t len;
    double *p = or_field(sy, field, &len);
    if (!p)
        return -1;
    memcpy(out, p, (size_t)len * sizeof(double));
    return 0;
}

int or_sys_set(or_sys *sy, int field, const double *in)
{
    int64_t len;
    double *p = or_field(sy, field, &len);
    if (!p)
        return -1;
    memcpy(p, in, (size_t)len * sizeof(double));
    return 0;
}

void or_sys_set_order(or_sys *sy, int order) { sy->order = order; }
double or_sys_time(const or_sys *sy) { return sy->t_sys; }
void or_sys_set_time(or_sys *sy, double t) { sy->t_sys = t; }
int64_t or_sys_steps(const or_sys *sy) { return sy->steps; }
int64_t or_sys_interactions(const or_sys *sy) { return sy->interactions; }

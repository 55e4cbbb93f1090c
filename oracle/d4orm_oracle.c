/*
 * d4orm_oracle.c -- FP64 CPU oracle of the D4orm denoising hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see d4orm_oracle.h).  Plain loops, no blocking,
 * no fusion, no reordering beyond what the paper's definitions state.
 *
 * Layouts (shared with the tests, not with the CUDA library):
 *   controls / deformations  u[t][k][d]   t<T, k<n, d<d_u
 *   states                   x[t][k][c]   t<=T (x[0] = S), c<d_x
 */
#include "d4orm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int orc_dims(int dyn, int *d_x, int *d_u, int *d_p)
{
    switch (dyn) {
    case ORC_HOLO2D:     *d_x = 4; *d_u = 2; *d_p = 2; return 0;
    case ORC_HOLO3D:     *d_x = 6; *d_u = 3; *d_p = 3; return 0;
    case ORC_UNICYCLE:   *d_x = 3; *d_u = 2; *d_p = 2; return 0;
    case ORC_DIFFDRIVE4: *d_x = 4; *d_u = 2; *d_p = 2; return 0;
    default: return -1;
    }
}

/* ------------------------------------------------------------------------
 * Noise.  Philox4x32-10 as defined by Salmon et al. (SC'11, Sec. 5):
 * ten rounds of  (X0,X1,X2,X3) -> (hi(M1*X2) ^ X1 ^ k0, lo(M1*X2),
 *                                  hi(M0*X0) ^ X3 ^ k1, lo(M0*X0))
 * with the round key bumped by the Weyl constants between rounds.
 * Pinned against an independent Philox4x32-10 (cuRAND's host generator)
 * in tests/test_oracle_philox.py.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Box-Muller (1958): u1 in (0,1], u2 in [0,1) built from the top 24 bits of
 * each word (exact in binary32 and binary64); z0 = r cos(2 pi u2),
 * z1 = r sin(2 pi u2) with r = sqrt(-2 ln u1).  Pinned by moment and
 * Kolmogorov-Smirnov tests against the standard normal. */
void orc_box_muller(uint32_t a, uint32_t b, double *z0, double *z1)
{
    const double two_m24 = 1.0 / 16777216.0;
    double u1 = ((double)(a >> 8) + 1.0) * two_m24;
    double u2 = (double)(b >> 8) * two_m24;
    double r = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    *z0 = r * cos(ang);
    *z1 = r * sin(ang);
}

/* Counter layout of the sample noise (a design choice of this library; both
 * implementations write it from this statement):
 *   element e = t*d_u + d of robot k's stream, quad q = e / 4, lane e % 4
 *   counter = (q, j, (k & 0xff) | (i << 8), it | (tag << 12))
 *   key     = (seed & 0xffffffff, seed >> 32)
 * The four words give two Box-Muller pairs (w0,w1) -> z0,z1 and
 * (w2,w3) -> z2,z3; the element takes z[e % 4]. */
double orc_noise(const orc_params *pp, int it, int i, int j, int k, int e)
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = (uint32_t)(e / 4);
    ctr[1] = (uint32_t)j;
    ctr[2] = ((uint32_t)k & 0xffu) | ((uint32_t)i << 8);
    ctr[3] = (uint32_t)it | (pp->tag << 12);
    key[0] = (uint32_t)(pp->seed & 0xffffffffu);
    key[1] = (uint32_t)(pp->seed >> 32);
    orc_philox4x32_10(ctr, key, w);
    double z[4];
    orc_box_muller(w[0], w[1], &z[0], &z[1]);
    orc_box_muller(w[2], w[3], &z[2], &z[3]);
    return z[e % 4];
}

/* Noise schedule, Sec. IV-B: alpha_i = 1 - beta_i with beta linear from
 * beta0 (i = 1) to beta1 (i = K), alpha_bar_i = prod_{j<=i} alpha_j (the
 * definition under Eq. (10)), alpha_bar_0 = 1. */
void orc_schedule(int K, double beta0, double beta1, double *alpha, double *alpha_bar)
{
    alpha_bar[0] = 1.0;
    alpha[0] = 1.0;
    for (int i = 1; i <= K; ++i) {
        double beta = (K == 1) ? beta0 : beta0 + (beta1 - beta0) * (double)(i - 1) / (double)(K - 1);
        alpha[i] = 1.0 - beta;
        alpha_bar[i] = alpha_bar[i - 1] * alpha[i];
    }
}

/* ------------------------------------------------------------------------
 * Dynamics, Sec. V: x_dot = f_dyn(x, u).
 * ---------------------------------------------------------------------- */
void orc_dynamics(int dyn, const double *x, const double *u, double *xdot)
{
    switch (dyn) {
    case ORC_HOLO2D:   /* double integrator [v_x, v_y, a_x, a_y] */
        xdot[0] = x[2]; xdot[1] = x[3]; xdot[2] = u[0]; xdot[3] = u[1];
        break;
    case ORC_HOLO3D:   /* 3D version of the double integrator */
        xdot[0] = x[3]; xdot[1] = x[4]; xdot[2] = x[5];
        xdot[3] = u[0]; xdot[4] = u[1]; xdot[5] = u[2];
        break;
    case ORC_UNICYCLE: /* [v cos th, v sin th, omega], u = [v, omega] */
        xdot[0] = u[0] * cos(x[2]); xdot[1] = u[0] * sin(x[2]); xdot[2] = u[1];
        break;
    case ORC_DIFFDRIVE4: /* [v cos th, v sin th, omega, a], u = [omega, a] */
        xdot[0] = x[3] * cos(x[2]); xdot[1] = x[3] * sin(x[2]);
        xdot[2] = u[0]; xdot[3] = u[1];
        break;
    }
}

/* One integration step of Eq. (1) (feasibility): classical RK4 with the
 * control held over the step, or forward Euler where a workload names it.
 * The holonomic speed bound is applied per component after the step;
 * the differential-drive speed state is bounded the same way. */
void orc_integrate(const orc_problem *p, const double *x, const double *u, double *xn)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    double k1[6], k2[6], k3[6], k4[6], tmp[6];
    orc_dynamics(p->dyn, x, u, k1);
    if (p->integ == ORC_EULER) {
        for (int c = 0; c < d_x; ++c) xn[c] = x[c] + p->dt * k1[c];
    } else {
        for (int c = 0; c < d_x; ++c) tmp[c] = x[c] + 0.5 * p->dt * k1[c];
        orc_dynamics(p->dyn, tmp, u, k2);
        for (int c = 0; c < d_x; ++c) tmp[c] = x[c] + 0.5 * p->dt * k2[c];
        orc_dynamics(p->dyn, tmp, u, k3);
        for (int c = 0; c < d_x; ++c) tmp[c] = x[c] + p->dt * k3[c];
        orc_dynamics(p->dyn, tmp, u, k4);
        for (int c = 0; c < d_x; ++c)
            xn[c] = x[c] + p->dt / 6.0 * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
    }
    if (p->v_max > 0.0) {
        if (p->dyn == ORC_HOLO2D || p->dyn == ORC_HOLO3D) {
            for (int c = d_p; c < 2 * d_p; ++c) {
                if (xn[c] > p->v_max) xn[c] = p->v_max;
                if (xn[c] < -p->v_max) xn[c] = -p->v_max;
            }
        } else if (p->dyn == ORC_DIFFDRIVE4) {
            if (xn[3] > p->v_max) xn[3] = p->v_max;
            if (xn[3] < -p->v_max) xn[3] = -p->v_max;
        }
    }
}

/* Rollout (Sec. IV-C): x[0] = S, x[t+1] = RK4(x[t], u[t]); controls are
 * first held to the control box U.  states: [T+1][n][d_x]. */
void orc_rollout(const orc_problem *p, const double *u, double *states)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    const int n = p->n;
    memcpy(states, p->start, sizeof(double) * (size_t)n * d_x);
    for (int t = 0; t < p->T; ++t) {
        for (int k = 0; k < n; ++k) {
            double uc[3];
            for (int d = 0; d < d_u; ++d) {
                double v = u[((size_t)t * n + k) * d_u + d];
                if (v < p->u_lo[d]) v = p->u_lo[d];
                if (v > p->u_hi[d]) v = p->u_hi[d];
                uc[d] = v;
            }
            orc_integrate(p, &states[((size_t)t * n + k) * d_x], uc,
                          &states[((size_t)(t + 1) * n + k) * d_x]);
        }
    }
}

static double pos_dist(const double *a, const double *b, int d_p)
{
    double s = 0.0;
    for (int c = 0; c < d_p; ++c) s += (a[c] - b[c]) * (a[c] - b[c]);
    return sqrt(s);
}

/* Team reward, Sec. IV-A, Eq. (3):
 *   r = 1/(nT) sum_{t=1..T} sum_k ( r_goal(k,t) + w * r_safe(k,t) )
 * Eq. (4): r_goal = 1 - |p_k[t] - g_k| / |p_k[0] - g_k|  (denominator at
 *          least R_a, so that a goal placed on its start stays finite);
 * Eq. (5): r_safe = -1 if some other robot l has |p_k[t]-p_l[t]| <= 2R_a+eps,
 *          else 0 (an indicator, not a per-pair count).
 * Appendix (obstacles): each state of robot k that lies within r_o + R_a +
 *          eps of an obstacle's centre (any obstacle; the same margin eps
 *          as between robots) adds a second binary penalty -w.
 * threshold_gap (optional) receives min over t>=1 and pairs of
 * | |p_k - p_l| - (2R_a + eps) | and over robots and obstacles of
 * | |p_k - c_o| - (r_o + R_a + eps) |: how far the sample is from a flip. */
double orc_reward(const orc_problem *p, double w_safe, const double *states,
                  double *threshold_gap)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    const int n = p->n, T = p->T;
    const double thr = 2.0 * p->radius + p->eps_margin;
    double gap = 1e300;
    double total = 0.0;
    for (int t = 1; t <= T; ++t) {
        for (int k = 0; k < n; ++k) {
            const double *pk = &states[((size_t)t * n + k) * d_x];
            double d0 = pos_dist(p->start + (size_t)k * d_x, p->goal + (size_t)k * d_x, d_p);
            if (d0 < p->radius) d0 = p->radius;
            double r_goal = 1.0 - pos_dist(pk, p->goal + (size_t)k * d_x, d_p) / d0;
            double r_safe = 0.0;
            for (int l = 0; l < n; ++l) {
                if (l == k) continue;
                double dkl = pos_dist(pk, &states[((size_t)t * n + l) * d_x], d_p);
                if (dkl <= thr) r_safe = -1.0;
                double g = fabs(dkl - thr);
                if (g < gap) gap = g;
            }
            double r_obs = 0.0;
            for (int o = 0; o < p->n_obs; ++o) {
                const double *ob = p->obstacles + (size_t)o * 4;
                const double thr_o = ob[3] + p->radius + p->eps_margin;
                double dko = pos_dist(pk, ob, d_p);
                if (dko <= thr_o) r_obs = -1.0;
                double g = fabs(dko - thr_o);
                if (g < gap) gap = g;
            }
            total += r_goal + w_safe * r_safe + w_safe * r_obs;
        }
    }
    if (threshold_gap) *threshold_gap = gap;
    return total / ((double)n * (double)T);
}

/* Fragility of the Eq. (5) indicator, for comparing a binary32 evaluation
 * against this one: the number of robot-timestep indicators (t >= 1, k; the
 * robot-pair indicator and the obstacle indicator counted separately) for
 * which some distance lies within delta of its threshold (2R_a + eps, or
 * r_o + R_a + eps).  Only those indicators can differ between two
 * evaluations whose distances agree to within delta; each such flip moves
 * Eq. (3) by w / (nT). */
int orc_fragile(const orc_problem *p, const double *states, double delta)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    const int n = p->n, T = p->T;
    const double thr = 2.0 * p->radius + p->eps_margin;
    int count = 0;
    for (int t = 1; t <= T; ++t)
        for (int k = 0; k < n; ++k) {
            int fragile = 0;
            for (int l = 0; l < n; ++l) {
                if (l == k) continue;
                double dkl = pos_dist(&states[((size_t)t * n + k) * d_x], &states[((size_t)t * n + l) * d_x], d_p);
                if (fabs(dkl - thr) < delta) fragile = 1;
            }
            count += fragile;
            int fragile_o = 0;
            for (int o = 0; o < p->n_obs; ++o) {
                const double *ob = p->obstacles + (size_t)o * 4;
                double dko = pos_dist(&states[((size_t)t * n + k) * d_x], ob, d_p);
                if (fabs(dko - (ob[3] + p->radius + p->eps_margin)) < delta) fragile_o = 1;
            }
            count += fragile_o;
        }
    return count;
}

/* Eq. (1) conditions and the Eq. (2) objective on a rolled-out plan.
 *   safety:   |p_k[t] - p_l[t]| > 2 R_a for all t in 0..T, k != l, and
 *             |p_k[t] - c_o| > r_o + R_a for every obstacle o (Appendix)
 *   terminal: |p_k[T] - g_k| <= goal_tol for all k (positions only)
 *   objective: 1/(nT) sum_k sum_{t=1..T} Ind[|p_k[t] - g_k| <= goal_tol] */
void orc_verdict_of(const orc_problem *p, double w_safe, const double *states,
                    orc_verdict *out)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    const int n = p->n, T = p->T;
    double min_d = 1e30;
    for (int t = 0; t <= T; ++t)
        for (int k = 0; k < n; ++k)
            for (int l = k + 1; l < n; ++l) {
                double d = pos_dist(&states[((size_t)t * n + k) * d_x],
                                    &states[((size_t)t * n + l) * d_x], d_p);
                if (d < min_d) min_d = d;
            }
    int reached = 1;
    double at_goal = 0.0;
    for (int k = 0; k < n; ++k) {
        for (int t = 1; t <= T; ++t) {
            double dg = pos_dist(&states[((size_t)t * n + k) * d_x], p->goal + (size_t)k * d_x, d_p);
            if (dg <= p->goal_tol) at_goal += 1.0;
            if (t == T && !(dg <= p->goal_tol)) reached = 0;
        }
    }
    int clear = 1;
    for (int t = 0; t <= T; ++t)
        for (int k = 0; k < n; ++k)
            for (int o = 0; o < p->n_obs; ++o) {
                const double *ob = p->obstacles + (size_t)o * 4;
                if (!(pos_dist(&states[((size_t)t * n + k) * d_x], ob, d_p) > ob[3] + p->radius)) clear = 0;
            }
    out->collision_free = (min_d > 2.0 * p->radius && clear) ? 1 : 0;
    out->goal_reached = reached;
    out->reward = orc_reward(p, w_safe, states, NULL);
    out->objective = at_goal / ((double)n * (double)T);
    out->min_pair_dist = min_d;
}

/* Sample weights.  Sec. IV-C: rewards are normalised within the batch
 * (z-score, population standard deviation; a degenerate batch with
 * s <= 1e-12 max(1,|mu|) gets z = 0).  Eq. (6): p0 ~ exp(z / lambda),
 * normalised over the batch as in Eq. (12), computed as a two-pass
 * log-sum-exp (subtract the maximum logit). */
void orc_weights(int N, const double *r, double lambda, double *w)
{
    double mu = 0.0;
    for (int j = 0; j < N; ++j) mu += r[j];
    mu /= (double)N;
    double var = 0.0;
    for (int j = 0; j < N; ++j) var += (r[j] - mu) * (r[j] - mu);
    var /= (double)N;
    double s = sqrt(var);
    double scale = fabs(mu) > 1.0 ? fabs(mu) : 1.0;
    int degenerate = !(s > 1e-12 * scale);
    double m = -1e300;
    for (int j = 0; j < N; ++j) {
        double z = degenerate ? 0.0 : (r[j] - mu) / s;
        w[j] = z / lambda;
        if (w[j] > m) m = w[j];
    }
    double Z = 0.0;
    for (int j = 0; j < N; ++j) { w[j] = exp(w[j] - m); Z += w[j]; }
    for (int j = 0; j < N; ++j) w[j] /= Z;
}

/* Scales of step i: the sample mean factor, the sample standard deviation
 * and the factor on the weighted mean.
 *   ORC_DENOISE (Eq. (12)-(13)): 1/sqrt(abar_i), sqrt(1/abar_i - 1),
 *                                sqrt(abar_{i-1}).
 *   ORC_MPPI: the softmax update the paper contrasts with in Sec. IV
 *             (Williams et al. 2018), with no noise schedule: samples
 *             dU + sigma eps around the current deformation, and the new
 *             deformation is their weighted mean: 1, sigma, 1. */
static void step_scales(const orc_params *pp, const double *abar, int i, double *mean_scale, double *sd,
                        double *g)
{
    if (pp->update_rule == ORC_MPPI) {
        *mean_scale = 1.0;
        *sd = pp->mppi_sigma;
        *g = 1.0;
    } else {
        *mean_scale = 1.0 / sqrt(abar[i]);
        *sd = sqrt(1.0 / abar[i] - 1.0);
        *g = sqrt(abar[i - 1]);
    }
}

/* Sample j of step i (Algorithm 1, sampling line; Eq. (12)):
 *   dU_j ~ N(dU_i / sqrt(abar_i), (1/abar_i - 1) I),
 * drawn as dU_i / sqrt(abar_i) + sqrt(1/abar_i - 1) * eps_j
 * (MPPI: dU_i + sigma * eps_j). */
static double sample_entry(const orc_params *pp, int it, int i, int j, int k, int e, double du,
                           double mean_scale, double sd)
{
    return du * mean_scale + sd * orc_noise(pp, it, i, j, k, e);
}

static void make_sample(const orc_problem *p, const orc_params *pp, int it, int i, int j,
                        const double *abar, const double *du_in, double *sample)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    double mean_scale, sd, g;
    step_scales(pp, abar, i, &mean_scale, &sd, &g);
    for (int t = 0; t < p->T; ++t)
        for (int k = 0; k < p->n; ++k)
            for (int d = 0; d < d_u; ++d) {
                size_t idx = ((size_t)t * p->n + k) * d_u + d;
                sample[idx] = sample_entry(pp, it, i, j, k, t * d_u + d, du_in[idx], mean_scale, sd);
            }
}

/* Fitness of selected samples: deformation sample j is added to the fixed
 * base trajectory (Sec. IV-D), rolled out from S and scored by Eq. (3). */
void orc_sample_fitness(const orc_problem *p, const orc_params *pp, int it, int i,
                        const double *u_base, const double *du_in,
                        int count, const int *js, double *fitness, double *gap,
                        double delta, int *fragile)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    const size_t nu = (size_t)p->T * p->n * d_u;
    double *alpha = malloc(sizeof(double) * (pp->K + 1));
    double *abar = malloc(sizeof(double) * (pp->K + 1));
    orc_schedule(pp->K, pp->beta0, pp->beta1, alpha, abar);
    /* samples are independent: each thread rolls out its own ones into
     * private buffers and writes only their own output entries */
#pragma omp parallel
    {
        double *sample = malloc(sizeof(double) * nu);
        double *ctrl = malloc(sizeof(double) * nu);
        double *states = malloc(sizeof(double) * (size_t)(p->T + 1) * p->n * d_x);
#pragma omp for schedule(dynamic, 4)
        for (int c = 0; c < count; ++c) {
            int j = js[c];
            make_sample(p, pp, it, i, j, abar, du_in, sample);
            for (size_t e = 0; e < nu; ++e) ctrl[e] = u_base[e] + sample[e];
            orc_rollout(p, ctrl, states);
            fitness[c] = orc_reward(p, pp->w_safe, states, gap ? &gap[c] : NULL);
            if (fragile) fragile[c] = orc_fragile(p, states, delta);
        }
        free(sample); free(ctrl); free(states);
    }
    free(alpha); free(abar);
}

/* Weighted mean and one-step denoise, Algorithm 1 / Eq. (12)-(13):
 *   dU_bar = sum_j w_j dU_j   (weights already normalised),
 *   dU_{i-1} = sqrt(abar_{i-1}) * dU_bar   (MPPI: dU_bar itself).
 * The mean is taken over the sampled (unclipped) deformations. */
void orc_weighted_update(const orc_problem *p, const orc_params *pp, int it, int i,
                         const double *du_in, const double *w, double *du_out)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    double *alpha = malloc(sizeof(double) * (pp->K + 1));
    double *abar = malloc(sizeof(double) * (pp->K + 1));
    orc_schedule(pp->K, pp->beta0, pp->beta1, alpha, abar);
    double mean_scale, sd, g;
    step_scales(pp, abar, i, &mean_scale, &sd, &g);
    /* every entry is summed over samples j = 0..N-1 in order; robots are
     * independent, so threads split them (same sums for any thread count).
     * Entry (t, k, d) of sample j is the same sample_entry as in make_sample. */
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < p->n; ++k) {
        for (int t = 0; t < p->T; ++t)
            for (int d = 0; d < d_u; ++d) {
                size_t idx = ((size_t)t * p->n + k) * d_u + d;
                double acc = 0.0;
                for (int j = 0; j < pp->N; ++j)
                    acc += w[j] * sample_entry(pp, it, i, j, k, t * d_u + d, du_in[idx], mean_scale, sd);
                du_out[idx] = g * acc;
            }
    }
    free(alpha); free(abar);
}

/* Thread count of the parallel sample loops (OpenMP builds; 1 otherwise). */
#ifdef _OPENMP
#include <omp.h>
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_max_threads(void) { return omp_get_max_threads(); }
#else
void orc_set_threads(int n) { (void)n; }
int orc_max_threads(void) { return 1; }
#endif

/* One denoising step (Algorithm 1 body for step i, applied to the
 * deformation of Algorithm 2).  fitness (optional, [N]) receives the
 * oracle's own per-sample reward; when fitness_in is given those rewards
 * are used for the weights instead (stage-isolated comparison). */
void orc_denoise_step(const orc_problem *p, const orc_params *pp, int it, int i,
                      const double *u_base, const double *du_in, double *du_out,
                      double *fitness, const double *fitness_in, double *gap)
{
    const int N = pp->N;
    double *r = malloc(sizeof(double) * N);
    double *w = malloc(sizeof(double) * N);
    if (fitness_in) {
        memcpy(r, fitness_in, sizeof(double) * N);
    } else {
        int *js = malloc(sizeof(int) * N);
        for (int j = 0; j < N; ++j) js[j] = j;
        orc_sample_fitness(p, pp, it, i, u_base, du_in, N, js, r, gap, 0.0, NULL);
        free(js);
    }
    if (fitness) memcpy(fitness, r, sizeof(double) * N);
    orc_weights(N, r, pp->lambda, w);
    orc_weighted_update(p, pp, it, i, du_in, w, du_out);
    free(r); free(w);
}

/* Iteration end of Algorithm 2: tau.u <- tau.u + dU, held to the control
 * box (the applied controls of the new rollout). */
void orc_apply(const orc_problem *p, const double *u_base, const double *du0, double *u_new)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    for (int t = 0; t < p->T; ++t)
        for (int k = 0; k < p->n; ++k)
            for (int d = 0; d < d_u; ++d) {
                size_t idx = ((size_t)t * p->n + k) * d_u + d;
                double v = u_base[idx] + du0[idx];
                if (v < p->u_lo[d]) v = p->u_lo[d];
                if (v > p->u_hi[d]) v = p->u_hi[d];
                u_new[idx] = v;
            }
}

/* Algorithm 2 with an iteration budget.  tau.u starts at zero; each
 * iteration restarts the schedule with dU_K = 0 (Sec. IV-D) -- or, for the
 * first iteration only, with dU_{start_step} = du_init when given -- runs
 * steps i = K..1 (start_step..1), applies dU_0 and rolls out.
 * verdicts[it] receives each iteration's plan verdict.  Returns the index
 * of the first successful iteration, or -1. */
int orc_solve(const orc_problem *p, const orc_params *pp, int max_iters, int stop_on_success,
              int start_step, const double *du_init, double *u_out, orc_verdict *verdicts,
              int *iters_run)
{
    int d_x, d_u, d_p;
    orc_dims(p->dyn, &d_x, &d_u, &d_p);
    const size_t nu = (size_t)p->T * p->n * d_u;
    double *u = calloc(nu, sizeof(double));
    double *du = malloc(sizeof(double) * nu);
    double *du_next = malloc(sizeof(double) * nu);
    double *states = malloc(sizeof(double) * (size_t)(p->T + 1) * p->n * d_x);
    int first = -1, it;
    for (it = 0; it < max_iters; ++it) {
        int i0 = pp->K;
        if (it == 0 && du_init) {
            i0 = start_step;
            memcpy(du, du_init, sizeof(double) * nu);
        } else {
            memset(du, 0, sizeof(double) * nu);
        }
        for (int i = i0; i >= 1; --i) {
            orc_denoise_step(p, pp, it, i, u, du, du_next, NULL, NULL, NULL);
            double *tmp = du; du = du_next; du_next = tmp;
        }
        orc_apply(p, u, du, u);
        orc_rollout(p, u, states);
        orc_verdict_of(p, pp->w_safe, states, &verdicts[it]);
        if (first < 0 && verdicts[it].collision_free && verdicts[it].goal_reached) first = it;
        if (stop_on_success && first >= 0) { ++it; break; }
    }
    if (iters_run) *iters_run = it;
    memcpy(u_out, u, sizeof(double) * nu);
    free(u); free(du); free(du_next); free(states);
    return first;
}

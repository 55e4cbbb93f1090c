/*
 * d4orm_oracle.h -- plain, slow, FP64 CPU oracle of the D4orm denoising
 * hot path (Zhang et al., "D4orm: Multi-Robot Trajectories with
 * Dynamics-aware Diffusion Denoised Deformations", IROS 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  The CUDA
 * library never includes, links or calls it, and it shares no header, table
 * or helper with the CUDA library.
 *
 * Every function follows the paper's definitions in the paper's order:
 *   Sec. III, Eq. (1)  problem conditions (feasibility, init, terminal, safety)
 *   Sec. III, Eq. (2)  quality objective (time at goal)
 *   Sec. IV-A, Eq. (3)-(5)  team reward r(tau), r_goal, r_safe
 *   Sec. IV-B, Eq. (6)  target distribution p0 ~ exp(r / lambda)
 *   Sec. IV-B, Eq. (12)-(13) Monte Carlo samples, weighted mean, one-step denoise
 *   Algorithm 1  denoising optimisation process (controls sampled, rolled out)
 *   Sec. IV-C  batch reward normalisation
 *   Sec. IV-D, Algorithm 2  iterative optimisation of deformations
 *   Sec. V  dynamics models (differential drive, 2D/3D holonomic)
 *
 * Parity pins: see the per-function comments.  Functions whose result is
 * fixed only by a reading of a silent point of the paper (noise schedule
 * constants, temperature, safety weight and margin) are pinned by
 * invariants and special cases, not by printed values: the paper prints no
 * worked example.
 */
#ifndef D4ORM_ORACLE_H
#define D4ORM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Dynamics models of Sec. V (+ the unicycle of the 8-robot workload). */
enum {
    ORC_HOLO2D = 0,     /* x=[px,py,vx,vy], u=[ax,ay]                 */
    ORC_HOLO3D = 1,     /* x=[px,py,pz,vx,vy,vz], u=[ax,ay,az]        */
    ORC_UNICYCLE = 2,   /* x=[px,py,theta], u=[v,omega]               */
    ORC_DIFFDRIVE4 = 3  /* x=[px,py,theta,v], u=[omega,a]  (Sec. V)    */
};
enum { ORC_EULER = 0, ORC_RK4 = 1 };

typedef struct {
    int n;              /* robots                                     */
    int T;              /* controls per robot (the paper's H)         */
    int dyn;            /* ORC_*                                      */
    int integ;          /* ORC_EULER / ORC_RK4                         */
    double dt;          /* integration step                           */
    double radius;      /* R_a                                        */
    double eps_margin;  /* epsilon of Eq. (5)                          */
    double goal_tol;    /* terminal-condition tolerance (position)    */
    double v_max;       /* holonomic per-axis speed bound (<=0: none) */
    double u_lo[3], u_hi[3]; /* per-component control box              */
    const double *start;     /* [n][d_x]  S                            */
    const double *goal;      /* [n][d_x]  T (positions used)           */
    int n_obs;               /* static spherical obstacles (Appendix)   */
    const double *obstacles; /* [n_obs][4]: centre x, y, z (z unused in
                                2D), radius r_o                         */
} orc_problem;

typedef struct {
    int N;              /* Monte Carlo samples (the paper's M)        */
    int K;              /* denoising steps (the paper's N)            */
    double lambda;      /* temperature of Eq. (6)                      */
    double w_safe;      /* weight w_t of Eq. (3)                       */
    double beta0, beta1;/* linear noise schedule end points           */
    uint64_t seed;      /* Philox key                                 */
    uint32_t tag;       /* instance tag (counter word)                */
    int update_rule;    /* ORC_DENOISE (Eq. (12)-(13)) or ORC_MPPI    */
    double mppi_sigma;  /* MPPI exploration standard deviation        */
} orc_params;

enum { ORC_DENOISE = 0, ORC_MPPI = 1 };

typedef struct {
    int collision_free; /* Eq. (1) safety over states 0..T            */
    int goal_reached;   /* Eq. (1) terminal condition, position only  */
    double reward;      /* Eq. (3)                                    */
    double objective;   /* Eq. (2)                                    */
    double min_pair_dist;
} orc_verdict;

int orc_dims(int dyn, int *d_x, int *d_u, int *d_p);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Box-Muller transform of two 32-bit words into two standard normals. */
void orc_box_muller(uint32_t a, uint32_t b, double *z0, double *z1);
/* Standard normal epsilon for (iteration it, step i, sample j, robot k,
 * element e = t*d_u + d of robot k's control stream). */
double orc_noise(const orc_params *pp, int it, int i, int j, int k, int e);

/* Linear beta schedule; alpha[1..K], alpha_bar[0..K] (alpha_bar[0] = 1). */
void orc_schedule(int K, double beta0, double beta1, double *alpha, double *alpha_bar);

void orc_dynamics(int dyn, const double *x, const double *u, double *xdot);
void orc_integrate(const orc_problem *p, const double *x, const double *u, double *xn);
void orc_rollout(const orc_problem *p, const double *u, double *states);
double orc_reward(const orc_problem *p, double w_safe, const double *states,
                  double *threshold_gap);
void orc_verdict_of(const orc_problem *p, double w_safe, const double *states,
                    orc_verdict *out);
void orc_weights(int N, const double *r, double lambda, double *w);

/* One denoising step of Algorithm 1 applied to deformations (Algorithm 2). */
int orc_fragile(const orc_problem *p, const double *states, double delta);
void orc_sample_fitness(const orc_problem *p, const orc_params *pp, int it, int i,
                        const double *u_base, const double *du_in,
                        int count, const int *js, double *fitness, double *gap,
                        double delta, int *fragile);
void orc_denoise_step(const orc_problem *p, const orc_params *pp, int it, int i,
                      const double *u_base, const double *du_in, double *du_out,
                      double *fitness, const double *fitness_in, double *gap);
void orc_weighted_update(const orc_problem *p, const orc_params *pp, int it, int i,
                         const double *du_in, const double *w, double *du_out);
void orc_apply(const orc_problem *p, const double *u_base, const double *du0, double *u_new);
/* Threads of the parallel sample loops (OpenMP builds only). */
void orc_set_threads(int n);
int orc_max_threads(void);

int orc_solve(const orc_problem *p, const orc_params *pp, int max_iters, int stop_on_success,
              int start_step, const double *du_init, double *u_out, orc_verdict *verdicts,
              int *iters_run);

#ifdef __cplusplus
}
#endif
#endif

/*
 * FP64 CPU oracle for the SPaSM hot path (test infrastructure only).
 *
 * This is a plain, slow restatement of what the paper's method computes, used by the
 * tests, by smoke() and by the CPU-baseline leg of the benchmark to check the CUDA
 * path.  It shares no code with the CUDA library.  It must never be called by the
 * product path.
 *
 * Every quantity is double precision.  Arrays are row-major.
 *
 *   Stage 1 particle  x[B][4]  = (x, y, z, yaw) of the block at each stack position.
 *   Stage 2 particle  q[C][7]  joint configurations, C = 2B(W-1)+1, q[0] = q_home.
 */
#ifndef SPASM_ORACLE_H
#define SPASM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    /* robot: 7 modified-DH rows (a, alpha, d, theta_offset), limits, spheres, tool */
    const double *dh;          /* 7 x 4 */
    const double *qlim;        /* 7 x 2 */
    int n_spheres;
    const int32_t *sphere_link;/* n_spheres, 0 = base */
    const double *sphere;      /* n_spheres x 4 (x, y, z, r) in the link frame */
    const double *ee;          /* 4 x 4 flange -> tool point */
    const double *q_home;      /* 7 */
    /* environment */
    int n_cub;
    const double *cub;         /* n_cub x 15: centre 3, R 9 (row-major), half 3 */
    int n_sph;
    const double *sph;         /* n_sph x 4 */
    /* goal / skeleton, in stack order (bottom to top) */
    int B;
    const double *half;        /* B x 3 */
    const double *init;        /* B x 4 */
    const double *box;         /* 6: lo xyz, hi xyz */
    double z_table, grasp_off;
    /* parameters */
    int N, M, P, Q, W, K_lin, K_quad, K_traj, K_al, K_ik;
    double eta_init, alpha, eta_traj, eps, eps_start;
    double w_stable, w_height, w_coll, w_start, w_arm, w_block, w_path, w_jl;
    double mu0, mu_max, ik_damp;
    uint64_t seed;
    int max_steps;
    int n_threads;
    /* goal kind: 0 = tower (the tower stacking costs of the appendix), 1 = packing (the
     * appendix's Tetris problem).  Packing: block i is a polyomino of unit cubes of edge
     * cell_size centred at the offsets cell[cell_start[i] .. cell_start[i+1]) (x, y in the
     * block frame); the walls are the environment cuboids; z_star is the target height. */
    int kind;
    const int32_t *cell_start; /* B + 1 */
    const double *cell;        /* cell_start[B] x 2 */
    double cell_size, z_star;
    /* lift IK: 0 = damped least squares from a perturbed home seed; 1 = analytic IK of the
     * Franka joint layout over OR_IK_Q6 values of the last joint (the seed's and one
     * draw per equal strip of its range), the in-limit solution nearest to that seed,
     * damped least squares where no in-limit analytic solution exists */
    int ik_mode;
} or_problem;

#define OR_IK_Q6 32  /* last-joint values tried per target by the analytic lift */

enum { OR_KIND_TOWER = 0, OR_KIND_PACK = 1, OR_KIND_P2P = 2 };
/* Point-to-point trajectory optimisation (kind 2, the paper's motion-planning use of stage
 * 2): B = 1 and the "block" is a zero-size virtual target at init[0..3]; the trajectory is
 * one transit segment, C = W configurations from q_home to the target's grasp
 * configuration; the residuals are the target alignment (position, roll, pitch) and the
 * arm collisions; there is no placement, no held block and no stage 1. */

/* constraint groups of the stage-2 augmented Lagrangian */
enum { OR_G_START = 0, OR_G_ARM, OR_G_BLOCK, OR_G_COLL, OR_G_STABLE, OR_G_HEIGHT, OR_NG };

void   or_philox4x32_10(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]);
double or_u01(uint32_t u);

void   or_fk(const or_problem *pr, const double q[7], double frames[8][16], double tee[16]);
double or_box_sd(const double c[3], double r, const double *cub, double dsd_dc[3]);
double or_pen_box(const double c[3], double r, const double centre[3], const double R[9],
                  const double half[3], double dpen_dc[3], double dpen_dp[3]);
double or_pen_sph(const double c[3], double r, const double *sph, double dpen_dc[3]);

/* stage 1 (Alg. 1 and the placement cost of the appendix: tower, or packing when kind = 1) */
double or_place_cost(const or_problem *pr, const double *x, int quad, double *grad, double terms[3]);
int    or_place_check(const or_problem *pr, const double *x, double metrics[3]);
void   or_place_sample(const or_problem *pr, int n, uint32_t attempt, double *x);
void   or_argsort(int n, const double *cost, int32_t *idx);
void   or_place_descend(const or_problem *pr, int m, double *x, int k_lin, int k_quad);
int    or_place_solve(const or_problem *pr, double *out, int *n_found, int *attempts, int *steps);

/* stage 2 (trajectory optimisation of Sec. III-B and the appendix) */
int    or_n_configs(const or_problem *pr);
void   or_ik(const or_problem *pr, const double target[16], const double q0[7], double q[7]);
int    or_ik_analytic_supported(const or_problem *pr);
int    or_ik_analytic(const or_problem *pr, const double target[16], double q6, double sol[8][7]);
int    or_ik_select(const or_problem *pr, const double target[16], const double seed[7], const double *q6,
                    int n_q6, double q[7]);
void   or_lift(const or_problem *pr, const double *place, int particle, uint32_t attempt, double *q);
/* or_lift, and where analytic != NULL, 2B flags: 1 where the grasp (2b) / place (2b+1)
 * configuration of block b came from the analytic IK, 0 where damped least squares */
void   or_lift_ex(const or_problem *pr, const double *place, int particle, uint32_t attempt, double *q,
                  int32_t *analytic);
int    or_n_residuals(const or_problem *pr);
double or_traj_cost(const or_problem *pr, const double *q, const double *lam, double mu,
                    double *grad, double c_groups[OR_NG], double *path, double *jl, double *h);
int    or_traj_check(const or_problem *pr, const double *q, double metrics[6]);
double or_traj_rank_cost(const or_problem *pr, const double *q);
void   or_traj_descend(const or_problem *pr, int n, double *q, double *lam, double *mu, int k_steps);
int    or_traj_solve(const or_problem *pr, const double *place, int n_place, double *out_q,
                     double *out_cost, int *n_found, int *attempts);

#ifdef __cplusplus
}
#endif
#endif

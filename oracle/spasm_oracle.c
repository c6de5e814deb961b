/*
 * FP64 CPU oracle for the SPaSM hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, smoke() and the benchmark's CPU-baseline leg may load this file.  The
 * product (the CUDA library) never calls it, and it shares no code, header or table
 * with the CUDA sources.
 *
 * Plain restatement, in double precision, of:
 *   - Alg. 1 (sample, cost, argsort top-M, linear descent with eta = eta_init(1-k/K_lin),
 *     quadratic refinement with fixed alpha, satisfying filter, best P, retry),
 *   - the tower placement cost C_placement = w_stable C_stable + w_height C_height
 *     + w_coll C_coll (Appendix, tower stacking),
 *   - the trajectory cost C_trajopt = C_placement(fk(q_{b,T})) + w_start C_start
 *     + w_arm C_arm + w_block C_block (Appendix), inside an augmented Lagrangian
 *     (Sec. III-B, trajectory optimisation),
 *   - the lift of placements to joint space (Sec. III-B): IK at grasp poses (damped least
 *     squares, or the analytic IK of the Franka joint layout), one intermediate waypoint
 *     per segment, linear interpolation.
 * Robot and objects are sphere sets; collisions are penetration depths (Sec. III).
 * Readings of points where the paper is silent are stated at each function.
 *
 * Gradients are analytic, written with explicit per-point Jacobians
 * (dc/dq_k = z_k x (c - o_k)) and explicit rotation derivatives (dR/dq_k = [z_k]x R),
 * evaluated in two passes (group values first, then the gradient with the
 * augmented-Lagrangian weights).  They are pinned against central differences.
 */
#include "spasm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2,  */
/* 3", SC'11).  Key (k0, k1) = (seed low word, seed high word); counter of four words.    */
/* ------------------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;   /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* top 24 bits -> [0, 1), exact in binary32 and binary64 */
double or_u01(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

static void philox(const or_problem *pr, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    or_philox4x32_10(ctr, pr->seed, out);
}

/* Philox stream tags */
enum { TAG_SAMPLE = 0, TAG_GRASP = 1, TAG_IKSEED = 2, TAG_VIA = 3, TAG_Q6 = 4 };

/* ------------------------------------------------------------------------------------ */
/* small linear algebra                                                                  */
/* ------------------------------------------------------------------------------------ */
static void mat4_mul(const double A[16], const double B[16], double C[16]) {
    double T[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
            T[4 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}

static void mat4_eye(double T[16]) {
    memset(T, 0, 16 * sizeof(double));
    T[0] = T[5] = T[10] = T[15] = 1.0;
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    c[0] = t0; c[1] = t1; c[2] = t2;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double relu(double v) { return v > 0.0 ? v : 0.0; }

/* column c of the rotation part of a 4x4 transform */
static void col3(const double T[16], int c, double v[3]) { v[0] = T[c]; v[1] = T[4 + c]; v[2] = T[8 + c]; }

/* transform a point */
static void xform(const double T[16], const double p[3], double out[3]) {
    for (int i = 0; i < 3; ++i) out[i] = T[4 * i] * p[0] + T[4 * i + 1] * p[1] + T[4 * i + 2] * p[2] + T[4 * i + 3];
}

static void rot_z3(double yaw, double R[9]) {
    double c = cos(yaw), s = sin(yaw);
    R[0] = c; R[1] = -s; R[2] = 0.0;
    R[3] = s; R[4] = c;  R[5] = 0.0;
    R[6] = 0.0; R[7] = 0.0; R[8] = 1.0;
}

static double wrap_angle(double a) { return a - 2.0 * PI * floor((a + PI) / (2.0 * PI)); }

/* ------------------------------------------------------------------------------------ */
/* Forward kinematics of the 7-R arm, modified (Craig) DH rows:                          */
/*   T_k = Rot_x(alpha_k) Trans_x(a_k) Rot_z(theta_k + q_k) Trans_z(d_k),                */
/*   frame_k = frame_{k-1} T_k, frame_0 = identity (base), tool = frame_7 * ee.          */
/* The convention is a reading: the paper only names fk(q) of the 7-DoF arm (appendix). */
/* ------------------------------------------------------------------------------------ */
static void dh_transform(double a, double alpha, double d, double theta, double T[16]) {
    double Rx[16], Tx[16], Rz[16], Tz[16], t1[16], t2[16];
    mat4_eye(Rx); Rx[5] = cos(alpha); Rx[6] = -sin(alpha); Rx[9] = sin(alpha); Rx[10] = cos(alpha);
    mat4_eye(Tx); Tx[3] = a;
    mat4_eye(Rz); Rz[0] = cos(theta); Rz[1] = -sin(theta); Rz[4] = sin(theta); Rz[5] = cos(theta);
    mat4_eye(Tz); Tz[11] = d;
    mat4_mul(Rx, Tx, t1);
    mat4_mul(t1, Rz, t2);
    mat4_mul(t2, Tz, T);
}

void or_fk(const or_problem *pr, const double q[7], double frames[8][16], double tee[16]) {
    mat4_eye(frames[0]);
    for (int k = 1; k <= 7; ++k) {
        const double *row = pr->dh + 4 * (k - 1);
        double Tk[16];
        dh_transform(row[0], row[1], row[2], row[3] + q[k - 1], Tk);
        mat4_mul(frames[k - 1], Tk, frames[k]);
    }
    if (tee) mat4_mul(frames[7], pr->ee, tee);
}

/* d c / d q_j for a point c rigidly attached to link `link`: z_j x (c - o_j), j <= link */
static void point_jacobian(double frames[8][16], int link, const double c[3], double J[3][7]) {
    for (int j = 0; j < 7; ++j) {
        if (j + 1 > link) { J[0][j] = J[1][j] = J[2][j] = 0.0; continue; }
        double z[3], o[3], r[3], v[3];
        col3(frames[j + 1], 2, z);
        col3(frames[j + 1], 3, o);
        for (int i = 0; i < 3; ++i) r[i] = c[i] - o[i];
        cross3(z, r, v);
        J[0][j] = v[0]; J[1][j] = v[1]; J[2][j] = v[2];
    }
}

/* d R / d q_j = [z_j]x R for a rotation attached to the tool (j = 0..6) */
static void rot_derivative(double frames[8][16], const double R[9], int j, double dR[9]) {
    double z[3];
    col3(frames[j + 1], 2, z);
    for (int c = 0; c < 3; ++c) {
        double v[3] = {R[c], R[3 + c], R[6 + c]}, w[3];
        cross3(z, v, w);
        dR[c] = w[0]; dR[3 + c] = w[1]; dR[6 + c] = w[2];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Signed distance sphere -> cuboid (penetration-depth collision, Sec. III).             */
/*   p = R^T (c - centre), q = |p| - h,                                                  */
/*   sd = || max(q, 0) || + min(max_k q_k, 0) - r,   pen = max(0, -sd).                  */
/* Gradient: outside (max q > 0): R (sign(p) * max(q,0) / ||max(q,0)||); inside: the     */
/* axis a of the largest q (lowest index on ties), R (sign(p_a) e_a); sign(0) = +1.      */
/* ------------------------------------------------------------------------------------ */
static double box_sd_local(const double c[3], double r, const double centre[3], const double R[9],
                           const double half[3], double dsd_dp[3], double p_out[3]) {
    double d[3] = {c[0] - centre[0], c[1] - centre[1], c[2] - centre[2]};
    double p[3], q[3], sg[3];
    for (int k = 0; k < 3; ++k) {
        p[k] = R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];   /* R^T d */
        sg[k] = p[k] >= 0.0 ? 1.0 : -1.0;
        q[k] = fabs(p[k]) - half[k];
    }
    int a = 0;
    for (int k = 1; k < 3; ++k) if (q[k] > q[a]) a = k;
    double sd;
    if (q[a] > 0.0) {
        double m[3], n2 = 0.0;
        for (int k = 0; k < 3; ++k) { m[k] = relu(q[k]); n2 += m[k] * m[k]; }
        double n = sqrt(n2);
        sd = n - r;
        for (int k = 0; k < 3; ++k) dsd_dp[k] = sg[k] * m[k] / n;
    } else {
        sd = q[a] - r;
        dsd_dp[0] = dsd_dp[1] = dsd_dp[2] = 0.0;
        dsd_dp[a] = sg[a];
    }
    if (p_out) { p_out[0] = p[0]; p_out[1] = p[1]; p_out[2] = p[2]; }
    return sd;
}

double or_box_sd(const double c[3], double r, const double *cub, double dsd_dc[3]) {
    double g[3];
    double sd = box_sd_local(c, r, cub, cub + 3, cub + 12, g, NULL);
    const double *R = cub + 3;
    for (int i = 0; i < 3; ++i) dsd_dc[i] = R[3 * i] * g[0] + R[3 * i + 1] * g[1] + R[3 * i + 2] * g[2];
    return sd;
}

/* pen = max(0, -sd); dpen_dc in world, dpen_dp in the cuboid frame (both zero if pen = 0) */
double or_pen_box(const double c[3], double r, const double centre[3], const double R[9],
                  const double half[3], double dpen_dc[3], double dpen_dp[3]) {
    double g[3], p[3];
    double sd = box_sd_local(c, r, centre, R, half, g, p);
    double pen = relu(-sd);
    for (int i = 0; i < 3; ++i) {
        double gw = R[3 * i] * g[0] + R[3 * i + 1] * g[1] + R[3 * i + 2] * g[2];
        if (dpen_dc) dpen_dc[i] = pen > 0.0 ? -gw : 0.0;
        if (dpen_dp) dpen_dp[i] = pen > 0.0 ? -g[i] : 0.0;
    }
    return pen;
}

/* sphere -> sphere penetration: pen = max(0, r + r_o - ||c - c_o||) */
double or_pen_sph(const double c[3], double r, const double *sph, double dpen_dc[3]) {
    double d[3] = {c[0] - sph[0], c[1] - sph[1], c[2] - sph[2]};
    double n = sqrt(dot3(d, d));
    double pen = relu(r + sph[3] - n);
    for (int i = 0; i < 3; ++i) dpen_dc[i] = (pen > 0.0 && n > 0.0) ? -d[i] / n : 0.0;
    return pen;
}

/* penetration of sphere (c, r) into the upright cuboid of a block pose (x, y, z, yaw) and
 * its derivatives w.r.t. c and w.r.t. the pose:  p = Rz(yaw)^T (c - P),
 * dpen/dP = -dpen/dc,  dpen/dyaw = dpen/dp . (p_y, -p_x, 0). */
static double pen_block(const double c[3], double r, const double pose[4], const double half[3],
                        double dpen_dc[3], double dpen_dpose[4]) {
    double R[9], g[3], p[3];
    rot_z3(pose[3], R);
    double sd = box_sd_local(c, r, pose, R, half, g, p);
    double pen = relu(-sd);
    if (dpen_dc) {
        for (int i = 0; i < 3; ++i) {
            double gw = R[3 * i] * g[0] + R[3 * i + 1] * g[1] + R[3 * i + 2] * g[2];
            dpen_dc[i] = pen > 0.0 ? -gw : 0.0;
        }
    }
    if (dpen_dpose) {
        if (pen > 0.0) {
            double dp[3] = {-g[0], -g[1], -g[2]};
            for (int i = 0; i < 3; ++i)
                dpen_dpose[i] = -(R[3 * i] * dp[0] + R[3 * i + 1] * dp[1] + R[3 * i + 2] * dp[2]);
            dpen_dpose[3] = dp[0] * p[1] - dp[1] * p[0];
        } else {
            dpen_dpose[0] = dpen_dpose[1] = dpen_dpose[2] = dpen_dpose[3] = 0.0;
        }
    }
    return pen;
}

/* Block i as a set of 8 spheres (objects are sphere sets, Sec. III): centres at
 * (+-hx/2, +-hy/2, +-hz/2) in the block frame, radius min(h)/2.  Bit 0/1/2 of m pick
 * the sign along x/y/z. */
static void block_sphere_local(const double half[3], int m, double l[3], double *r) {
    l[0] = ((m & 1) ? 0.5 : -0.5) * half[0];
    l[1] = ((m & 2) ? 0.5 : -0.5) * half[1];
    l[2] = ((m & 4) ? 0.5 : -0.5) * half[2];
    double h = half[0] < half[1] ? half[0] : half[1];
    h = h < half[2] ? h : half[2];
    *r = 0.5 * h;
}

/* sum of penetrations of a sphere against every environment cuboid and sphere */
static double pen_env(const or_problem *pr, const double c[3], double r, double grad[3], double *maxpen) {
    double total = 0.0, g[3];
    if (grad) grad[0] = grad[1] = grad[2] = 0.0;
    for (int o = 0; o < pr->n_cub; ++o) {
        const double *cb = pr->cub + 15 * o;
        double pen = or_pen_box(c, r, cb, cb + 3, cb + 12, g, NULL);
        total += pen;
        if (maxpen && pen > *maxpen) *maxpen = pen;
        if (grad) for (int i = 0; i < 3; ++i) grad[i] += g[i];
    }
    for (int o = 0; o < pr->n_sph; ++o) {
        double pen = or_pen_sph(c, r, pr->sph + 4 * o, g);
        total += pen;
        if (maxpen && pen > *maxpen) *maxpen = pen;
        if (grad) for (int i = 0; i < 3; ++i) grad[i] += g[i];
    }
    return total;
}

/* ------------------------------------------------------------------------------------ */
/* Stage 1: tower placement cost (Appendix, tower stacking).                             */
/*                                                                                       */
/* Readings: blocks are indexed by stack position (skeleton order, bottom first).        */
/*  C_height = sum_i (z_i - zt_i)^2 with zt_i the centre height of a block resting on    */
/*    the blocks below it: z_table + sum_{k<i} 2 hz_k + hz_i (for equal blocks the top   */
/*    face is at i * h_block, as in the appendix).                                      */
/*  C_stable = sum_{i<B-1} Dist(mean_{j>i} (x_j, y_j), footprint_i), the distance from   */
/*    the centre of mass of the blocks above (equal masses) to block i's rotated         */
/*    rectangle, zero inside.                                                            */
/*  C_coll = sum_{i<j} Pen(spheres of block j, cuboid of block i)                        */
/*         + sum_i sum_o Pen(spheres of block i, o)  over the environment.               */
/*  "Linear" and "quadratic" forms differ only in the penetration terms: pen or pen^2.   */
/* ------------------------------------------------------------------------------------ */
static double z_target(const or_problem *pr, int i) {
    double z = pr->z_table;
    for (int k = 0; k < i; ++k) z += 2.0 * pr->half[3 * k + 2];
    return z + pr->half[3 * i + 2];
}

/* block sphere world centre and its derivative w.r.t. yaw of the block */
static void block_sphere_world(const double pose[4], const double l[3], double c[3], double dc_dyaw[3]) {
    double cy = cos(pose[3]), sy = sin(pose[3]);
    c[0] = pose[0] + cy * l[0] - sy * l[1];
    c[1] = pose[1] + sy * l[0] + cy * l[1];
    c[2] = pose[2] + l[2];
    if (dc_dyaw) {
        dc_dyaw[0] = -sy * l[0] - cy * l[1];
        dc_dyaw[1] = cy * l[0] - sy * l[1];
        dc_dyaw[2] = 0.0;
    }
}

/* Penetration of sphere (c, r) into the unit cube of a packing block whose centre is the
 * block origin plus Rz(yaw) times the cell offset `off`; the gradient with respect to the
 * block pose goes through that centre (chain rule on pen_block's cube-pose gradient). */
static double pen_cell(const double c[3], double r, const double pose[4], const double off[2], double u,
                       double dpen_dc[3], double dpen_dpose[4]) {
    double cy = cos(pose[3]), sy = sin(pose[3]);
    double cp[4] = {pose[0] + cy * off[0] - sy * off[1], pose[1] + sy * off[0] + cy * off[1], pose[2], pose[3]};
    double half[3] = {0.5 * u, 0.5 * u, 0.5 * u};
    double gp[4];
    double pen = pen_block(c, r, cp, half, dpen_dc, gp);
    if (dpen_dpose) {
        double dcx = -sy * off[0] - cy * off[1], dcy = cy * off[0] - sy * off[1];
        dpen_dpose[0] = gp[0];
        dpen_dpose[1] = gp[1];
        dpen_dpose[2] = gp[2];
        dpen_dpose[3] = gp[3] + gp[0] * dcx + gp[1] * dcy;
    }
    return pen;
}

/* Packing residuals (appendix, Tetris problem): e[i] = z_i - z*, and the penetration sum
 * (pen, or pen^2 when `quad`) of every sphere of block j against every unit cube of each
 * block i < j and against the walls (the environment).  A unit cube of edge u carries 8
 * spheres of radius u/4 at (+-u/4, +-u/4, +-u/4) from its centre (objects as sphere sets,
 * Sec. III), so cubes in face contact do not penetrate.  With g != NULL accumulates
 * g += sum_i b[i] de_i/dx + s_coll dC_coll/dx.  metrics = (largest penetration, 0,
 * largest |e|). */
static void pack_residuals(const or_problem *pr, const double *x, int quad, double *e, double *c_coll,
                           const double *b, double s_coll, double *g, double metrics[3]) {
    const int B = pr->B;
    const double u = pr->cell_size, r = 0.25 * u;
    double cc = 0.0, maxpen = 0.0, maxdz = 0.0;
    for (int i = 0; i < B; ++i) {
        e[i] = x[4 * i + 2] - pr->z_star;
        if (fabs(e[i]) > maxdz) maxdz = fabs(e[i]);
        if (g) g[4 * i + 2] += b[i];
    }
    for (int j = 0; j < B; ++j) {
        for (int k = pr->cell_start[j]; k < pr->cell_start[j + 1]; ++k) {
            for (int m = 0; m < 8; ++m) {
                double l[3] = {pr->cell[2 * k] + ((m & 1) ? 0.25 : -0.25) * u,
                               pr->cell[2 * k + 1] + ((m & 2) ? 0.25 : -0.25) * u, ((m & 4) ? 0.25 : -0.25) * u};
                double c[3], dc_dyaw[3];
                block_sphere_world(x + 4 * j, l, c, dc_dyaw);
                for (int o = 0; o < pr->n_cub + pr->n_sph; ++o) {
                    double gc[3], pen;
                    if (o < pr->n_cub) {
                        const double *cb = pr->cub + 15 * o;
                        pen = or_pen_box(c, r, cb, cb + 3, cb + 12, gc, NULL);
                    } else {
                        pen = or_pen_sph(c, r, pr->sph + 4 * (o - pr->n_cub), gc);
                    }
                    if (pen > maxpen) maxpen = pen;
                    cc += quad ? pen * pen : pen;
                    if (g && pen > 0.0) {
                        double sc = s_coll * (quad ? 2.0 * pen : 1.0);
                        for (int d = 0; d < 3; ++d) g[4 * j + d] += sc * gc[d];
                        g[4 * j + 3] += sc * dot3(gc, dc_dyaw);
                    }
                }
                for (int i = 0; i < j; ++i)
                    for (int kk = pr->cell_start[i]; kk < pr->cell_start[i + 1]; ++kk) {
                        double gc[3], gp[4];
                        double pen = pen_cell(c, r, x + 4 * i, pr->cell + 2 * kk, u, gc, gp);
                        if (pen > maxpen) maxpen = pen;
                        cc += quad ? pen * pen : pen;
                        if (g && pen > 0.0) {
                            double sc = s_coll * (quad ? 2.0 * pen : 1.0);
                            for (int d = 0; d < 3; ++d) g[4 * j + d] += sc * gc[d];
                            g[4 * j + 3] += sc * dot3(gc, dc_dyaw);
                            for (int d = 0; d < 4; ++d) g[4 * i + d] += sc * gp[d];
                        }
                    }
            }
        }
    }
    *c_coll = cc;
    if (metrics) { metrics[0] = maxpen; metrics[1] = 0.0; metrics[2] = maxdz; }
}

/* Placement residuals: D[i] = CoM distance for block i (i < B-1; D[B-1] = 0),
 * e[i] = z_i - zt_i, and the collision sum (pen, or pen^2 when `quad`).  With g != NULL
 * accumulates  g += sum_i a[i] dD_i/dx + sum_i b[i] de_i/dx + s_coll dC_coll/dx.
 * metrics = (largest single penetration, largest D, largest |e|). */
static void place_residuals(const or_problem *pr, const double *x, int quad, double *D, double *e,
                            double *c_coll, const double *a, const double *b, double s_coll, double *g,
                            double metrics[3]) {
    const int B = pr->B;
    double cc = 0.0, maxpen = 0.0, maxd = 0.0, maxdz = 0.0;

    /* height */
    for (int i = 0; i < B; ++i) {
        e[i] = x[4 * i + 2] - z_target(pr, i);
        if (fabs(e[i]) > maxdz) maxdz = fabs(e[i]);
        if (g) g[4 * i + 2] += b[i];
    }

    /* stability */
    D[B - 1] = 0.0;
    for (int i = 0; i + 1 < B; ++i) {
        int n_above = B - 1 - i;
        double m[2] = {0.0, 0.0};
        for (int j = i + 1; j < B; ++j) { m[0] += x[4 * j]; m[1] += x[4 * j + 1]; }
        m[0] /= n_above; m[1] /= n_above;
        double yaw = x[4 * i + 3], cy = cos(yaw), sy = sin(yaw);
        double v[2] = {m[0] - x[4 * i], m[1] - x[4 * i + 1]};
        double u[2] = {cy * v[0] + sy * v[1], -sy * v[0] + cy * v[1]};   /* Rz(-yaw) v */
        double ex[2], sg[2];
        for (int k = 0; k < 2; ++k) {
            sg[k] = u[k] >= 0.0 ? 1.0 : -1.0;
            ex[k] = relu(fabs(u[k]) - pr->half[3 * i + k]);
        }
        D[i] = sqrt(ex[0] * ex[0] + ex[1] * ex[1]);
        if (D[i] > maxd) maxd = D[i];
        if (g && D[i] > 0.0 && a[i] != 0.0) {
            double dD_du[2] = {sg[0] * ex[0] / D[i], sg[1] * ex[1] / D[i]};
            /* du/dv = Rz(-yaw) -> dD/dv = Rz(-yaw)^T dD/du */
            double dD_dv[2] = {cy * dD_du[0] - sy * dD_du[1], sy * dD_du[0] + cy * dD_du[1]};
            g[4 * i] -= a[i] * dD_dv[0];
            g[4 * i + 1] -= a[i] * dD_dv[1];
            /* du/dyaw = (u_y, -u_x) */
            g[4 * i + 3] += a[i] * (dD_du[0] * u[1] - dD_du[1] * u[0]);
            for (int j = i + 1; j < B; ++j) {
                g[4 * j] += a[i] * dD_dv[0] / n_above;
                g[4 * j + 1] += a[i] * dD_dv[1] / n_above;
            }
        }
    }

    /* collisions: spheres of block j vs the cuboid of block i (i < j), and vs the environment */
    for (int j = 0; j < B; ++j) {
        const double *hj = pr->half + 3 * j;
        for (int m = 0; m < 8; ++m) {
            double l[3], r, c[3], dc_dyaw[3];
            block_sphere_local(hj, m, l, &r);
            block_sphere_world(x + 4 * j, l, c, dc_dyaw);
            for (int o = 0; o < pr->n_cub + pr->n_sph; ++o) {
                double gc[3], pen;
                if (o < pr->n_cub) {
                    const double *cb = pr->cub + 15 * o;
                    pen = or_pen_box(c, r, cb, cb + 3, cb + 12, gc, NULL);
                } else {
                    pen = or_pen_sph(c, r, pr->sph + 4 * (o - pr->n_cub), gc);
                }
                if (pen > maxpen) maxpen = pen;
                cc += quad ? pen * pen : pen;
                if (g && pen > 0.0) {
                    double sc = s_coll * (quad ? 2.0 * pen : 1.0);
                    g[4 * j] += sc * gc[0];
                    g[4 * j + 1] += sc * gc[1];
                    g[4 * j + 2] += sc * gc[2];
                    g[4 * j + 3] += sc * dot3(gc, dc_dyaw);
                }
            }
            for (int i = 0; i < j; ++i) {
                double gc[3], gp[4];
                double pen = pen_block(c, r, x + 4 * i, pr->half + 3 * i, gc, gp);
                if (pen > maxpen) maxpen = pen;
                cc += quad ? pen * pen : pen;
                if (g && pen > 0.0) {
                    double sc = s_coll * (quad ? 2.0 * pen : 1.0);
                    g[4 * j] += sc * gc[0];
                    g[4 * j + 1] += sc * gc[1];
                    g[4 * j + 2] += sc * gc[2];
                    g[4 * j + 3] += sc * dot3(gc, dc_dyaw);
                    for (int k = 0; k < 4; ++k) g[4 * i + k] += sc * gp[k];
                }
            }
        }
    }
    *c_coll = cc;
    if (metrics) { metrics[0] = maxpen; metrics[1] = maxd; metrics[2] = maxdz; }
}

/* Cost (linear or quadratic form), gradient (B x 4, may be NULL) and the three terms
 * (C_stable, C_height, C_coll).  Two passes: residuals, then the gradient. */
double or_place_cost(const or_problem *pr, const double *x, int quad, double *grad, double terms[3]) {
    const int B = pr->B;
    if (pr->kind == OR_KIND_PACK) {
        /* C = w_coll (sum of block-block and block-wall penetrations) + w_height sum |z_i - z*|;
         * the absolute value keeps its form in both phases (only penetrations turn quadratic) */
        double e[64], b[64], cc, ch = 0.0;
        pack_residuals(pr, x, quad, e, &cc, NULL, 0.0, NULL, NULL);
        for (int i = 0; i < B; ++i) ch += fabs(e[i]);
        if (grad) {
            for (int i = 0; i < B; ++i) b[i] = pr->w_height * (e[i] > 0.0 ? 1.0 : (e[i] < 0.0 ? -1.0 : 0.0));
            memset(grad, 0, sizeof(double) * 4 * B);
            double e2[64], cc2;
            pack_residuals(pr, x, quad, e2, &cc2, b, pr->w_coll, grad, NULL);
        }
        if (terms) { terms[0] = 0.0; terms[1] = ch; terms[2] = cc; }
        return pr->w_height * ch + pr->w_coll * cc;
    }
    double *buf = (double *)malloc(sizeof(double) * 4 * B);
    double *D = buf, *e = buf + B, *a = buf + 2 * B, *b = buf + 3 * B;
    double cc;
    place_residuals(pr, x, quad, D, e, &cc, NULL, NULL, 0.0, NULL, NULL);
    double cs = 0.0, ch = 0.0;
    for (int i = 0; i < B; ++i) { cs += D[i]; ch += e[i] * e[i]; }
    double cost = pr->w_stable * cs + pr->w_height * ch + pr->w_coll * cc;
    if (grad) {
        for (int i = 0; i < B; ++i) { a[i] = pr->w_stable; b[i] = 2.0 * pr->w_height * e[i]; }
        memset(grad, 0, sizeof(double) * 4 * B);
        double D2[64], e2[64], cc2;
        place_residuals(pr, x, quad, D2, e2, &cc2, a, b, pr->w_coll, grad, NULL);
    }
    if (terms) { terms[0] = cs; terms[1] = ch; terms[2] = cc; }
    free(buf);
    return cost;
}

/* GetSatisfyingParticles (Alg. 1): every single penetration, every CoM distance and
 * every height error within eps (|f(x)| < eps, Sec. III). */
int or_place_check(const or_problem *pr, const double *x, double metrics[3]) {
    double D[64], e[64], cc, m[3];
    if (pr->kind == OR_KIND_PACK)
        pack_residuals(pr, x, 0, e, &cc, NULL, 0.0, NULL, m);
    else
        place_residuals(pr, x, 0, D, e, &cc, NULL, NULL, 0.0, NULL, m);
    if (metrics) { metrics[0] = m[0]; metrics[1] = m[1]; metrics[2] = m[2]; }
    return m[0] <= pr->eps && m[1] <= pr->eps && m[2] <= pr->eps;
}

/* Clamp to the problem bounding box (Sec. III-A: poses clamped to the box); yaw wrapped. */
static void place_clamp(const or_problem *pr, double *x) {
    for (int i = 0; i < pr->B; ++i) {
        double zlo = pr->box[2];
        double zr = pr->z_table + pr->half[3 * i + 2];
        if (zr > zlo) zlo = zr;
        x[4 * i] = clampd(x[4 * i], pr->box[0], pr->box[3]);
        x[4 * i + 1] = clampd(x[4 * i + 1], pr->box[1], pr->box[4]);
        x[4 * i + 2] = clampd(x[4 * i + 2], zlo, pr->box[5]);
        x[4 * i + 3] = wrap_angle(x[4 * i + 3]);
    }
}

/* SampleUniform (Alg. 1): block i of particle n from Philox counter (i, n, 0, attempt). */
void or_place_sample(const or_problem *pr, int n, uint32_t attempt, double *x) {
    const int B = pr->B;
    for (int p = 0; p < n; ++p)
        for (int i = 0; i < B; ++i) {
            uint32_t u[4];
            philox(pr, (uint32_t)i, (uint32_t)p, TAG_SAMPLE, attempt, u);
            double zlo = pr->box[2];
            double zr = pr->z_table + pr->half[3 * i + 2];
            if (zr > zlo) zlo = zr;
            double *xi = x + (size_t)4 * B * p + 4 * i;
            xi[0] = pr->box[0] + or_u01(u[0]) * (pr->box[3] - pr->box[0]);
            xi[1] = pr->box[1] + or_u01(u[1]) * (pr->box[4] - pr->box[1]);
            xi[2] = zlo + or_u01(u[2]) * (pr->box[5] - zlo);
            xi[3] = -PI + or_u01(u[3]) * (2.0 * PI);
        }
}

/* ArgSort (Alg. 1): stable ascending order of the costs; NaN sorts last. */
typedef struct { double c; int32_t i; } keyed;
static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    double cx = isnan(x->c) ? INFINITY : x->c, cy = isnan(y->c) ? INFINITY : y->c;
    if (cx < cy) return -1;
    if (cx > cy) return 1;
    return (x->i > y->i) - (x->i < y->i);
}

void or_argsort(int n, const double *cost, int32_t *idx) {
    keyed *k = (keyed *)malloc(sizeof(keyed) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) { k[i].c = cost[i]; k[i].i = i; }
    qsort(k, (size_t)n, sizeof(keyed), cmp_keyed);
    for (int i = 0; i < n; ++i) idx[i] = k[i].i;
    free(k);
}

/* Alg. 1 linear cost descent then quadratic refinement, each particle independently:
 *   k = 1..K_lin : eta = eta_init (1 - k/K_lin);  x <- clamp(x - eta grad C_linear)
 *   k = 1..K_quad: x <- clamp(x - alpha grad C_quadratic) */
void or_place_descend(const or_problem *pr, int m, double *x, int k_lin, int k_quad) {
    const int B = pr->B;
#pragma omp parallel for schedule(dynamic) num_threads(pr->n_threads > 0 ? pr->n_threads : 1)
    for (int p = 0; p < m; ++p) {
        double *xp = x + (size_t)4 * B * p;
        double *g = (double *)malloc(sizeof(double) * 4 * B);
        for (int k = 1; k <= k_lin; ++k) {
            double eta = pr->eta_init * (1.0 - (double)k / (double)k_lin);
            or_place_cost(pr, xp, 0, g, NULL);
            for (int v = 0; v < 4 * B; ++v) xp[v] -= eta * g[v];
            place_clamp(pr, xp);
        }
        for (int k = 1; k <= k_quad; ++k) {
            or_place_cost(pr, xp, 1, g, NULL);
            for (int v = 0; v < 4 * B; ++v) xp[v] -= pr->alpha * g[v];
            place_clamp(pr, xp);
        }
        free(g);
    }
}

/* Alg. 1 with the re-initialisation loop (Sec. III-A): repeat until a satisfying
 * particle exists or max_steps gradient steps were spent (the experiments' cap).
 * Returns the best P (fewer if fewer satisfy) by quadratic-form cost in `out`. */
int or_place_solve(const or_problem *pr, double *out, int *n_found, int *attempts, int *steps) {
    const int B = pr->B, N = pr->N, M = pr->M;
    double *xs = (double *)malloc(sizeof(double) * 4 * B * (size_t)N);
    double *xm = (double *)malloc(sizeof(double) * 4 * B * (size_t)M);
    double *cost = (double *)malloc(sizeof(double) * (size_t)N);
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int spent = 0, a = 0, found = 0;
    while (spent < pr->max_steps) {
        or_place_sample(pr, N, (uint32_t)a, xs);
#pragma omp parallel for schedule(dynamic) num_threads(pr->n_threads > 0 ? pr->n_threads : 1)
        for (int p = 0; p < N; ++p) cost[p] = or_place_cost(pr, xs + (size_t)4 * B * p, 0, NULL, NULL);
        or_argsort(N, cost, idx);
        for (int r = 0; r < M; ++r) memcpy(xm + (size_t)4 * B * r, xs + (size_t)4 * B * idx[r], sizeof(double) * 4 * B);
        or_place_descend(pr, M, xm, pr->K_lin, pr->K_quad);
        spent += pr->K_lin + pr->K_quad;
        ++a;
        /* satisfying particles, ranked by their final (quadratic-form) cost */
        int ns = 0;
        for (int r = 0; r < M; ++r)
            if (or_place_check(pr, xm + (size_t)4 * B * r, NULL)) {
                cost[ns] = or_place_cost(pr, xm + (size_t)4 * B * r, 1, NULL, NULL);
                slot[ns++] = r;
            }
        if (ns > 0) {
            or_argsort(ns, cost, idx);
            found = ns < pr->P ? ns : pr->P;
            for (int s = 0; s < found; ++s)
                memcpy(out + (size_t)4 * B * s, xm + (size_t)4 * B * slot[idx[s]], sizeof(double) * 4 * B);
            break;
        }
    }
    if (n_found) *n_found = found;
    if (attempts) *attempts = a;
    if (steps) *steps = spent;
    free(xs); free(xm); free(cost); free(idx); free(slot);
    return found > 0;
}

/* ------------------------------------------------------------------------------------ */
/* Stage 2: trajectory optimisation.                                                      */
/*                                                                                       */
/* Readings (the appendix indexes only q_{b,t}, t = 0..T):                                */
/*  - two motion segments per block, each of W waypoints (S = W-1 steps): a transit      */
/*    segment from the previous place configuration (q_home for the first block) to the  */
/*    grasp configuration, then a transfer segment to the place configuration.  Shared   */
/*    endpoints are stored once: C = 2B S + 1 configurations, q[0] = q_home (fixed).      */
/*  - configuration t >= 1 belongs to segment s = (t-1)/S, block b = s/2, and is a      */
/*    transfer waypoint when s is odd.  Grasp of block b: t = (2b+1)S; place: (2b+2)S.   */
/*  - obstacles of a configuration: the environment, the blocks already placed (k < b,  */
/*    at the pose fk gives at their place configuration) and the blocks not yet moved    */
/*    (k > b, initial pose); block b itself is excluded.                                */
/*  - C_arm sums every arm sphere over t = 1..C-1; C_block the held block's spheres over */
/*    the transfer interior (t in [1, T-1] of the transfer segment).                     */
/*  - the block frame held by the tool: EE z-axis points down onto the block's top face, */
/*    block = tool * Rx(pi) * Trans(0, 0, -(hz + grasp_off)).  Placement poses are the   */
/*    (x, y, z, yaw) reduction of it, yaw = atan2(R10, R00).                             */
/*  - C_start: squared position error and squared roll/pitch (ZYX) of the block frame at */
/*    each grasp configuration; the block must also stay upright, so roll^2 + pitch^2 at  */
/*    each place configuration is added to the same group.                               */
/*  - path cost sum ||q_{t+1} - q_t||^2 (configuration-space distance, Sec. III), joint  */
/*    limit residual sum relu(q - hi)^2 + relu(lo - q)^2.                                */
/*  - augmented Lagrangian over the residual vector h (see or_n_residuals), scaled by   */
/*    sqrt of the group weight: L = w_path path + w_jl jl                               */
/*                                 + sum_r lambda_r hw_r + mu/2 hw_r^2, hw = sqrt(w) h. */
/* ------------------------------------------------------------------------------------ */
int or_n_configs(const or_problem *pr) {
    return pr->kind == OR_KIND_P2P ? pr->W : 2 * pr->B * (pr->W - 1) + 1;
}

static int t_grasp(const or_problem *pr, int b) { return (2 * b + 1) * (pr->W - 1); }
static int t_place(const or_problem *pr, int b) { return (2 * b + 2) * (pr->W - 1); }

/* block frame held by the tool of frames/tee: R_blk = R_ee diag(1,-1,-1),
 * p_blk = p_ee + (hz + grasp_off) z_ee */
static void held_block_frame(const or_problem *pr, int b, const double tee[16], double R[9], double p[3]) {
    double off = pr->half[3 * b + 2] + pr->grasp_off;
    for (int i = 0; i < 3; ++i) {
        R[3 * i] = tee[4 * i];
        R[3 * i + 1] = -tee[4 * i + 1];
        R[3 * i + 2] = -tee[4 * i + 2];
        p[i] = tee[4 * i + 3] + off * tee[4 * i + 2];
    }
}

static void pose4_of(const or_problem *pr, int b, const double tee[16], double pose[4]) {
    double R[9], p[3];
    held_block_frame(pr, b, tee, R, p);
    pose[0] = p[0]; pose[1] = p[1]; pose[2] = p[2];
    pose[3] = atan2(R[3], R[0]);
}

/* 4 x 7 Jacobian of pose4 w.r.t. the joints of the configuration it comes from */
static void pose4_jacobian(const or_problem *pr, int b, double frames[8][16], const double tee[16], double J[4][7]) {
    double R[9], p[3], Jp[3][7];
    held_block_frame(pr, b, tee, R, p);
    point_jacobian(frames, 7, p, Jp);
    double e[3] = {R[0], R[3], R[6]};
    double den = e[0] * e[0] + e[1] * e[1];
    for (int j = 0; j < 7; ++j) {
        double z[3], de[3];
        col3(frames[j + 1], 2, z);
        cross3(z, e, de);
        J[0][j] = Jp[0][j]; J[1][j] = Jp[1][j]; J[2][j] = Jp[2][j];
        J[3][j] = (e[0] * de[1] - e[1] * de[0]) / den;
    }
}

/* roll, pitch (ZYX) of a rotation and their derivatives w.r.t. the joints */
static void roll_pitch(double frames[8][16], const double R[9], double *roll, double *pitch,
                       double droll[7], double dpitch[7]) {
    double r21 = R[7], r22 = R[8], r20 = R[6];
    double h2 = r21 * r21 + r22 * r22, h = sqrt(h2);
    *roll = atan2(r21, r22);
    *pitch = atan2(-r20, h);
    if (!droll) return;
    for (int j = 0; j < 7; ++j) {
        double dR[9];
        rot_derivative(frames, R, j, dR);
        droll[j] = (r22 * dR[7] - r21 * dR[8]) / h2;
        double dh = (r21 * dR[7] + r22 * dR[8]) / h;
        dpitch[j] = (h * (-dR[6]) - (-r20) * dh) / (r20 * r20 + h2);
    }
}

/* Residual vector of the stage-2 augmented Lagrangian, NR = 9B + 3 entries:
 *   [5b .. 5b+4]        grasp of block b: position error (3), roll, pitch      (w_start)
 *   [5B + 2b .. +1]     place of block b: roll, pitch (upright block)         (w_start)
 *   [7B + b]            height residual z_b - zt_b                             (w_height)
 *   [8B + b]            CoM distance D_b (b < B-1; the last entry stays 0)     (w_stable)
 *   [9B], [9B+1], [9B+2] placement collision sum, C_arm, C_block             (w_coll, w_arm, w_block)
 * The squared norms of these residual groups are the appendix terms C_start, C_height;
 * the others are the (non-negative) penetration and distance sums themselves. */
int or_n_residuals(const or_problem *pr) { return 9 * pr->B + 3; }

static double residual_weight(const or_problem *pr, int r) {
    const int B = pr->B;
    if (r < 7 * B) return pr->w_start;
    if (r < 8 * B) return pr->w_height;
    if (r < 9 * B) return pr->w_stable;
    if (r == 9 * B) return pr->w_coll;
    if (r == 9 * B + 1) return pr->w_arm;
    return pr->w_block;
}

typedef struct {
    double c[OR_NG];      /* appendix terms: C_start, C_arm, C_block, C_coll, C_stable, C_height */
    double path, jl;
    double maxpen;        /* largest single arm / held-block penetration */
    double max_start;     /* largest grasp alignment value (squared residual norm) */
    double max_tilt;      /* largest placement tilt value */
    double place_metrics[3];
    int limits_ok;
} traj_eval;

/* One configuration's collision terms.  With grad != NULL, adds s_arm * dC_arm/dq_t and
 * s_block * dC_block/dq_t to grad_t and the pose derivatives of placed blocks to g4. */
static void config_collisions(const or_problem *pr, const double *q, int t, double (*P4)[4],
                              double *c_arm, double *c_block, double *maxpen,
                              double s_arm, double s_block, double *grad_t, double (*g4)[4]) {
    const int S = pr->W - 1, B = pr->B;
    int s = (t - 1) / S, b = s / 2, j = t - s * S;
    int held = (s & 1) && (j < S);
    double frames[8][16], tee[16];
    or_fk(pr, q + 7 * t, frames, tee);

    /* context blocks */
    double ctx_pose[64][4];
    int ctx_blk[64], n_ctx = 0;
    for (int k = 0; k < B; ++k) {
        if (k == b) continue;
        const double *src = k < b ? P4[k] : pr->init + 4 * k;
        memcpy(ctx_pose[n_ctx], src, sizeof(double) * 4);
        ctx_blk[n_ctx++] = k;
    }

    int n_items = pr->n_spheres + (held ? 8 : 0);
    for (int it = 0; it < n_items; ++it) {
        double c[3], r;
        int link;
        if (it < pr->n_spheres) {
            link = pr->sphere_link[it];
            xform(frames[link], pr->sphere + 4 * it, c);
            r = pr->sphere[4 * it + 3];
        } else {
            double Rb[9], pb[3], l[3];
            held_block_frame(pr, b, tee, Rb, pb);
            block_sphere_local(pr->half + 3 * b, it - pr->n_spheres, l, &r);
            for (int i = 0; i < 3; ++i) c[i] = pb[i] + Rb[3 * i] * l[0] + Rb[3 * i + 1] * l[1] + Rb[3 * i + 2] * l[2];
            link = 7;
        }
        int is_block = it >= pr->n_spheres;
        double gsum[3];
        double tot = pen_env(pr, c, r, grad_t ? gsum : NULL, maxpen);
        for (int k = 0; k < n_ctx; ++k) {
            double g[3], gp[4];
            double pen = pen_block(c, r, ctx_pose[k], pr->half + 3 * ctx_blk[k], g, gp);
            tot += pen;
            if (maxpen && pen > *maxpen) *maxpen = pen;
            if (grad_t) {
                for (int i = 0; i < 3; ++i) gsum[i] += g[i];
                if (ctx_blk[k] < b) {
                    double sc = is_block ? s_block : s_arm;
                    for (int i = 0; i < 4; ++i) g4[ctx_blk[k]][i] += sc * gp[i];
                }
            }
        }
        if (is_block) *c_block += tot; else *c_arm += tot;
        if (grad_t) {
            double J[3][7];
            double sc = is_block ? s_block : s_arm;
            point_jacobian(frames, link, c, J);
            for (int jj = 0; jj < 7; ++jj)
                grad_t[jj] += sc * (J[0][jj] * gsum[0] + J[1][jj] * gsum[1] + J[2][jj] * gsum[2]);
        }
    }
}

/* Evaluate residuals h (NR) and the appendix terms; with grad != NULL also the gradient
 * sum_r s[r] dh_r/dq + w_path dpath/dq + w_jl djl/dq, where s = dL/dh. */
static void traj_evaluate(const or_problem *pr, const double *q, traj_eval *ev, double *h,
                          const double *s, double *grad) {
    const int B = pr->B, C = or_n_configs(pr);
    const int p2p = pr->kind == OR_KIND_P2P;
    double (*P4)[4] = (double (*)[4])calloc((size_t)4 * B, sizeof(double));
    double (*g4)[4] = (double (*)[4])calloc((size_t)4 * B, sizeof(double));
    memset(ev, 0, sizeof *ev);
    for (int b = 0; b < B && !p2p; ++b) {
        double fr[8][16], tee[16];
        or_fk(pr, q + 7 * t_place(pr, b), fr, tee);
        pose4_of(pr, b, tee, P4[b]);
    }
    if (grad) memset(grad, 0, sizeof(double) * 7 * (size_t)C);

    /* C_arm, C_block over all configurations */
    for (int t = 1; t < C; ++t)
        config_collisions(pr, q, t, P4, &ev->c[OR_G_ARM], &ev->c[OR_G_BLOCK], &ev->maxpen,
                          grad ? s[9 * B + 1] : 0.0, grad ? s[9 * B + 2] : 0.0,
                          grad ? grad + 7 * t : NULL, g4);
    h[9 * B + 1] = ev->c[OR_G_ARM];
    h[9 * B + 2] = ev->c[OR_G_BLOCK];

    /* C_placement residuals on the placed poses (none point to point) */
    if (!p2p) {
        double cc;
        place_residuals(pr, &P4[0][0], 0, h + 8 * B, h + 7 * B, &cc,
                        grad ? s + 8 * B : NULL, grad ? s + 7 * B : NULL, grad ? s[9 * B] : 0.0,
                        grad ? &g4[0][0] : NULL, ev->place_metrics);
        h[9 * B] = cc;
        ev->c[OR_G_COLL] = cc;
        for (int b = 0; b < B; ++b) {
            ev->c[OR_G_STABLE] += h[8 * B + b];
            ev->c[OR_G_HEIGHT] += h[7 * B + b] * h[7 * B + b];
        }
    }

    /* placed-pose derivatives -> place configurations */
    if (grad && !p2p) {
        for (int b = 0; b < B; ++b) {
            int t = t_place(pr, b);
            double fr[8][16], tee[16], J[4][7];
            or_fk(pr, q + 7 * t, fr, tee);
            pose4_jacobian(pr, b, fr, tee, J);
            for (int j = 0; j < 7; ++j)
                for (int i = 0; i < 4; ++i) grad[7 * t + j] += J[i][j] * g4[b][i];
        }
    }

    /* C_start residuals: grasp alignment (position, roll, pitch) and upright placement */
    for (int b = 0; b < B; ++b) {
        for (int which = 0; which < (p2p ? 1 : 2); ++which) {
            int t = which == 0 ? t_grasp(pr, b) : t_place(pr, b);
            double fr[8][16], tee[16], R[9], p[3], roll, pitch, dr[7], dp[7];
            or_fk(pr, q + 7 * t, fr, tee);
            held_block_frame(pr, b, tee, R, p);
            roll_pitch(fr, R, &roll, &pitch, dr, dp);
            double *hr = which == 0 ? h + 5 * b : h + 5 * B + 2 * b;
            const double *sr = grad ? (which == 0 ? s + 5 * b : s + 5 * B + 2 * b) : NULL;
            double val;
            if (which == 0) {
                for (int i = 0; i < 3; ++i) hr[i] = p[i] - pr->init[4 * b + i];
                hr[3] = roll; hr[4] = pitch;
                val = hr[0] * hr[0] + hr[1] * hr[1] + hr[2] * hr[2] + roll * roll + pitch * pitch;
                if (val > ev->max_start) ev->max_start = val;
            } else {
                hr[0] = roll; hr[1] = pitch;
                val = roll * roll + pitch * pitch;
                if (val > ev->max_tilt) ev->max_tilt = val;
            }
            ev->c[OR_G_START] += val;
            if (grad) {
                double J[3][7];
                point_jacobian(fr, 7, p, J);
                for (int j = 0; j < 7; ++j) {
                    double gj;
                    if (which == 0)
                        gj = sr[0] * J[0][j] + sr[1] * J[1][j] + sr[2] * J[2][j] + sr[3] * dr[j] + sr[4] * dp[j];
                    else
                        gj = sr[0] * dr[j] + sr[1] * dp[j];
                    grad[7 * t + j] += gj;
                }
            }
        }
    }

    /* path length and joint limits */
    ev->limits_ok = 1;
    for (int t = 0; t + 1 < C; ++t)
        for (int j = 0; j < 7; ++j) {
            double d = q[7 * (t + 1) + j] - q[7 * t + j];
            ev->path += d * d;
            if (grad) {
                grad[7 * (t + 1) + j] += pr->w_path * 2.0 * d;
                grad[7 * t + j] -= pr->w_path * 2.0 * d;
            }
        }
    for (int t = 1; t < C; ++t)
        for (int j = 0; j < 7; ++j) {
            double v = q[7 * t + j], lo = pr->qlim[2 * j], hi = pr->qlim[2 * j + 1];
            double over = relu(v - hi), under = relu(lo - v);
            ev->jl += over * over + under * under;
            if (over > 0.0 || under > 0.0) ev->limits_ok = 0;
            if (grad) grad[7 * t + j] += pr->w_jl * (2.0 * over - 2.0 * under);
        }
    if (grad) for (int j = 0; j < 7; ++j) grad[j] = 0.0;   /* q_home is not a variable */
    free(P4); free(g4);
}

/* L = w_path path + w_jl jl + sum_r (lambda_r hw_r + mu/2 hw_r^2), hw_r = sqrt(w_r) h_r
 * (augmented Lagrangian on the scaled residual vector; Nocedal & Wright, Numerical
 * Optimization, Sec. 17.3).  With the sqrt(w) scaling the quadratic part is mu/2 times the
 * weighted squared-error terms of the appendix (w_start C_start, w_height C_height).
 * grad (C x 7) and h (NR) may be NULL. */
double or_traj_cost(const or_problem *pr, const double *q, const double *lam, double mu,
                    double *grad, double c_groups[OR_NG], double *path, double *jl, double *h_out) {
    const int NR = or_n_residuals(pr);
    double *h = (double *)calloc((size_t)NR, sizeof(double));
    double *s = (double *)calloc((size_t)NR, sizeof(double));
    double *h2 = (double *)calloc((size_t)NR, sizeof(double));
    traj_eval ev;
    traj_evaluate(pr, q, &ev, h, NULL, NULL);            /* pass 1: residuals */
    double L = pr->w_path * ev.path + pr->w_jl * ev.jl;
    for (int r = 0; r < NR; ++r) {
        double sw = sqrt(residual_weight(pr, r)), hw = sw * h[r];
        L += lam[r] * hw + 0.5 * mu * hw * hw;
        s[r] = (lam[r] + mu * hw) * sw;                  /* dL/dh_r */
    }
    if (grad) {                                          /* pass 2: gradient */
        traj_eval ev2;
        traj_evaluate(pr, q, &ev2, h2, s, grad);
    }
    if (c_groups) for (int g = 0; g < OR_NG; ++g) c_groups[g] = ev.c[g];
    if (path) *path = ev.path;
    if (jl) *jl = ev.jl;
    if (h_out) memcpy(h_out, h, sizeof(double) * NR);
    free(h); free(s); free(h2);
    return L;
}

/* final feasibility: metrics = (max penetration, max grasp alignment, max tilt,
 * placement max penetration, max CoM distance, max height error) */
int or_traj_check(const or_problem *pr, const double *q, double metrics[6]) {
    traj_eval ev;
    double *h = (double *)calloc((size_t)or_n_residuals(pr), sizeof(double));
    traj_evaluate(pr, q, &ev, h, NULL, NULL);
    free(h);
    if (metrics) {
        metrics[0] = ev.maxpen; metrics[1] = ev.max_start; metrics[2] = ev.max_tilt;
        metrics[3] = ev.place_metrics[0]; metrics[4] = ev.place_metrics[1]; metrics[5] = ev.place_metrics[2];
    }
    return ev.maxpen <= pr->eps && ev.max_start <= pr->eps_start && ev.max_tilt <= pr->eps_start &&
           ev.place_metrics[0] <= pr->eps && ev.place_metrics[1] <= pr->eps && ev.place_metrics[2] <= pr->eps &&
           ev.limits_ok;
}

/* ranking cost of a returned trajectory: C_trajopt (appendix) + w_path path */
double or_traj_rank_cost(const or_problem *pr, const double *q) {
    traj_eval ev;
    double *h = (double *)calloc((size_t)or_n_residuals(pr), sizeof(double));
    traj_evaluate(pr, q, &ev, h, NULL, NULL);
    free(h);
    return pr->w_path * ev.path + pr->w_stable * ev.c[OR_G_STABLE] + pr->w_height * ev.c[OR_G_HEIGHT] +
           pr->w_coll * ev.c[OR_G_COLL] + pr->w_start * ev.c[OR_G_START] + pr->w_arm * ev.c[OR_G_ARM] +
           pr->w_block * ev.c[OR_G_BLOCK];
}

/* Inverse kinematics by damped least squares (Wampler 1986; Nakamura & Hanafusa 1986):
 *   e = (p* - p, 1/2 sum_i R[:,i] x R*[:,i]),  J_k = (z_k x (p - o_k), z_k),
 *   dq = J^T (J J^T + damp^2 I)^-1 e,  q <- clamp(q + dq),  K_ik iterations.
 * The paper uses an analytic Franka IK and allows any parallel differentiable IK
 * (Sec. III-B); the arm here is synthetic, so an iterative one is used. */
void or_ik(const or_problem *pr, const double target[16], const double q0[7], double q[7]) {
    memcpy(q, q0, 7 * sizeof(double));
    for (int it = 0; it < pr->K_ik; ++it) {
        double fr[8][16], tee[16], e[6], J[6][7], A[6][6], y[6];
        or_fk(pr, q, fr, tee);
        double p[3] = {tee[3], tee[7], tee[11]};
        for (int i = 0; i < 3; ++i) e[i] = target[4 * i + 3] - p[i];
        e[3] = e[4] = e[5] = 0.0;
        for (int c = 0; c < 3; ++c) {
            double r[3], rs[3], w[3];
            col3(tee, c, r);
            col3(target, c, rs);
            cross3(r, rs, w);
            for (int i = 0; i < 3; ++i) e[3 + i] += 0.5 * w[i];
        }
        double Jp[3][7];
        point_jacobian(fr, 7, p, Jp);
        for (int j = 0; j < 7; ++j) {
            double z[3];
            col3(fr[j + 1], 2, z);
            for (int i = 0; i < 3; ++i) { J[i][j] = Jp[i][j]; J[3 + i][j] = z[i]; }
        }
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 6; ++b) {
                double s = 0.0;
                for (int j = 0; j < 7; ++j) s += J[a][j] * J[b][j];
                A[a][b] = s + (a == b ? pr->ik_damp * pr->ik_damp : 0.0);
            }
        /* Gaussian elimination with partial pivoting on A y = e */
        double Mx[6][7];
        for (int a = 0; a < 6; ++a) { for (int b = 0; b < 6; ++b) Mx[a][b] = A[a][b]; Mx[a][6] = e[a]; }
        for (int col = 0; col < 6; ++col) {
            int piv = col;
            for (int r = col + 1; r < 6; ++r) if (fabs(Mx[r][col]) > fabs(Mx[piv][col])) piv = r;
            if (piv != col) for (int c = 0; c < 7; ++c) { double tmp = Mx[col][c]; Mx[col][c] = Mx[piv][c]; Mx[piv][c] = tmp; }
            for (int r = col + 1; r < 6; ++r) {
                double f = Mx[r][col] / Mx[col][col];
                for (int c = col; c < 7; ++c) Mx[r][c] -= f * Mx[col][c];
            }
        }
        for (int r = 5; r >= 0; --r) {
            double s = Mx[r][6];
            for (int c = r + 1; c < 6; ++c) s -= Mx[r][c] * y[c];
            y[r] = s / Mx[r][r];
        }
        for (int j = 0; j < 7; ++j) {
            double dq = 0.0;
            for (int a = 0; a < 6; ++a) dq += J[a][j] * y[a];
            q[j] = clampd(q[j] + dq, pr->qlim[2 * j], pr->qlim[2 * j + 1]);
        }
    }
}

/* top-down grasp of a block pose (x, y, z, yaw): tool z-axis along -world z, tool at the
 * block's top face (+grasp_off), tool yaw = block yaw + k pi/2 (k drawn by the lift) */
static void grasp_target(const or_problem *pr, int b, const double pose[4], int k, double T[16]) {
    double yaw = pose[3] + 0.5 * PI * (double)k, c = cos(yaw), s = sin(yaw);
    double off = pr->half[3 * b + 2] + pr->grasp_off;
    mat4_eye(T);
    /* Rz(yaw) Rx(pi) */
    T[0] = c;  T[1] = s;  T[2] = 0.0;
    T[4] = s;  T[5] = -c; T[6] = 0.0;
    T[8] = 0.0; T[9] = 0.0; T[10] = -1.0;
    T[3] = pose[0]; T[7] = pose[1]; T[11] = pose[2] + off;
}

static void perturbed_home(const or_problem *pr, uint32_t c0, int particle, uint32_t tag, uint32_t attempt,
                           double amp, double q[7]) {
    uint32_t u0[4], u1[4];
    philox(pr, 2u * c0, (uint32_t)particle, tag, attempt, u0);
    philox(pr, 2u * c0 + 1u, (uint32_t)particle, tag, attempt, u1);
    double u[7] = {or_u01(u0[0]), or_u01(u0[1]), or_u01(u0[2]), or_u01(u0[3]),
                   or_u01(u1[0]), or_u01(u1[1]), or_u01(u1[2])};
    for (int j = 0; j < 7; ++j)
        q[j] = clampd(pr->q_home[j] + amp * (2.0 * u[j] - 1.0), pr->qlim[2 * j], pr->qlim[2 * j + 1]);
}

/* ------------------------------------------------------------------------------------ */
/* Analytic IK (Sec. III-B lifts placements with the analytical IK of He and Liu, 2021,   */
/* for the Franka arm).  The arm here has that arm's joint layout: alpha = (0, -pi/2,     */
/* pi/2, pi/2, -pi/2, pi/2, pi/2), a_0 = a_1 = a_2 = a_5 = 0, d_1 = d_3 = d_5 = d_6 = 0;  */
/* the lengths d_0, d_2, a_3, a_4, d_4, a_6 and the tool are free.  Geometric solution,   */
/* with the last joint q_6 as the free parameter (written from the geometry):            */
/*  1. frame 7 = target E^-1, frame 6 = frame 7 T_6(q_6)^-1 (orientation and origin O6). */
/*  2. the first three axes meet at the shoulder S = (0, 0, d_0); |O6 - S|^2 depends on   */
/*     theta_3 only: K + 2 (a3 a4 + d2 d4) cos + 2 (d2 a4 - a3 d4) sin -> two theta_3.   */
/*  3. u = S - O6 in frame 4 is (-a3 c3 - d2 s3 - a4, a3 s3 - d2 c3 - d4, 0); w = S - O6 */
/*     in frame 6 is known; R_6^4(theta_4, theta_5)^T u = w gives                         */
/*     w_x sin t5 + w_y cos t5 = u_y (two theta_5), then u_x sin t4 = w_z and             */
/*     u_x cos t4 = w_x cos t5 - w_y sin t5 (theta_4).                                    */
/*  4. frame 3's orientation R3 = R6 (R_4^3 R_5^4 R_6^5)^T = Rz(t0) Ry(t1) Rz(t2) is split */
/*     as z-y-z Euler angles, both signs of sin t1.                                        */
/* Up to 8 solutions; each is brought into the joint limits by +-2 pi where possible and  */
/* kept only if every joint is within them.                                              */
/* ------------------------------------------------------------------------------------ */
static const double IK_ALPHA[7] = {0.0, -PI / 2, PI / 2, PI / 2, -PI / 2, PI / 2, PI / 2};

int or_ik_analytic_supported(const or_problem *pr) {
    const double *dh = pr->dh;
    for (int k = 0; k < 7; ++k)
        if (fabs(dh[4 * k + 1] - IK_ALPHA[k]) > 1e-9) return 0;
    const int zero_a[4] = {0, 1, 2, 5}, zero_d[4] = {1, 3, 5, 6};
    for (int i = 0; i < 4; ++i)
        if (dh[4 * zero_a[i]] != 0.0 || dh[4 * zero_d[i] + 2] != 0.0) return 0;
    double a3 = dh[12], a4 = dh[16], d2 = dh[10], d4 = dh[18];
    return hypot(a3 * a4 + d2 * d4, d2 * a4 - a3 * d4) > 0.0;
}

/* inverse of a rigid 4x4 transform */
static void rigid_inverse(const double T[16], double Ti[16]) {
    mat4_eye(Ti);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ti[4 * i + j] = T[4 * j + i];
    for (int i = 0; i < 3; ++i) Ti[4 * i + 3] = -(Ti[4 * i] * T[3] + Ti[4 * i + 1] * T[7] + Ti[4 * i + 2] * T[11]);
}

/* rotation part of a DH row: Rot_x(alpha) Rot_z(theta), 3x3 row-major */
static void rot_xz(double alpha, double theta, double R[9]) {
    double ca = cos(alpha), sa = sin(alpha), ct = cos(theta), st = sin(theta);
    R[0] = ct;      R[1] = -st;     R[2] = 0.0;
    R[3] = ca * st; R[4] = ca * ct; R[5] = -sa;
    R[6] = sa * st; R[7] = sa * ct; R[8] = ca;
}

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

/* C = A B^T */
static void mat3_mul_bt(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[3 * j] + A[3 * i + 1] * B[3 * j + 1] + A[3 * i + 2] * B[3 * j + 2];
}

/* joint angle theta_k -> q_k inside [lo, hi] (shifted by 2 pi where that helps); 0 if outside */
static int to_limits(const or_problem *pr, int k, double theta, double *q) {
    double v = wrap_angle(theta - pr->dh[4 * k + 3]);
    double lo = pr->qlim[2 * k], hi = pr->qlim[2 * k + 1];
    if (v < lo) v += 2.0 * PI;
    if (v > hi) v -= 2.0 * PI;
    *q = v;
    return v >= lo && v <= hi;
}

int or_ik_analytic(const or_problem *pr, const double target[16], double q6, double sol[8][7]) {
    const double *dh = pr->dh;
    const double d0 = dh[2], d2 = dh[10], a3 = dh[12], a4 = dh[16], d4 = dh[18];
    double Einv[16], F7[16], T6[16], T6i[16], F6[16];
    rigid_inverse(pr->ee, Einv);
    mat4_mul(target, Einv, F7);
    dh_transform(dh[24], dh[25], dh[26], dh[27] + q6, T6);
    rigid_inverse(T6, T6i);
    mat4_mul(F7, T6i, F6);
    double R6[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R6[3 * i + j] = F6[4 * i + j];
    const double v[3] = {-F6[3], -F6[7], d0 - F6[11]};            /* S - O6, world */
    double w[3];                                                /* S - O6, frame 6 */
    for (int i = 0; i < 3; ++i) w[i] = R6[i] * v[0] + R6[3 + i] * v[1] + R6[6 + i] * v[2];
    const double A = a3 * a4 + d2 * d4, Bs = d2 * a4 - a3 * d4, Rn = hypot(A, Bs);
    const double D = 0.5 * (dot3(v, v) - (a3 * a3 + d2 * d2 + a4 * a4 + d4 * d4));
    if (fabs(D) > Rn) return 0;                                 /* out of reach for this q6 */
    const double phi = atan2(Bs, A), c_3 = acos(D / Rn);
    const double rho = hypot(w[0], w[1]), psi = atan2(w[0], w[1]);
    int n = 0;
    for (int i3 = 0; i3 < 2; ++i3) {
        const double t3 = i3 == 0 ? phi + c_3 : phi - c_3;
        const double ux = -a3 * cos(t3) - d2 * sin(t3) - a4, uy = a3 * sin(t3) - d2 * cos(t3) - d4;
        if (fabs(uy) > rho) continue;
        const double c_5 = acos(uy / rho);
        for (int i5 = 0; i5 < 2; ++i5) {
            const double t5 = i5 == 0 ? psi + c_5 : psi - c_5;
            const double sg = ux < 0.0 ? -1.0 : 1.0;
            const double t4 = atan2(sg * w[2], sg * (cos(t5) * w[0] - sin(t5) * w[1]));
            double R34[9], R45[9], R56[9], R35[9], R36[9], R3[9];
            rot_xz(dh[13], t3, R34);
            rot_xz(dh[17], t4, R45);
            rot_xz(dh[21], t5, R56);
            mat3_mul(R34, R45, R35);
            mat3_mul(R35, R56, R36);
            mat3_mul_bt(R6, R36, R3);
            const double sb = hypot(R3[2], R3[5]);
            for (int sgn = 1; sgn >= -1; sgn -= 2) {
                double t0, t1, t2;
                if (sb < 1e-12) {                               /* t1 = 0: only t0 + t2 is fixed */
                    if (sgn < 0) break;
                    t0 = 0.0; t1 = atan2(0.0, R3[8]); t2 = atan2(R3[3], R3[0]);
                } else {
                    t1 = atan2(sgn * sb, R3[8]);
                    t0 = atan2(sgn * R3[5], sgn * R3[2]);
                    t2 = atan2(sgn * R3[7], -sgn * R3[6]);
                }
                const double th[6] = {t0, t1, t2, t3, t4, t5};
                double q[7];
                int ok = 1;
                for (int k = 0; k < 6 && ok; ++k) ok = to_limits(pr, k, th[k], &q[k]);
                if (!ok) continue;
                q[6] = q6;
                memcpy(sol[n++], q, sizeof q);
            }
        }
    }
    return n;
}

/* The in-limit analytic solution nearest to seed (squared joint distance) over the
 * candidate values of the last joint, first found on ties; 0 if there is none. */
int or_ik_select(const or_problem *pr, const double target[16], const double seed[7], const double *q6,
                 int n_q6, double q[7]) {
    double best = INFINITY;
    for (int c = 0; c < n_q6; ++c) {
        double sol[8][7];
        const int n = or_ik_analytic(pr, target, q6[c], sol);
        for (int i = 0; i < n; ++i) {
            double d = 0.0;
            for (int j = 0; j < 7; ++j) d += (sol[i][j] - seed[j]) * (sol[i][j] - seed[j]);
            if (d < best) { best = d; memcpy(q, sol[i], sizeof(double) * 7); }
        }
    }
    return best < INFINITY;
}

/* Candidate values of the last joint for one IK target: the seed's own value, then one
 * uniform draw in each of OR_IK_Q6 - 1 equal strips of its limit range, strip i taking
 * word i mod 4 of the Philox counter (8 c0 + i/4, particle, TAG_Q6, attempt). */
static void q6_candidates(const or_problem *pr, uint32_t c0, int particle, uint32_t attempt, double seed6,
                          double q6[OR_IK_Q6]) {
    const int n = OR_IK_Q6 - 1;
    uint32_t u[4 * ((OR_IK_Q6 + 2) / 4)];
    for (int w = 0; 4 * w < n; ++w) philox(pr, 8u * c0 + (uint32_t)w, (uint32_t)particle, TAG_Q6, attempt, u + 4 * w);
    const double lo = pr->qlim[12], hi = pr->qlim[13];
    q6[0] = seed6;
    for (int i = 0; i < n; ++i) q6[1 + i] = lo + (((double)i + or_u01(u[i])) / (double)n) * (hi - lo);
}

/* IK of one lift target: analytic (ik_mode 1) over the seed's and the stratified last-joint
 * values, else (ik_mode 0, or no in-limit analytic solution) damped least squares.
 * Returns 1 where the analytic solution was taken. */
static int lift_ik(const or_problem *pr, const double T[16], uint32_t c0, int particle, uint32_t attempt,
                   double *q) {
    double seed[7];
    perturbed_home(pr, c0, particle, TAG_IKSEED, attempt, 0.3, seed);
    if (pr->ik_mode == 1) {
        double q6[OR_IK_Q6];
        q6_candidates(pr, c0, particle, attempt, seed[6], q6);
        if (or_ik_select(pr, T, seed, q6, OR_IK_Q6, q)) return 1;
    }
    or_ik(pr, T, seed, q);
    return 0;
}

/* Lift (Sec. III-B): IK at the grasp of each block's initial pose and at its placement,
 * one intermediate waypoint per segment (q_home perturbed, standing in for a retract
 * configuration), then linear interpolation start -> via -> goal over the segment. */
void or_lift(const or_problem *pr, const double *place, int particle, uint32_t attempt, double *q) {
    or_lift_ex(pr, place, particle, attempt, q, NULL);
}

void or_lift_ex(const or_problem *pr, const double *place, int particle, uint32_t attempt, double *q,
                int32_t *analytic) {
    const int B = pr->B, S = pr->W - 1, p2p = pr->kind == OR_KIND_P2P;
    memcpy(q, pr->q_home, 7 * sizeof(double));
    for (int b = 0; b < B; ++b) {
        uint32_t k[4];
        philox(pr, (uint32_t)b, (uint32_t)particle, TAG_GRASP, attempt, k);
        double T[16];
        int how;
        grasp_target(pr, b, pr->init + 4 * b, (int)(k[0] & 3u), T);
        how = lift_ik(pr, T, (uint32_t)(2 * b), particle, attempt, q + 7 * t_grasp(pr, b));
        if (analytic) analytic[2 * b] = how;
        if (p2p) continue;   /* one segment: no placement */
        grasp_target(pr, b, place + 4 * b, (int)(k[1] & 3u), T);
        how = lift_ik(pr, T, (uint32_t)(2 * b + 1), particle, attempt, q + 7 * t_place(pr, b));
        if (analytic) analytic[2 * b + 1] = how;
    }
    int m = S / 2;
    for (int s = 0; s < (p2p ? 1 : 2 * B); ++s) {
        double via[7];
        perturbed_home(pr, (uint32_t)s, particle, TAG_VIA, attempt, 0.3, via);
        const double *qa = q + 7 * (s * S), *qb = q + 7 * ((s + 1) * S);
        for (int jj = 1; jj < S; ++jj) {
            double *qt = q + 7 * (s * S + jj);
            for (int j = 0; j < 7; ++j) {
                if (jj <= m) qt[j] = qa[j] + ((double)jj / m) * (via[j] - qa[j]);
                else qt[j] = via[j] + ((double)(jj - m) / (S - m)) * (qb[j] - via[j]);
            }
        }
    }
}

/* Gradient descent with the learning-rate schedule eta_k = eta_traj (1 - k/K) inside
 * the augmented Lagrangian: every K_al steps lambda_r += mu sqrt(w_r) h_r, mu = min(2 mu, mu_max).
 * q_home stays fixed; joints are clamped to their limits after each step.  lam is n x NR. */
void or_traj_descend(const or_problem *pr, int n, double *q, double *lam, double *mu, int k_steps) {
    const int C = or_n_configs(pr), NR = or_n_residuals(pr);
#pragma omp parallel for schedule(dynamic) num_threads(pr->n_threads > 0 ? pr->n_threads : 1)
    for (int p = 0; p < n; ++p) {
        double *qp = q + (size_t)7 * C * p;
        double *lp = lam + (size_t)NR * p;
        double *g = (double *)malloc(sizeof(double) * 7 * (size_t)C);
        double *h = (double *)malloc(sizeof(double) * (size_t)NR);
        for (int k = 1; k <= k_steps; ++k) {
            double eta = pr->eta_traj * (1.0 - (double)k / (double)k_steps);
            or_traj_cost(pr, qp, lp, mu[p], g, NULL, NULL, NULL, h);
            for (int t = 1; t < C; ++t)
                for (int j = 0; j < 7; ++j)
                    qp[7 * t + j] = clampd(qp[7 * t + j] - eta * g[7 * t + j], pr->qlim[2 * j], pr->qlim[2 * j + 1]);
            if (pr->K_al > 0 && k % pr->K_al == 0) {
                for (int r = 0; r < NR; ++r) lp[r] += mu[p] * sqrt(residual_weight(pr, r)) * h[r];
                mu[p] = mu[p] * 2.0 < pr->mu_max ? mu[p] * 2.0 : pr->mu_max;
            }
        }
        free(g); free(h);
    }
}

/* Stage 2 end to end: lift Q particles (particle p from placement p mod n_place), descend,
 * keep the satisfying ones ranked by their final cost; re-lift with the next attempt
 * counter if none satisfies, within max_steps gradient steps. */
int or_traj_solve(const or_problem *pr, const double *place, int n_place, double *out_q,
                  double *out_cost, int *n_found, int *attempts) {
    const int B = pr->B, C = or_n_configs(pr), Q = pr->Q;
    double *q = (double *)malloc(sizeof(double) * 7 * (size_t)C * Q);
    const int NR = or_n_residuals(pr);
    double *lam = (double *)malloc(sizeof(double) * NR * (size_t)Q);
    double *mu = (double *)malloc(sizeof(double) * (size_t)Q);
    double *cost = (double *)malloc(sizeof(double) * (size_t)Q);
    int32_t *slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)Q);
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)Q);
    int found = 0, a = 0, spent = 0;
    while (spent < pr->max_steps && n_place > 0) {
#pragma omp parallel for schedule(dynamic) num_threads(pr->n_threads > 0 ? pr->n_threads : 1)
        for (int p = 0; p < Q; ++p) or_lift(pr, place + (size_t)4 * B * (p % n_place), p, (uint32_t)a, q + (size_t)7 * C * p);
        for (int p = 0; p < Q; ++p) { mu[p] = pr->mu0; for (int r = 0; r < NR; ++r) lam[(size_t)NR * p + r] = 0.0; }
        or_traj_descend(pr, Q, q, lam, mu, pr->K_traj);
        spent += pr->K_traj;
        ++a;
        int ns = 0;
        for (int p = 0; p < Q; ++p)
            if (or_traj_check(pr, q + (size_t)7 * C * p, NULL)) {
                cost[ns] = or_traj_rank_cost(pr, q + (size_t)7 * C * p);
                slot[ns++] = p;
            }
        if (ns > 0) {
            or_argsort(ns, cost, ord);
            found = ns < pr->P ? ns : pr->P;
            for (int s = 0; s < found; ++s) {
                memcpy(out_q + (size_t)7 * C * s, q + (size_t)7 * C * slot[ord[s]], sizeof(double) * 7 * C);
                if (out_cost) out_cost[s] = cost[ord[s]];
            }
            break;
        }
    }
    if (n_found) *n_found = found;
    if (attempts) *attempts = a;
    free(q); free(lam); free(mu); free(cost); free(slot); free(ord);
    return found > 0;
}

/*
 * SPaSM hot path on one GPU: C ABI.
 *
 * Sequential pick-and-place with a fixed action skeleton (Sec. III of the paper: known
 * object geometry and initial poses, environment obstacles, a given order of pick-and-
 * place actions), solved in two stages:
 *   stage 1  object-placement CSP by particle optimisation (Alg. 1),
 *   stage 2  lift to joint space and trajectory optimisation of all waypoints and
 *            placements (Sec. III-B; cost terms of the appendix, tower stacking).
 *
 * Conventions for every entry point:
 *   - Returns SPASM_OK or a negative spasm_status; on error, spasm_last_error() gives a
 *     thread-local message.  No C++ exception crosses this boundary.
 *   - "host" pointers are CPU memory owned by the caller; "device" pointers are CUDA
 *     device memory owned by the caller, on the device current when the problem was
 *     created.  The library copies every input array given to spasm_create_problem;
 *     the caller keeps ownership of all pointers it passes.
 *   - Work is enqueued on the problem's CUDA stream (set at creation) and is
 *     asynchronous unless the function says it synchronises.
 *   - Calls on one problem handle are not thread-safe; distinct handles are.
 *   - Device errors (a bounded wait that gave up, a size outside the compiled limits)
 *     are recorded in a per-problem error word and reported as SPASM_ERR_DEVICE by the
 *     next synchronising call.
 *
 * Layouts (row-major, float32 on the device):
 *   stage-1 particles  x[4B][n]   (structure of arrays: row 4i+k, k = x, y, z, yaw of the
 *                                  block at stack position i; column = particle)
 *   stage-2 particles  q[n][C][8] (C = 2B(W-1)+1 configurations, 7 joints + 1 pad;
 *                                  q[.][0] = q_home)
 *   placements         [P][B][4]  (x, y, z, yaw per block, stack order)
 */
#ifndef SPASM_H
#define SPASM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spasm_problem* spasm_problem_t;

typedef enum {
    SPASM_OK = 0,
    SPASM_ERR_INVALID = -1,     /* bad argument, size beyond the compiled limits */
    SPASM_ERR_NOMEM = -2,       /* device allocation failed */
    SPASM_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    SPASM_ERR_NOSOLUTION = -4,  /* no satisfying particle within max_steps (Sec. IV-C cap) */
    SPASM_ERR_TIMEOUT = -5,     /* reserved for bounded host waits */
    SPASM_ERR_DEVICE = -6,      /* a kernel recorded an error (see spasm_last_error) */
    SPASM_ERR_CANCELLED = -7    /* a service request cancelled by the caller */
} spasm_status;

/* Robot (Sec. III: the manipulator as a collection of spheres; fk of a 7-R arm, appendix).
 * dh: 7 x 4 modified-DH rows (a, alpha, d, theta_offset), joint k transform
 *     Rot_x(alpha) Trans_x(a) Rot_z(theta_offset + q_k) Trans_z(d);
 * qlim: 7 x 2 (lower, upper); sphere: n_spheres x 4 (x, y, z, r) in the frame of link
 * sphere_link[i] (0 = base, k = link k); ee: 4 x 4 flange -> tool transform; q_home: 7. */
typedef struct {
    int dof;                     /* must be 7 */
    const double* dh;
    const double* qlim;
    int n_spheres;               /* <= 56 */
    const int32_t* sphere_link;
    const double* sphere;
    const double* ee;
    const double* q_home;
} spasm_robot;

/* Environment (Sec. III; Pen(.,.) of the appendix): cuboids n x 15 = centre (3), rotation
 * (9, row-major), half extents (3); spheres n x 4 = centre (3), radius. */
typedef struct {
    int n_cuboids;               /* <= 256 */
    const double* cuboid;
    int n_spheres;               /* <= 64 */
    const double* sphere;
} spasm_obstacles;

/* Goal and action skeleton (Sec. III; tower stacking, appendix).  Blocks are given in
 * stack order (bottom first): block i is picked i-th and placed at stack position i.
 * half_ext: B x 3; init_pose: B x 4 (x, y, z, yaw); goal_box: 6 = lo (3), hi (3) bounds
 * of the placed block centres; z_table: table top height; grasp_off: tool standoff above
 * a block's top face. */
typedef struct {
    int n_blocks;                /* 1..16 */
    const double* half_ext;
    const double* init_pose;
    const double* goal_box;
    double z_table;
    double grasp_off;
} spasm_goal;

/* Packing goal (the appendix's Tetris problem): block i is a polyomino of n_cells[i] unit
 * cubes of edge cell_size, centred at the offsets cell[2k], cell[2k+1] (k over the block's
 * cells, in block order) in its frame, the frame origin being the point the block pose
 * (x, y, z, yaw) places.  The blocks are packed into region = (x_lo, y_lo, x_hi, y_hi)
 * between four walls (slabs of thickness and height cell_size just outside the region,
 * centred at height z_star) at the resting height z_star; block origins are clamped to the
 * region in x, y and to [z_star, z_star + z_span] in z (0: one tight layer).  Cost of a
 * placement: w_coll (sum over block pairs i < j of the penetration of block j's spheres
 * into block i's cubes + sum over blocks and walls) + w_height sum |z_i - z_star|, each cube
 * carrying 8 spheres of radius cell_size/4 at (+-cell_size/4, +-cell_size/4, +-cell_size/4). */
typedef struct {
    int n_blocks;                /* 1..16 */
    const int32_t* n_cells;      /* B: 1..8 each, at most 64 in total */
    const double* cell;          /* sum(n_cells) x 2 */
    double cell_size;
    const double* region;        /* 4 */
    double z_star;
    double z_span;               /* >= 0 */
} spasm_packing;

/* Solver parameters (Alg. 1 and Sec. III-B): N sample / M optimised particles, P
 * returned solutions, Q trajectory particles, W waypoints per motion segment, step
 * counts, learning rates, weights of the appendix cost terms, augmented-Lagrangian
 * penalty schedule, IK iterations/damping, Philox seed, the cap on total gradient
 * steps (30 000 in the paper's experiments, Sec. IV-C), and the lift's IK:
 *   ik_mode 0: damped least squares (K_ik iterations, ik_damp) from a perturbed home seed;
 *   ik_mode 1: analytic IK of the Franka joint layout (the paper lifts with an analytic
 *              Franka IK, Sec. III-B): the last joint takes the seed's value and one draw
 *              in each of 31 equal strips of its limit range, every in-limit branch (up to
 *              8 per value) is solved in closed form and the one nearest the seed is kept;
 *              targets without one fall back to damped least squares.  Needs twists (0, -pi/2, pi/2, pi/2, -pi/2,
 *              pi/2, pi/2) and a_0 = a_1 = a_2 = a_5 = d_1 = d_3 = d_5 = d_6 = 0, else
 *              create returns SPASM_ERR_INVALID. */
typedef struct {
    int N, M, P, Q, W;
    int K_lin, K_quad, K_traj, K_al, K_ik;
    double eta_init, alpha, eta_traj, eps, eps_start;
    double w_stable, w_height, w_coll, w_start, w_arm, w_block, w_path, w_jl;
    double mu0, mu_max, ik_damp;
    uint64_t seed;
    int max_steps;
    int ik_mode;
} spasm_params;

/* Validate and copy the problem to the device and allocate its working memory.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  Limits: B <= 16, W >= 3,
 * C <= 1024, N <= 32768, M <= 8192, P <= M, Q >= 1.  Synchronises once. */
spasm_status spasm_create_problem(const spasm_robot* robot, const spasm_obstacles* obstacles, const spasm_goal* goal,
                                  const spasm_params* params, void* cuda_stream, spasm_problem_t* out);
/* Device memory, in bytes, that spasm_create_problem would allocate for this problem (the
 * same buffer list, each rounded up to the pool's 512-byte granule); robot arrays do not
 * matter.  The solver service admits requests against its budget with this figure. */
spasm_status spasm_problem_bytes(const spasm_obstacles* obstacles, const spasm_goal* goal, const spasm_params* params,
                                 long long* bytes);
/* A packing problem (the appendix's Tetris problem) for stage 1 (spasm_place, the
 * kernel-level stage-1 entry points); the robot is validated and kept as for
 * spasm_create_problem, and spasm_optimize reports SPASM_ERR_INVALID (stage 2 is built for
 * the tower goal).  Limits as spasm_create_problem plus those of spasm_packing. */
spasm_status spasm_create_packing(const spasm_robot* robot, const spasm_packing* packing, const spasm_params* params,
                                  void* cuda_stream, spasm_problem_t* out);
/* Point-to-point trajectory optimisation (the paper's motion-planning use of stage 2, Sec.
 * IV): one transit segment of W configurations from q_home to a configuration whose tool,
 * pointing down (tool z along -world z), reaches target = (x, y, z, yaw); the yaw is free
 * up to quarter turns (the lift draws one).  The objective is that of stage 2 with the
 * target-alignment residuals (tool position, roll, pitch) and the arm-collision group,
 * without placement, held block or stage 1 (spasm_place reports SPASM_ERR_INVALID).
 * spasm_optimize, spasm_result (C = W) and spasm_optimize_batch apply.  Limits as
 * spasm_create_problem. */
spasm_status spasm_create_p2p(const spasm_robot* robot, const spasm_obstacles* obstacles, const double* target,
                              const spasm_params* params, void* cuda_stream, spasm_problem_t* out);
/* Stage-1 result: *n_place satisfying placements found (0 before spasm_place), placements
 * P x B x 4 (x, y, z, yaw), best first.  SPASM_ERR_NOSOLUTION when none.  Synchronises. */
spasm_status spasm_placements(spasm_problem_t problem, int* n_place, double* placements);
spasm_status spasm_destroy_problem(spasm_problem_t problem);
const char* spasm_last_error(void);

/* Stage 1, Alg. 1 with re-initialisation until a satisfying particle exists or max_steps
 * gradient steps are spent (Sec. III-A, the cap of Sec. IV-C).  Enqueues and returns: the
 * attempt loop runs on the device (a CUDA graph whose conditional while node repeats an
 * attempt while no particle satisfies), and the host does not wait for it.  The best P
 * placements stay on the device for stage 2; spasm_placements reads them.  The graphs of
 * both stages are built when the problem is created (they read the seed from device memory,
 * so spasm_set_seed keeps them).
 * SPASM_ERR_NOSOLUTION, when no attempt satisfies, is reported by spasm_placements /
 * spasm_result. */
spasm_status spasm_place(spasm_problem_t problem);

/* Stage 2: lift the stage-1 placements to Q trajectory particles, optimise, keep the
 * satisfying ones (re-lifting with the next Philox attempt while none does, within
 * max_steps), FP64-check the best P.  Enqueues stage 1 first if it has not run.  Like
 * spasm_place it enqueues one graph with a device-side attempt loop and returns without
 * waiting; the outcome (including SPASM_ERR_NOSOLUTION) is read by spasm_result. */
spasm_status spasm_optimize(spasm_problem_t problem);

/* Launch mode of spasm_place / spasm_optimize.  SPASM_LAUNCH_GRAPH (the default): each stage
 * is one CUDA graph whose attempt loop is a conditional while node.  SPASM_LAUNCH_EAGER: the
 * same kernels with the same arguments in the same order, launched one at a time on the
 * problem's stream, the attempt loop on the host, which reads the loop decision after every
 * attempt (one wait each: the calls return once the last attempt is enqueued); the results
 * are the same bits.  It serves tools that cannot look inside graphs with conditional nodes
 * (kernel profilers).  spasm_optimize_batch and the service always use graphs.  Completes the
 * pending stages first.  SPASM_ERR_INVALID for another mode. */
#define SPASM_LAUNCH_GRAPH 0
#define SPASM_LAUNCH_EAGER 1
spasm_status spasm_set_launch_mode(spasm_problem_t problem, int mode);

/* Copy results to host memory (synchronises: the one host wait of a solve).  Any output
 * pointer may be NULL.
 * n_found: number of returned solutions (<= P); placements: P x B x 4;
 * traj: P x C x 7; cost: P (ranking cost, ascending); success: P (1 if the solution
 * passes the FP64 re-evaluation of every penetration, the grasp and tilt errors, the
 * placement conditions and the joint limits). 
 * Returns SPASM_ERR_NOSOLUTION if stage 2 found nothing. */
spasm_status spasm_result(spasm_problem_t problem, int* n_found, double* placements, double* traj, double* cost,
                          int* success);

/* Sizes of this problem: configurations C per trajectory particle and residuals NR of the
 * augmented Lagrangian (9B + 3). */
spasm_status spasm_sizes(spasm_problem_t problem, int* C, int* NR);

/* ---- kernel-level entry points (device pointers; used by parity tests and autograd) ---- */

/* Alg. 1 SampleUniform + Cost: n particles from Philox counter (block, particle, 0,
 * attempt); x (device, 4B x n SoA, written), cost (device, n, linear form). */
spasm_status spasm_place_sample(spasm_problem_t problem, int n, uint32_t attempt, float* x, float* cost);

/* Placement cost of n particles (linear form, or quadratic when quadratic != 0) and its
 * gradient.  x: device 4B x n; cost: device n; grad: device 4B x n or NULL; metrics:
 * device n x 3 (largest penetration, CoM distance, height error) or NULL; terms: device
 * n x 3 (C_stable, C_height, C_coll) or NULL. */
spasm_status spasm_place_eval(spasm_problem_t problem, int n, const float* x, int quadratic, float* cost, float* grad,
                              float* metrics, float* terms);

/* Alg. 1 descent on n particles in place (device x, 4B x n): k_lin linear steps with
 * eta_init (1 - k/k_lin), k_quad quadratic steps with alpha, box projection after each.
 * cost: device n (final quadratic cost) or NULL; sat: device n (GetSatisfyingParticles)
 * or NULL. */
spasm_status spasm_place_descend(spasm_problem_t problem, int n, float* x, int k_lin, int k_quad, float* cost,
                                 int* sat);

/* ArgSort(cost)[:k]: the k smallest of n costs by (cost, index); NaN last.  cost: device n;
 * idx: device k (written); n <= 32768, k <= 8192. */
spasm_status spasm_select_topk(spasm_problem_t problem, int n, const float* cost, int k, int* idx);

/* Lift (Sec. III-B): n trajectory particles from placements (device, n_place x B x 4):
 * particle p uses placement p mod n_place; IK at each grasp and placement, one
 * intermediate waypoint per segment, linear interpolation.  q: device n x C x 8. */
spasm_status spasm_lift(spasm_problem_t problem, int n, const float* placements, int n_place, uint32_t attempt,
                        float* q);

/* Augmented-Lagrangian objective of n trajectory particles and its gradient.
 * q: device n x C x 8; lam: device n x NR or NULL (zeros); mu: device n or NULL (mu0);
 * L: device n; grad: device n x C x 8 or NULL; groups: device n x 6 (C_start, C_arm,
 * C_block, C_coll, C_stable, C_height) or NULL; h: device n x NR residuals or NULL. */
spasm_status spasm_traj_eval(spasm_problem_t problem, int n, const float* q, const float* lam, const float* mu,
                             float* L, float* grad, float* groups, float* h);

/* k_steps of gradient descent with eta_traj (1 - k/k_steps) inside the augmented
 * Lagrangian (multiplier update every K_al steps), in place on q (device n x C x 8);
 * lam (n x NR) and mu (n) are read and written; when init_multipliers != 0 they start at
 * 0 and mu0.  metrics: device n x 8 or NULL; sat: device n or NULL (final check). */
spasm_status spasm_traj_descend(spasm_problem_t problem, int n, float* q, float* lam, float* mu, int k_steps,
                                int init_multipliers, float* metrics, int* sat);

/* FP64 final check (GetSatisfyingParticles of Alg. 1 applied to returned solutions, Sec.
 * III; the check spasm_optimize runs on the best P) of n caller-given trajectories.
 * q: device n x C x 8 floats (joints 0..6 of each configuration; q[.][0] is taken as
 * given).  metrics: device n x 6 doubles, written: largest arm / held-block penetration
 * over all configurations, largest grasp alignment (squared position error + roll^2 +
 * pitch^2 at the grasp configurations), largest placement tilt (roll^2 + pitch^2), and on
 * the placed blocks (fk of the place configurations): largest penetration, largest CoM
 * distance, largest height error.  ok: device n ints, 1 where every penetration, CoM
 * distance and height error is <= eps, the alignment and tilt <= eps_start and every joint
 * within its limits (the limits rounded to float32, as the FP32 optimiser holds them).
 * Evaluated in double precision from the float32 joint values. */
spasm_status spasm_traj_check(spasm_problem_t problem, int n, const float* q, double* metrics, int* ok);

/* Stage-1 sampling and elite selection that allocates no device memory (the paper has no
 * counterpart: this serves callers that cannot allocate while they plan, such as a planner
 * in a real-time control loop that must not stall on cudaMalloc, or a plug-in in a
 * framework that owns all device memory).  Same result as spasm_place_sample(n, attempt)
 * followed by spasm_select_topk(m) and a gather: x_elite (device, 4B x m SoA) receives the
 * m lowest-cost particles in ascending (cost, index) order and cost_elite (device, m) their
 * linear-form costs.  Intermediates live in one fixed 4 MiB device array of the library:
 * 4B*n + n + m floats must fit (else SPASM_ERR_INVALID), n <= 32768, m <= 8192.  The first
 * call on a device is its set-up: it looks the array up, which may load the library's device
 * code and create the array (so that call may allocate and synchronise); make it before any
 * stream capture.  Later calls allocate nothing.  Calls share the array, so calls that
 * overlap on the GPU race and must be serialised by the caller. */
spasm_status spasm_place_select_static(spasm_problem_t problem, int n, uint32_t attempt, int m, float* x_elite,
                                       float* cost_elite);

/* ---- checkpoint / resume (not in the paper: bookkeeping of this library) ----
 * A snapshot holds a problem's search state as its last completed stage left it: the Philox
 * key, the attempt and step counters of both stages, the stage-1 outcome (count and the best
 * P placements) and the returned solutions (count, P x C configurations, ranking costs, FP64
 * success flags), behind a header with the problem's kind and sizes, a digest of its
 * obstacle set and a digest of the payload.  The trajectory particles themselves are not
 * kept.  spasm_snapshot_bytes gives the size for this problem.  spasm_snapshot writes one to
 * caller memory (host, at least that many bytes; completes the pending stages first and
 * synchronises).  spasm_restore loads one into a problem created from the same inputs (the
 * library checks the kind, the sizes and the obstacle digest; SPASM_ERR_INVALID otherwise, and
 * for a truncated or corrupted snapshot, leaving the problem as it was); afterwards
 * spasm_placements / spasm_result return what the snapshotted problem returned, and after a
 * snapshot taken between the stages spasm_optimize runs stage 2 only, from the restored
 * placements with the restored key, and returns the solutions the uninterrupted solve
 * returns.  Synchronises. */
spasm_status spasm_snapshot_bytes(spasm_problem_t problem, size_t* bytes);
spasm_status spasm_snapshot(spasm_problem_t problem, void* host, size_t bytes);
spasm_status spasm_restore(spasm_problem_t problem, const void* host, size_t bytes);

/* ---- run control and statistics (not in the paper: bookkeeping of this library) ---- */

/* Counters and device times of the spasm_place / spasm_optimize calls since the last
 * reset.  Times are CUDA-event durations on the problem's stream and are filled only
 * while timing is enabled.  Reading them synchronises the problem's stream when a solve's
 * outcome has not been read yet. */
typedef struct {
    int place_attempts;        /* Alg. 1 attempts (re-initialisations + 1) */
    int traj_attempts;         /* stage-2 lift + descent attempts */
    int n_found;               /* solutions returned */
    int n_success;             /* of those, passing the FP64 check */
    long long kernel_launches; /* kernels launched by spasm_place / spasm_optimize */
    int traj_launches;         /* launches of the fused trajectory-descent kernel */
    long long particle_iters;  /* stage-2 particle-iterations executed (Q x K_traj x attempts) */
    double ms_place;           /* stage 1, all attempts */
    double ms_lift;            /* stage-2 lifts */
    double ms_traj;            /* fused trajectory-descent kernels */
    double ms_finish;          /* ranking, selection and FP64 check */
    long long h2d_bytes;       /* host -> device bytes copied by create / place / optimize */
    long long d2h_bytes;       /* device -> host bytes copied by place / optimize / result */
    long long tests_executed;  /* sphere-obstacle tests run by the trajectory kernels after the
                                  exact box cull (pairs whose boxes are disjoint are skipped) */
    long long cull_configs;    /* configurations whose kinematics and cull the trajectory kernels
                                  ran (the others kept a candidate-free cull from an earlier
                                  iteration, valid while they moved less than its clearance) */
    long long cand_configs;    /* of those, configurations with a candidate obstacle, whose sphere
                                  centres, tests and gradient chain ran */
    double ms_retry;           /* stage-2 attempts after the first (re-lift and descent), and the
                                  satisfying selection; ms_lift and ms_traj time the first */
    long long host_waits;      /* times the library made the host wait for the problem's stream
                                  (spasm_place and spasm_optimize never do; the first of
                                  spasm_result, spasm_placements and spasm_get_stats after a solve
                                  waits once to read its outcome) */
} spasm_stats;

/* Measured FP32 fused-multiply-add throughput of the current device (not in the paper: the
 * roofline denominator of the trajectory kernels, which are FP32 ALU work).  Runs a kernel of
 * independent FMA chains filling every SM (8 CTAs of 256 threads each) for about target_ms
 * (0 < target_ms <= 10000) on the legacy default stream and returns *tflops = 2 x FMAs /
 * CUDA-event time; *ms and *flop (may be NULL) receive the time and the flop count.  Allocates
 * and frees a small device buffer; synchronises the device's default stream. */
spasm_status spasm_fp32_fma_peak(double target_ms, double* tflops, double* ms, double* flop);

/* Wait for the problem's stream and report what its kernels recorded: SPASM_ERR_DEVICE when a
 * bounded device wait gave up or a kernel rejected its sizes (the error word is sticky: every
 * later synchronising call of this problem reports it again), else SPASM_OK. */
spasm_status spasm_synchronize(spasm_problem_t problem);

/* ---- fault injection for tests (not in the paper: exercises the failure paths without a GPU
 * fault) ----
 * spasm_inject_wait_timeout enqueues on the problem's stream one CTA that waits, with the
 * bounded wait of the kernels' table staging, on an mbarrier whose expected bytes no copy
 * delivers (no copy is issued: nothing is left in flight); after max_polls polls
 * (1..2^22) it records the timeout in the problem's error word and returns, and the next
 * synchronising call reports SPASM_ERR_DEVICE.  spasm_inject_alloc_failure makes the nth
 * device allocation of the library from now on (0: the next one) fail as if
 * cudaMallocAsync had failed (SPASM_ERR_NOMEM); -1 turns the injection off.  The injection
 * is process-wide and one-shot. */
spasm_status spasm_inject_wait_timeout(spasm_problem_t problem, int max_polls);
spasm_status spasm_inject_alloc_failure(int nth);

/* Launch shape of the trajectory kernels (not in the paper: the tiling choices the autotuner
 * searches).  sphere_tiling: how a warp's lanes hold the (up to 64) sphere items of a
 * configuration, 0 strided (lane L holds items L and L + 32), 1 blocked (items 2L and 2L + 1);
 * particles_per_cta: particles one CTA optimises at once, 1 (8 warps) or 2 (16 warps, each
 * particle on its own 8 warps and shared-memory region; needs twice the shared memory).  The
 * tiling reorders sums of the same terms (results agree to float32 rounding); the particles
 * per CTA change nothing in a particle's arithmetic. */
typedef struct {
    int sphere_tiling;
    int particles_per_cta;
} spasm_kernel_config;
/* Sets the launch shape of the problem's trajectory kernels (spasm_optimize and the
 * kernel-level trajectory calls) and rebuilds its stage graphs; SPASM_ERR_INVALID for values
 * outside the above or two particles whose shared memory does not fit one CTA.  Synchronises. */
spasm_status spasm_set_kernel_config(spasm_problem_t problem, const spasm_kernel_config* cfg);

/* Resident CTAs per SM of this problem's trajectory kernels under its launch shape: *single for
 * the per-problem kernel of spasm_optimize, *batched for the batched kernel of
 * spasm_optimize_batch in a batch whose largest problem is this one (CUDA's occupancy
 * calculator with the shared memory the launches request; 0 where they do not fit).  Not in
 * the paper: what a caller sizing batches, and a test guarding the shared-memory budget,
 * read. */
spasm_status spasm_traj_residency(spasm_problem_t problem, int* single, int* batched);

/* Replace the Philox seed (the key of every random stream) and forget previous results;
 * the next spasm_optimize re-runs both stages. */
spasm_status spasm_set_seed(spasm_problem_t problem, uint64_t seed);
/* Enable (1) or disable (0) CUDA-event timing of the phases. */
spasm_status spasm_set_timing(spasm_problem_t problem, int enable);
/* Copy the statistics (host struct); spasm_reset_stats zeroes them. */
spasm_status spasm_get_stats(spasm_problem_t problem, spasm_stats* out);
spasm_status spasm_reset_stats(spasm_problem_t problem);

/* ---- batched form (not in the paper: the throughput form of the hot path for many
 * independent problems; the per-particle computation is that of Alg. 1 and Sec. IV as in
 * spasm_optimize) ----
 * spasm_optimize_batch solves n problems together on `cuda_stream`, which must be a created
 * stream (not the legacy default stream: the batch is captured as CUDA graphs).  The first
 * attempt of stage 1 of every problem not yet placed runs as one graph; stage 2 of every
 * placed problem (lift, one persistent launch of the trajectory kernel over the particles
 * of all problems, selection, FP64 check) runs as a second graph.  A problem that needs
 * further attempts continues alone on its own stream, as spasm_optimize would.  Each
 * problem's outcome is then read with spasm_result, and equals what spasm_optimize gives
 * (the same arithmetic for every particle, whatever the schedule).  Returns SPASM_OK unless
 * an argument is invalid or a CUDA call fails; a problem without a solution reports
 * SPASM_ERR_NOSOLUTION from spasm_result.  Every problem's own stream is synchronised
 * first, and the problems must not be used by another thread during the call.
 * The schedule of the persistent launch: */
typedef struct {
    int per_fetch;     /* particles per work item a group takes from the shared counter (1..64) */
    int ctas_per_sm;   /* resident CTAs per SM (0: as many as fit) */
    int order;         /* 0: the largest problem (particles x configurations) first, 1: as given */
    int sphere_tiling;       /* 0 strided, 1 blocked (see spasm_kernel_config) */
    int particles_per_cta;   /* 1 or 2 (see spasm_kernel_config) */
} spasm_batch_config;
/* per_fetch 1, ctas_per_sm 0, order 0, sphere_tiling 0, particles_per_cta 1. */
spasm_status spasm_batch_default_config(spasm_batch_config* cfg);
/* cfg NULL: the default schedule. */
spasm_status spasm_optimize_batch(spasm_problem_t* problems, int n, void* cuda_stream, const spasm_batch_config* cfg);
/* Autotuner of the batched launch: places the problems not yet placed (stage 1, as above),
 * lifts them, times each trajectory shape (sphere tiling in {strided, blocked} x particles per
 * CTA in {1, 2}, where its shared memory fits) over one full descent of every particle, then,
 * under the fastest shape, one evaluation of every particle per schedule (per_fetch in
 * {1, 2, 4} x ctas_per_sm in {all, 1} x both orders; CUDA events, the better of two runs), and
 * returns the fastest in *best (and that schedule's evaluation time in *best_ms when not
 * NULL).  The tuning writes only buffers a solve sets again (the particles are lifted again
 * and the multipliers start fresh).  The schedule and the particles per CTA change no result;
 * the sphere tiling changes results at float32 rounding. */
spasm_status spasm_batch_autotune(spasm_problem_t* problems, int n, void* cuda_stream, spasm_batch_config* best,
                                  double* best_ms);

/* ---- solver service with continuous batching (not in the paper: the serving form of the
 * hot path) ----
 * Requests are whole problems (copied at submission).  One scheduler thread runs the device
 * work in epochs, each one trajectory attempt of every request in flight: queued requests are
 * admitted in arrival order while fewer than max_inflight are in flight and their device
 * memory (spasm_problem_bytes) fits budget_bytes (a request larger than the whole budget is
 * admitted when nothing else is in flight), created on the scheduler's stream of the device
 * current at creation, and their stage 1 runs (with its device-side attempt loop); then one
 * persistent launch of the trajectory kernel runs the descent of the particles of every
 * request in flight, followed per request by its satisfying selection, its attempt decision
 * and the FP64 check; requests that finished retire, the others re-lift with their next
 * attempt counter for the next epoch.  A request that arrives during an epoch joins at the
 * next one.  Each request's result is the one spasm_optimize gives for it, whatever else is in
 * flight.  Results stay with the server until spasm_server_release. */
typedef struct spasm_server* spasm_server_t;
/* Counters of a server: epochs run, requests and particles summed over epochs (their means
 * are the batch sizes), requests completed, device bytes of the requests in flight. */
typedef struct {
    long long epochs;
    long long requests_in_epochs;
    long long particles_in_epochs;
    long long completed;
    long long bytes_in_use;
} spasm_server_stats;
spasm_status spasm_server_create(long long budget_bytes, int max_inflight, spasm_server_t* out);
/* Validates sizes on the host (SPASM_ERR_INVALID) and queues; *ticket identifies the request. */
spasm_status spasm_server_submit(spasm_server_t server, const spasm_robot* robot, const spasm_obstacles* obstacles,
                                 const spasm_goal* goal, const spasm_params* params, long long* ticket);
/* *state = 0 queued, 1 running, 2 done, 3 cancelled. */
spasm_status spasm_server_poll(spasm_server_t server, long long ticket, int* state);
/* Bounded wait for completion: SPASM_ERR_TIMEOUT after timeout_s seconds. */
spasm_status spasm_server_wait(spasm_server_t server, long long ticket, double timeout_s);
/* Outputs of a finished request (host buffers sized as for spasm_result; any may be NULL);
 * *status is the request's own status; latency_ms = submission to completion, queue_ms =
 * submission to admission.  SPASM_ERR_TIMEOUT if it has not finished. */
spasm_status spasm_server_result(spasm_server_t server, long long ticket, int* status, int* n_found,
                                 double* placements, double* traj, double* cost, int* success, double* latency_ms,
                                 double* queue_ms);
spasm_status spasm_server_release(spasm_server_t server, long long ticket);
/* Cancel a request: a queued one at once (state 3), one in flight at the next epoch boundary
 * (its device memory is returned then); its status becomes SPASM_ERR_CANCELLED.  Finished
 * requests are not affected. */
spasm_status spasm_server_cancel(spasm_server_t server, long long ticket);
spasm_status spasm_server_get_stats(spasm_server_t server, spasm_server_stats* out);
/* Finishes the queued and running requests, then joins the slots. */
spasm_status spasm_server_destroy(spasm_server_t server);

#ifdef __cplusplus
}
#endif
#endif

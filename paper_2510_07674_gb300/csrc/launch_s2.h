// Host-side launchers of the stage-2 kernels (internal to the library).
#pragma once
#include "launch.h"

namespace spasm {

// Buffers of one trajectory-kernel launch (device pointers; any may be null unless noted).
struct TrajIO {
    float* q;          // [n][C][8] joint configurations (required); updated by a descent
    float* lam;        // [n][NR] multipliers
    float* mu;         // [n] penalty parameters
    float* L;          // [n] augmented-Lagrangian objective
    float* grad;       // [n][C][8] dL/dq (evaluation mode)
    float* groups;     // [n][6] C_start, C_arm, C_block, C_coll, C_stable, C_height
    float* h;          // [n][NR] residual vector
    float* metrics;    // [n][8] max pen, max grasp error, max tilt, placement max pen / CoM / height, path, rank cost
    int* sat;          // [n] satisfying flag
    unsigned long long* tests;   // [0] sphere-obstacle tests executed (after the exact cull), [1]
                                 // configurations whose kinematics and cull ran, [2] of those, the
                                 // ones with a candidate obstacle (sphere-level work); accumulated
    int k_steps;       // descent steps
    int init_multipliers;   // descent starts from lambda = 0, mu = mu0
    const int* active;  // optional device word: when it holds 0 or less the launch does nothing (the
                        // trajectory stage of a problem whose stage 1 found no placement)
};
enum TrajModeHost { kTrajModeEval = 0, kTrajModeDescend = 1, kTrajModeCheck = 2 };

// One problem of a batched trajectory launch (device array, sorted by `first`).
struct TrajJob {
    const Scalars* sc;   // device copy of the problem constants
    DevTables tab;
    TrajIO io;
    int* err;
    int n;               // particles
    int first;           // index of the problem's first work item
};

size_t traj_smem_bytes(const Scalars& sc);
// IK at grasp/place poses + interpolation; particle p lifts placement p % n_place.  With
// ctl != nullptr the attempt counter, the placement count and the Philox key are read on the
// device (ctl->t_attempt, ctl->n_place, ctl->seed) in place of `attempt`, `n_place` and
// sc.seed, and the launch writes nothing when ctl->n_place is 0.
cudaError_t launch_lift(const Scalars& sc, int n, const float* place, int n_place, uint32_t attempt, float* q,
                        cudaStream_t st, const LoopCtl* ctl = nullptr);
cudaError_t launch_traj(const Scalars& sc, DevTables t, int n, int mode, const TrajIO& io, int* err, cudaStream_t st);
// Persistent batched launch over jobs[0..n_jobs) (n_items work items of per_fetch particles;
// *next must be 0); smem_bytes = the largest traj_smem_bytes of the jobs.
// tiling, ppc: the sphere tiling (Scalars::sphere_tiling) and the particles per CTA
// (Scalars::particles_per_cta) of the launch, the same for every job.
cudaError_t launch_traj_batch(const TrajJob* jobs, int n_jobs, int n_items, int per_fetch, int mode, int* next,
                              size_t smem_bytes, int grid, cudaStream_t st, int tiling = 0, int ppc = 1);
// Resident CTAs per SM of the batched kernel at that per-particle shared-memory size (0 on error
// or when it does not fit).
int traj_batch_ctas_per_sm(size_t smem_bytes, int tiling = 0, int ppc = 1);
// Resident CTAs per SM of the per-problem trajectory kernel for this problem's sizes and launch
// shape (0 if it does not fit).
int traj_ctas_per_sm(const Scalars& sc);
// Dynamic shared memory of one trajectory CTA with ppc particles.
size_t traj_cta_smem_bytes(const Scalars& sc, int ppc);

}  // namespace spasm

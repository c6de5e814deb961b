// FP64 feasibility check of returned trajectories (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace spasm {

// Double-precision copy of the problem tables used by the final check.
struct Scalars64 {
    int B, S, C, n_rsph, n_cub, n_osph;
    double ca[7], sa[7], a[7], d[7], th0[7], qlo[7], qhi[7];
    double ee_R[9], ee_p[3];
    double rsph[kMaxRobotSpheres][4];
    int rlink[kMaxRobotSpheres];
    double half[kMaxB][3], hmin[kMaxB], init[kMaxB][4], zt[kMaxB];
    double grasp_off, eps, eps_start;
    int p2p;   // point to point: one segment, no placement
};

// Per-solution accumulator of the split check (zeroed once at allocation; the check leaves it
// zeroed).
struct CheckAcc {
    unsigned long long mp;   // largest arm / held-block penetration (bit pattern of a non-negative double)
    double pp, ms, mt, mD, mz;
    int viol;                // a joint outside its limits
    int count;               // slices done
};

// cub: n_cub x 4 x double4 (centre, then R columns with half extents); osph: n_osph x double4.
// q: P x C x 8 floats; n_sol: device count of the rows that hold solutions (rows from
// min(*n_sol, P) on get ok = 0 and keep their metrics), or nullptr when all P rows do.
// metrics: P x 6 (max arm/held penetration, max grasp error, max tilt, placement max
// penetration, max CoM distance, max height error); ok: P flags.
cudaError_t launch_check64(const Scalars64& s, const void* cub, const void* osph, const float* q, const int* n_sol, int P,
                           double* metrics, int* ok, CheckAcc* acc, cudaStream_t st);

}  // namespace spasm

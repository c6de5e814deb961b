// Host-side launchers of the SPaSM kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace spasm {

struct DevTables {
    const float4* cub;    // n_cub x 4 float4 (environment cuboids)
    const float4* osph;   // n_osph float4 (environment spheres)
};

// Device-side state of the two stages' re-initialisation loops (Alg. 1 restarts until a
// particle satisfies, Sec. III-A; at most max_steps gradient steps, Sec. IV-C).  The
// attempt counters are the Philox counters of the next attempt's draws.
struct LoopCtl {
    uint32_t attempt;     // stage 1: attempts done
    int steps;            // stage 1: gradient steps spent
    int n_place;          // satisfying placements kept, min(count, P); 0 until stage 1 ends
    int more;             // stage 1 run attempt by attempt from the host (the eager launch mode): 1 while
                          // another attempt is due
    uint32_t t_attempt;   // stage 2: attempts done
    int t_steps;          // stage 2: gradient steps spent
    int found;            // stage 2: solutions kept, min(count, P); 0 until stage 2 ends
    int t_more;           // stage 2 run attempt by attempt from the host (the service, the eager mode): 1 while
                          // another attempt is due
    uint64_t seed;        // the Philox key of both stages' draws (the problem's seed)
};

// ---- stage 1 ----
// SampleUniform + Cost (linear form) for n particles; x is SoA [4B][n].
// ctl (optional): the attempt counter and the Philox key are read from ctl->attempt and
// ctl->seed on the device in place of `attempt` and sc.seed (the attempt loop runs there).
cudaError_t launch_place_sample_cost(const Scalars& sc, DevTables t, int n, uint32_t attempt, float* x, float* cost,
                                     int* err, cudaStream_t st, const LoopCtl* ctl = nullptr);
// Cost (linear or quadratic) and optional gradient / metrics / terms for n particles (SoA [4B][n]).
cudaError_t launch_place_eval(const Scalars& sc, DevTables t, int n, const float* x, int quad, float* cost,
                              float* grad, float* metrics, float* terms, int* err, cudaStream_t st);
// Fused descent: gathers rows idx (or all when idx == nullptr) of x_src (ld_src), runs k_lin
// linear and k_quad quadratic steps, writes x_dst (SoA [4B][m]), the final quadratic cost and
// the satisfying flag (and metrics when non-null).
cudaError_t launch_place_descend(const Scalars& sc, DevTables t, int m, const float* x_src, int ld_src, const int* idx,
                                 float* x_dst, int k_lin, int k_quad, float* cost, int* sat, float* metrics, int* err,
                                 cudaStream_t st);
// k smallest of n costs by (cost, index), ascending.  n <= 32768, k <= 8192.
cudaError_t launch_topk(const float* cost, int n, int k, int* idx, float* cost_out, cudaStream_t st);
size_t topk_smem_bytes(int n, int k);

// Masked selection: cost_masked[i] = sat[i] ? cost[i] : NaN; count of satisfying -> *n_sat.
cudaError_t launch_mask_costs(const float* cost, const int* sat, int n, float* cost_masked, int* n_sat, cudaStream_t st);

// Gather rows of a SoA [nv][ld_src] array into AoS [k][nv]: out[r][v] = src[v][idx[r]].
cudaError_t launch_gather_soa_to_aos(const float* src, int ld_src, int nv, const int* idx, int k, float* out,
                                     cudaStream_t st);

}  // namespace spasm
